// probe.cu -- atsfft_mufu_probe: the measured rate of the two special-function
// operations the residue-stream binning spends on every (sample, hash) pair.
//
// Each tap of the flat window (Section II-A-2: Gaussian envelope times the sampled box
// car) costs the binning one exp2 and one reciprocal on the multi-function unit.  This
// kernel issues nothing else of consequence: every thread runs kChains independent
// chains, each iteration one ex2.approx and one rcp.approx per chain with a single FMA
// or add feeding each, so that the issue slots stay mostly free and the MUFU pipe is
// the limit.  Its rate (operations per second, timed with CUDA events) is the ALU peak
// the benchmark reports the binning against.
#include "devmath.cuh"

namespace atsfft {

constexpr int kChains = 8;

static __device__ float g_probe_sink;   // written only if the chains went negative (never)

__global__ void __launch_bounds__(256) k_mufu_probe(int iters, float seed)
{
    float a[kChains], r[kChains];
#pragma unroll
    for (int c = 0; c < kChains; c++) {
        a[c] = -(float)(threadIdx.x + c) * 1e-3f * seed;
        r[c] = 1.0f + (float)c * seed;
    }
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int c = 0; c < kChains; c++) {
            a[c] = fast_exp2(fmaf(a[c], -0.5f, -0.25f));   // stays in (0, 1]
            r[c] = fast_rcp(r[c] + 1.0f);                  // stays in (0.5, 1]
        }
    }
    float acc = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; c++) acc += a[c] + r[c];
    if (acc < 0.f) g_probe_sink = acc;   // keeps the chains live; every term is positive
}

}  // namespace atsfft

using namespace atsfft;

extern "C" atsfft_status atsfft_mufu_probe(int64_t iters, double *h_ops_per_s, void *stream)
{
    if (!h_ops_per_s || iters < 1 || iters > (1 << 24)) return ATSFFT_E_INVALID_ARG;
    if (caller_error_pending()) return ATSFFT_E_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_status(e);
    const int blocks = sms * 8;   // 2048 threads per SM
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float ms = 0.f;
    if (e == cudaSuccess) {
        k_mufu_probe<<<blocks, 256, 0, s>>>((int)iters / 8 + 1, 1.0f);   // warm-up
        cudaEventRecord(e0, s);
        k_mufu_probe<<<blocks, 256, 0, s>>>((int)iters, 1.0f);
        cudaEventRecord(e1, s);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_status(e);
    if (!(ms > 0.f)) return ATSFFT_E_CUDA;
    const double ops = 2.0 * kChains * (double)iters * (double)blocks * 256.0;
    *h_ops_per_s = ops / (ms * 1e-3);
    return ATSFFT_OK;
}
