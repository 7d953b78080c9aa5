// inspect.cu -- per-exec reset of the device state, and the bucket-order view of one
// hash's spectrum used by the inspection call atsfft_hash_spectrum.
#include "common.cuh"

namespace atsfft {

void launch_reset(const atsfft_plan_s *P, cudaStream_t s)
{
    cudaMemsetAsync(P->d_stats, 0, sizeof(HashStats) * (kMaxLogB + kMaxLoops), s);
    cudaMemsetAsync(P->d_state, 0, sizeof(ExecState), s);
    cudaMemsetAsync(P->d_hist, 0, sizeof(uint32_t) * kHistBins * (kMaxLogB + kMaxLoops), s);
}

// Inspection: Zhat[c] = P[sigma' c] exp(2 pi i c sigma' tau / B) in bucket order.
__global__ void k_unpermute(const float2 *spec, const HashParam *hp_dev, int ndim, int logB,
                            float2 *out)
{
    const HashParam hp = *hp_dev;
    const uint64_t B = 1ull << logB, Bm = B - 1;
    const int64_t nb = ndim == 1 ? (int64_t)B : (int64_t)(B * B);
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nb;
         c += (int64_t)gridDim.x * blockDim.x) {
        uint64_t idx, k;
        if (ndim == 1) {
            const uint64_t sp = hp.sinv[0] & Bm;
            idx = (sp * (uint64_t)c) & Bm;
            k = (idx * (hp.tau[0] & Bm)) & Bm;
        } else {
            const uint64_t c1 = (uint64_t)c >> logB, c2 = (uint64_t)c & Bm;
            const uint64_t j1 = ((hp.sinv[0] & Bm) * c1) & Bm, j2 = ((hp.sinv[1] & Bm) * c2) & Bm;
            idx = (j1 << logB) | j2;
            k = ((j1 * (hp.tau[0] & Bm)) + (j2 * (hp.tau[1] & Bm))) & Bm;
        }
        double sn, cs;
        sincospi(2.0 * (double)k / (double)B, &sn, &cs);
        const float2 v = spec[idx];
        out[c] = make_float2((float)(v.x * cs - v.y * sn), (float)(v.x * sn + v.y * cs));
    }
}

void launch_unpermute(const atsfft_plan_s *P, const float2 *spec, const HashParam *hash_dev,
                      int logB, float2 *out, cudaStream_t s)
{
    count_launch(P);
    k_unpermute<<<P->num_sms * 2, 256, 0, s>>>(spec, hash_dev, P->ndim, logB, out);
}

}  // namespace atsfft
