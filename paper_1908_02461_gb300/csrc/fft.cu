// fft.cu -- batched B-point bucket DFTs ("do DFT with length B" in Algorithms 1-2;
// B x B in 2D): Zhat_c = sum_b z_b exp(-2 pi i c b / B), unscaled.
//
// One CTA transforms up to kSmallFFT points in shared memory (radix-2 decimation in
// time, bit-reversed load, table twiddles).  Larger 1D transforms use the four-step
// split B = P1 * P2 (j = j1 + P1 j2, k = k2 + P2 k1):
//   pass 0: Y[j1 + P1 k2] = exp(-2 pi i j1 k2 / B) * sum_j2 z[j1 + P1 j2] w_P2^(j2 k2)
//   pass 1: X[k2 + P2 k1] = sum_j1 Y[j1 + P1 k2] w_P1^(j1 k1).
// 2D is rows (pass 0) then columns (pass 1).  The first pass also sums the binning
// partials over their row chunks.
#include "common.cuh"

namespace atsfft {

struct FftShape {
    int logP;            // transform length
    int ntrans;          // transforms per hash
    int64_t in_es, in_bs, out_es, out_bs;
    int64_t hash_stride; // per-hash stride of both arrays
    int tw_logB;         // >= 0: post-multiply by exp(-2 pi i t k / 2^tw_logB)
    int valid;
};

__device__ FftShape fft_shape(int ndim, int logB, int pass)
{
    FftShape f;
    f.valid = 1;
    f.tw_logB = -1;
    if (ndim == 1) {
        const int64_t B = (int64_t)1 << logB;
        f.hash_stride = B;
        if (logB <= 12) {
            if (pass == 1) { f.valid = 0; return f; }
            f.logP = logB; f.ntrans = 1;
            f.in_es = 1; f.in_bs = B; f.out_es = 1; f.out_bs = B;
        } else {
            const int l1 = logB / 2, l2 = logB - l1;
            const int64_t P1 = (int64_t)1 << l1, P2 = (int64_t)1 << l2;
            if (pass == 0) {
                f.logP = l2; f.ntrans = (int)P1;
                f.in_es = P1; f.in_bs = 1; f.out_es = P1; f.out_bs = 1;
                f.tw_logB = logB;
            } else {
                f.logP = l1; f.ntrans = (int)P2;
                f.in_es = 1; f.in_bs = P1; f.out_es = P2; f.out_bs = 1;
            }
        }
    } else {
        const int64_t B = (int64_t)1 << logB;
        f.hash_stride = B * B;
        f.logP = logB; f.ntrans = (int)B;
        if (pass == 0) { f.in_es = 1; f.in_bs = B; f.out_es = 1; f.out_bs = B; }
        else { f.in_es = B; f.in_bs = 1; f.out_es = B; f.out_bs = 1; }
    }
    return f;
}

// part: chunks x (nh x hash_stride) partial arrays, summed on load (chunk stride
// nh * hash_stride).  Pass 0 reads `part`; 1D four-step pass 0 writes `tmp` and pass 1
// reads it; everything else ends in `fin` (2D pass 1 in place).
__global__ void __launch_bounds__(256) k_fft_pass(int ndim, int pass, const Job *job_dev,
                                                  int logB_static, int nh_static, int chunks_static,
                                                  const float2 *__restrict__ part,
                                                  float2 *tmp, float2 *fin,
                                                  const float2 *__restrict__ tw)
{
    __shared__ float2 sm[kSmallFFT];
    int logB = logB_static, nh = nh_static, chunks = chunks_static;
    if (job_dev) {
        if (!job_dev->active) return;
        logB = job_dev->logB;
        nh = job_dev->nh;
        chunks = job_dev->chunks;
    }
    if (pass == 1) chunks = 1;
    const FftShape f = fft_shape(ndim, logB, pass);
    if (!f.valid) return;
    const bool four_step = ndim == 1 && logB > 12;
    const float2 *in = pass == 0 ? part : (ndim == 1 ? tmp : fin);
    float2 *out = (pass == 0 && four_step) ? tmp : fin;
    const int P = 1 << f.logP;
    const int64_t total = (int64_t)nh * f.ntrans;
    const int64_t chunk_stride = (int64_t)nh * f.hash_stride;
    for (int64_t tr = blockIdx.x; tr < total; tr += gridDim.x) {
        const int h = (int)(tr / f.ntrans);
        const int t = (int)(tr % f.ntrans);
        const float2 *src = in + (int64_t)h * f.hash_stride + (int64_t)t * f.in_bs;
        for (int j = threadIdx.x; j < P; j += blockDim.x) {
            float2 v = src[(int64_t)j * f.in_es];
            for (int c = 1; c < chunks; c++) {
                const float2 w = src[(int64_t)c * chunk_stride + (int64_t)j * f.in_es];
                v.x += w.x;
                v.y += w.y;
            }
            const int r = (int)(__brev((unsigned)j) >> (32 - f.logP));
            sm[f.logP ? r : 0] = v;
        }
        __syncthreads();
        for (int lm = 1; lm <= f.logP; lm++) {
            const int half = 1 << (lm - 1);
            const int twstep = kSmallFFT >> lm;
            for (int k = threadIdx.x; k < P / 2; k += blockDim.x) {
                const int q = k & (half - 1);
                const int i0 = ((k >> (lm - 1)) << lm) + q;
                const int i1 = i0 + half;
                const float2 w = tw[q * twstep];
                const float2 a = sm[i0], b = sm[i1];
                const float2 wb = make_float2(w.x * b.x - w.y * b.y, w.x * b.y + w.y * b.x);
                sm[i0] = make_float2(a.x + wb.x, a.y + wb.y);
                sm[i1] = make_float2(a.x - wb.x, a.y - wb.y);
            }
            __syncthreads();
        }
        float2 *dst = out + (int64_t)h * f.hash_stride + (int64_t)t * f.out_bs;
        for (int k = threadIdx.x; k < P; k += blockDim.x) {
            float2 v = sm[k];
            if (f.tw_logB >= 0) {
                const int64_t Bm = ((int64_t)1 << f.tw_logB) - 1;
                const int64_t m = ((int64_t)t * k) & Bm;
                float s, c;
                sincospif(-ldexpf((float)m, 1 - f.tw_logB), &s, &c);
                v = make_float2(v.x * c - v.y * s, v.x * s + v.y * c);
            }
            dst[(int64_t)k * f.out_es] = v;
        }
        __syncthreads();
    }
}

// part (residue-order partials, chunked) -> spectra in `out` (nh x B or nh x B^2).
// Both passes are always launched; each works out from the job whether it has work.
void launch_bucket_fft(const atsfft_plan_s *P, const Job *job_dev, bool dynamic, int logB_static,
                       int nh_static, const float2 *part, float2 *out, cudaStream_t s)
{
    const Job *jd = dynamic ? job_dev : nullptr;
    const int grid = P->num_sms * 8;
    const int chunks_static = dynamic ? 1 : P->h_tjob[logB_static].chunks;
    const bool two = P->ndim == 2 || (dynamic ? P->b_hi > 12 : logB_static > 12);
    k_fft_pass<<<grid, 256, 0, s>>>(P->ndim, 0, jd, logB_static, nh_static, chunks_static, part,
                                    P->d_fft_tmp, out, P->d_tw);
    if (two)
        k_fft_pass<<<grid, 256, 0, s>>>(P->ndim, 1, jd, logB_static, nh_static, chunks_static,
                                        part, P->d_fft_tmp, out, P->d_tw);
}

}  // namespace atsfft
