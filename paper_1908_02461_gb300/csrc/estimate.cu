// estimate.cu -- coefficient estimation (Eq. (11)) and the median over the estimation
// loops (Section II-B, Algorithm 1 last step), plus the final status words.
//
// For kept coordinate i and estimation hash (sigma, tau) at B* = B buckets (D = n/B):
//   p = sigma i mod n, h = round((p + 1/2)/D) mod B, o = p + 1/2 - h D     (Eq. (10), offset)
//   xhat'_i = Zhat[h] omega^{tau i} / Ghat'(o)                             (Eq. (11))
// with Zhat[h] = P[sigma' h] exp(2 pi i h sigma' tau / B) from the residue-order spectrum.
// Index arithmetic is exact 64-bit integer; the two phases are combined into one angle
// 2 pi k / n with k = ((h sigma' tau mod B) D - tau i) mod n, evaluated in FP64, and the
// product and division are done in FP64.  Median: componentwise, element floor(L/2).
#include "common.cuh"

namespace atsfft {

struct RespOffsets {
    int64_t off[kMaxLogB];
};

__device__ __forceinline__ void axis_terms(uint64_t i, const HashParam &hp, int axis, int logn,
                                           int logB, uint64_t &jP, uint64_t &kph, int64_t &oidx,
                                           uint64_t &mtau)
{
    const uint64_t n = 1ull << logn, D = 1ull << (logn - logB), Bm = (1ull << logB) - 1;
    const uint64_t p = ((uint64_t)hp.sigma[axis] * i) & (n - 1);
    const uint64_t q = (2 * p + 1 + D) / (2 * D);
    const int64_t o2 = (int64_t)(2 * p + 1) - (int64_t)(2 * q * D);   // odd, in (-D, D)
    const uint64_t h = q & Bm;
    const uint64_t sp = (uint64_t)hp.sinv[axis] & Bm;                   // sigma^{-1} mod B
    jP = (sp * h) & Bm;
    kph = ((jP * ((uint64_t)hp.tau[axis] & Bm)) & Bm);                  // h sigma' tau mod B
    oidx = (o2 + (int64_t)D - 1) / 2;
    mtau = ((uint64_t)hp.tau[axis] * i) & (n - 1);
}

__global__ void k_estimate(const int64_t *loc, float2 *val, int64_t capacity,
                           const ExecState *state, const float2 *z, const HashParam *est,
                           int L_loc, int L_est, const double *resp, RespOffsets ro, int ndim,
                           int logn)
{
    if (state->empty) return;
    const int64_t cnt = min(state->count, capacity);
    const int b = state->b_star;
    const uint64_t n = 1ull << logn, D = 1ull << (logn - b);
    const int64_t nb = ndim == 1 ? ((int64_t)1 << b) : ((int64_t)1 << (2 * b));
    const double *G = resp + ro.off[b];
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < cnt;
         s += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t coord = (uint64_t)loc[s];
        double re[kMaxLoops], im[kMaxLoops];
        for (int l = 0; l < L_est; l++) {
            const HashParam hp = est[L_loc + l];
            const float2 *Pz = z + (int64_t)(L_loc + l) * nb;
            uint64_t jP, kph, m;
            int64_t oi;
            float2 pv;
            double gain;
            uint64_t kang;
            if (ndim == 1) {
                axis_terms(coord, hp, 0, logn, b, jP, kph, oi, m);
                pv = Pz[jP];
                gain = G[oi];
                kang = (kph * D + n - m) & (n - 1);
            } else {
                const uint64_t i = coord >> logn, j = coord & (n - 1);
                uint64_t jP2, kph2, m2;
                int64_t oi2;
                axis_terms(i, hp, 0, logn, b, jP, kph, oi, m);
                axis_terms(j, hp, 1, logn, b, jP2, kph2, oi2, m2);
                pv = Pz[(jP << b) | jP2];
                gain = G[oi] * G[oi2];
                kang = ((kph + kph2) * D + 2 * n - m - m2) & (n - 1);
            }
            double sn, cs;
            sincospi(2.0 * (double)kang / (double)n, &sn, &cs);
            re[l] = ((double)pv.x * cs - (double)pv.y * sn) / gain;
            im[l] = ((double)pv.x * sn + (double)pv.y * cs) / gain;
        }
        // componentwise median: insertion sort of each part
        for (int a = 1; a < L_est; a++) {
            const double r = re[a], q = im[a];
            int k = a - 1;
            while (k >= 0 && re[k] > r) { re[k + 1] = re[k]; k--; }
            re[k + 1] = r;
            k = a - 1;
            while (k >= 0 && im[k] > q) { im[k + 1] = im[k]; k--; }
            im[k + 1] = q;
        }
        val[s] = make_float2((float)re[L_est / 2], (float)im[L_est / 2]);
    }
}

__global__ void k_finalize(const ExecState *state, int64_t capacity, int64_t *d_count,
                           int64_t *d_k, int32_t *d_status)
{
    if (threadIdx.x || blockIdx.x) return;
    int st = state->status;
    const int64_t cnt = state->empty ? 0 : state->count;
    if (cnt > capacity && st == ATSFFT_OK) st = ATSFFT_E_CAPACITY;
    *d_count = cnt;
    *d_k = state->k_star;
    *d_status = st;
}

void launch_estimate(const atsfft_plan_s *P, const int64_t *d_loc, float2 *d_val,
                     int64_t capacity, int64_t *d_count, int64_t *d_k, int32_t *d_status,
                     cudaStream_t s)
{
    RespOffsets ro;
    for (int b = 0; b < kMaxLogB; b++) ro.off[b] = P->resp_off[b];
    count_launch(P, 2);
    k_estimate<<<P->num_sms * 2, 128, 0, s>>>(d_loc, d_val, capacity, P->d_state, P->d_z, P->d_le,
                                              P->L_loc, P->L_est, P->d_resp, ro, P->ndim, P->logn);
    k_finalize<<<1, 32, 0, s>>>(P->d_state, capacity, d_count, d_k, d_status);
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
