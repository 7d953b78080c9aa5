// adjoint.cu -- the estimate of Eq. (11) as a linear map of the signal at a fixed
// recovered support, and its adjoint (the transpose of filter -> bin -> bucket FFT ->
// Eq. (11)), for gradients through the transform.
//
// With the support S and, per coordinate i, the hashes l_r(i), l_i(i) whose values the
// componentwise median selected (Section II-B), the output is real-linear in x:
//   Re y_i = Re v_{l_r(i)}(i),  Im y_i = Im v_{l_i(i)}(i),
//   v_l(i) = C_l(i) Pz_l[j_l(i)],  Pz_l = DFT_B(z_l),  z_l[r] = sum_{a = r mod B} c_l(a) x[a],
// where C_l(i) is the phase and inverse gain of Eq. (11) and c_l(a) the permuted,
// modulated window tap of sample a (the binning's coefficient).  For a real loss with
// gradient g_i = dL/dRe y_i + i dL/dIm y_i, the gradient with respect to x is
//   g_x[a] = sum_l conj(c_l(a) F_l[a mod B]),  F_l = DFT_B(Q_l),
//   Q_l[j] = sum_{i: l_r(i) = l, j_l(i) = j} Re g_i C_l(i) - i sum_{i: l_i(i) = l, ...} Im g_i C_l(i)
// (conjugating twice turns the inverse DFT of the transpose into the forward one).
#include <string.h>

#include "devmath.cuh"

namespace atsfft {

struct EstArgs {
    const int64_t *loc;
    const uint8_t *msel;
    int64_t count;
    const HashParam *est;    // the L_est estimation hashes
    int L_est;
    int logn, logB;
    const float *rgain_b;
    const float2 *phase;
    int phase_s;
};

// y_i = (Re v_{l_r}(i), Im v_{l_i}(i)) from the estimation spectra Pz ([L_est][B]).
__global__ void k_est_apply(const EstArgs E, const float2 *__restrict__ Pz, float2 *out)
{
    const int64_t B = (int64_t)1 << E.logB;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < E.count;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t coord = (uint64_t)E.loc[i];
        const int lr = E.msel[2 * i], li = E.msel[2 * i + 1];
        int64_t jr, ji;
        const float2 cr = estimate_coef(coord, E.est[lr], 1, E.logn, E.logB, E.rgain_b, E.phase,
                                        E.phase_s, &jr);
        const float2 ci = estimate_coef(coord, E.est[li], 1, E.logn, E.logB, E.rgain_b, E.phase,
                                        E.phase_s, &ji);
        out[i] = make_float2(cmul(Pz[lr * B + jr], cr).x, cmul(Pz[li * B + ji], ci).y);
    }
}

// Q_l (zeroed, [L_est][B]) += the output gradients through Eq. (11).
__global__ void k_adj_scatter(const EstArgs E, const float2 *__restrict__ g, float2 *Q)
{
    const int64_t B = (int64_t)1 << E.logB;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < E.count;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t coord = (uint64_t)E.loc[i];
        const int lr = E.msel[2 * i], li = E.msel[2 * i + 1];
        const float2 gi = g[i];
        int64_t jr, ji;
        const float2 cr = estimate_coef(coord, E.est[lr], 1, E.logn, E.logB, E.rgain_b, E.phase,
                                        E.phase_s, &jr);
        const float2 ci = estimate_coef(coord, E.est[li], 1, E.logn, E.logB, E.rgain_b, E.phase,
                                        E.phase_s, &ji);
        float2 *qr = Q + lr * B + jr, *qi = Q + li * B + ji;
        atomicAdd(&qr->x, gi.x * cr.x);
        atomicAdd(&qr->y, gi.x * cr.y);
        atomicAdd(&qi->x, gi.y * ci.y);    // -i Im(g) C
        atomicAdd(&qi->y, -gi.y * ci.x);
    }
}

// F'_l[r] = F_l[r] S_b (b = the bucket of residue r under hash l), or F_l[r] A D for
// bucket 0, whose only tap is the centre one.
__global__ void k_adj_prep(const HashParam *est, int L_est, int logn, int logB, float cAD,
                           const float2 *__restrict__ F, float2 *Fp)
{
    const int64_t B = (int64_t)1 << logB, total = (int64_t)L_est * B;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int l = (int)(k >> logB);
        const uint32_t r = (uint32_t)(k & (B - 1));
        const uint32_t sinv = (uint32_t)est[l].sinv[0], c0 = 0u - sinv * (uint32_t)est[l].tau[0];
        const uint32_t b = (sinv * r + c0) & (uint32_t)(B - 1);
        const float2 f = F[k];
        Fp[k] = b == 0 ? make_float2(cAD * f.x, cAD * f.y) : cmul(f, bucket_factor(b, logB, logn));
    }
}

// g_x[a] = sum_l conj(tap_l(a) F'_l[a mod B]), tap = f_t R_u of the binning (1 at the
// centre tap of bucket 0, 0 elsewhere in bucket 0 and outside the window).
__global__ void __launch_bounds__(256) k_adj_stream(const HashParam *est, int L_est, int logn,
                                                    int logB, const WindowParam w,
                                                    const float2 *__restrict__ Fp, float2 *gx)
{
    extern __shared__ float2 rot[];   // R_u = (-1)^u exp(i pi u / D), u in [0, 2D), if it fits
    __shared__ uint32_t sh_sinv[kMaxLoops], sh_c0[kMaxLoops];
    const uint32_t n = 1u << logn, mask = n - 1, B = 1u << logB, D = n >> logB;
    const bool table = 2 * D <= kAdjRotMax;
    if (table)
        for (uint32_t u = threadIdx.x; u < 2 * D; u += blockDim.x) {
            float sn, cs;
            sincospif(ldexpf((float)u, -(logn - logB)), &sn, &cs);
            rot[u] = (u & 1) ? make_float2(-cs, -sn) : make_float2(cs, sn);
        }
    if (threadIdx.x < L_est) {
        sh_sinv[threadIdx.x] = (uint32_t)est[threadIdx.x].sinv[0];
        sh_c0[threadIdx.x] = 0u - (uint32_t)est[threadIdx.x].sinv[0] * (uint32_t)est[threadIdx.x].tau[0];
    }
    __syncthreads();
    const uint32_t two_h = 2u * (uint32_t)w.h;
    for (int64_t ai = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; ai < n;
         ai += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t a = (uint32_t)ai, r = a & (B - 1);
        float2 acc = make_float2(0.f, 0.f);
        for (int l = 0; l < L_est; l++) {
            const uint32_t tsh = (sh_sinv[l] * a + sh_c0[l] + (uint32_t)w.h) & mask;
            if (tsh > two_h) continue;
            const int ts = (int)tsh - w.h;            // t = sigma^{-1}(a - tau), signed
            const uint32_t b = (uint32_t)ts & (B - 1);
            float2 tap;
            if (b == 0) {
                if (ts != 0) continue;
                tap = make_float2(1.f, 0.f);
            } else {
                const float tf = (float)ts;
                const float f = fast_exp2(fmaf(-w.k2 * tf, tf, w.log2c)) * fast_rcp(tf);
                const int u = ts >> logB;
                float2 Ru;
                if (table) {
                    Ru = rot[(uint32_t)u & (2 * D - 1)];
                } else {
                    float sn, cs;
                    sincospif(ldexpf((float)u, -(logn - logB)), &sn, &cs);
                    Ru = (u & 1) ? make_float2(-cs, -sn) : make_float2(cs, sn);
                }
                tap = make_float2(f * Ru.x, f * Ru.y);
            }
            const float2 v = cmul(tap, __ldg(&Fp[((int64_t)l << logB) + r]));
            acc.x += v.x;
            acc.y -= v.y;
        }
        gx[a] = acc;
    }
}

static atsfft_status est_args(const atsfft_plan_s *P, int64_t B, const int64_t *d_loc,
                              const uint8_t *d_msel, int64_t count, EstArgs *E, int *b_out)
{
    if (!P || P->ndim != 1 || P->p.precision != 0 || B <= 0 || (B & (B - 1)) || count < 0 ||
        (count > 0 && (!d_loc || !d_msel)))
        return ATSFFT_E_INVALID_ARG;
    int b = 0;
    while (((int64_t)1 << b) < B) b++;
    if (b < P->b0 || b > P->b_hi) return ATSFFT_E_INVALID_ARG;
    E->loc = d_loc;
    E->msel = d_msel;
    E->count = count;
    E->est = P->d_le + P->est_base;
    E->L_est = P->L_est;
    E->logn = P->logn;
    E->logB = b;
    E->rgain_b = P->d_rgain + P->resp_off[b];
    E->phase = P->d_phase;
    E->phase_s = P->phase_s;
    *b_out = b;
    return ATSFFT_OK;
}

}  // namespace atsfft

using namespace atsfft;

extern "C" atsfft_status atsfft_estimate_apply(atsfft_plan_t P, int64_t B, const void *d_u,
                                               const int64_t *d_loc, const uint8_t *d_medsel,
                                               int64_t count, void *d_out, void *stream)
{
    EstArgs E;
    int b = 0;
    atsfft_status st = est_args(P, B, d_loc, d_medsel, count, &E, &b);
    if (st != ATSFFT_OK) return st;
    if (!d_u || (count > 0 && !d_out)) return ATSFFT_E_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (caller_error_pending()) return ATSFFT_E_CUDA;
    // the L_est estimation spectra of u at B, as the transform computes them
    const int chunks = launch_est_bin(P, (const float2 *)d_u, b, s);
    int lb[kMaxLoops], ch[kMaxLoops];
    int64_t in_off[kMaxLoops], out_off[kMaxLoops];
    for (int l = 0; l < P->L_est; l++) {
        lb[l] = b;
        ch[l] = chunks;
        in_off[l] = ((int64_t)l * chunks) << b;
        out_off[l] = (int64_t)l << b;
    }
    launch_bucket_fft_batch(P, P->L_est, lb, ch, in_off, out_off, P->d_part, P->d_z, nullptr,
                            nullptr, s);
    if (count > 0)
        k_est_apply<<<P->num_sms * 4, 256, 0, s>>>(E, P->d_z, (float2 *)d_out);
    return cuda_status(cudaGetLastError());
}

extern "C" atsfft_status atsfft_estimate_adjoint(atsfft_plan_t P, int64_t B, const int64_t *d_loc,
                                                 const uint8_t *d_medsel, int64_t count,
                                                 const void *d_gval, void *d_gx, void *stream)
{
    EstArgs E;
    int b = 0;
    atsfft_status st = est_args(P, B, d_loc, d_medsel, count, &E, &b);
    if (st != ATSFFT_OK) return st;
    if (!d_gx || (count > 0 && !d_gval)) return ATSFFT_E_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (caller_error_pending()) return ATSFFT_E_CUDA;
    const int64_t LB = (int64_t)P->L_est << b;
    float2 *Q = P->d_part, *F = P->d_z;
    cudaError_t e = cudaMemsetAsync(Q, 0, sizeof(float2) * (size_t)LB, s);
    if (e != cudaSuccess) return cuda_status(e);
    if (count > 0) k_adj_scatter<<<P->num_sms * 4, 256, 0, s>>>(E, (const float2 *)d_gval, Q);
    int lb[kMaxLoops], ch[kMaxLoops];
    int64_t off[kMaxLoops];
    for (int l = 0; l < P->L_est; l++) {
        lb[l] = b;
        ch[l] = 1;
        off[l] = (int64_t)l << b;
    }
    launch_bucket_fft_batch(P, P->L_est, lb, ch, off, off, Q, F, nullptr, nullptr, s);
    const WindowParam &w = P->h_win[b];
    k_adj_prep<<<P->num_sms * 4, 256, 0, s>>>(E.est, P->L_est, P->logn, b, w.cA_D, F, Q);
    const size_t smem = 2 * (size_t)(P->n >> b) <= (size_t)kAdjRotMax
                            ? sizeof(float2) * 2 * (size_t)(P->n >> b) : 0;
    cudaFuncSetAttribute((const void *)k_adj_stream, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(sizeof(float2) * kAdjRotMax));
    k_adj_stream<<<P->num_sms * 8, 256, smem, s>>>(E.est, P->L_est, P->logn, b, w, Q,
                                                   (float2 *)d_gx);
    return cuda_status(cudaGetLastError());
}
