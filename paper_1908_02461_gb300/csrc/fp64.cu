// fp64.cu -- the FP64 precision path (1D and 2D): the transform locates in FP32 on a
// rounded copy of the complex128 input (the same kernels and decisions as the FP32 path),
// then the estimation stage runs in FP64 from the complex128 input: the L_est estimation
// hashes at B* (B* x B* in 2D) are binned with FP64 taps (Eqs. (8), (9), Lemma 2; in 2D
// the separable window of Section II-A-2), transformed by an FP64 radix-2 Stockham FFT in
// global memory (2D: rows, a transpose, rows, a transpose back), and Eq. (11) is
// evaluated with the phase exp(2 pi i m / N) of the exact integer m (2D:
// m = tau1 i + tau2 j mod N) in FP64 and the FP64 window gain (2D: the product of the two
// axes' gains), followed by the componentwise median.  GB300 runs FP64 at 1/64 of the
// FP32 rate: this path is for accuracy (values to ~1e-12 of the FP64 oracle), not speed.
#include "devmath.cuh"

namespace atsfft {

// complex128 -> complex64 (round to nearest) for the FP32 location stages.
__global__ void k_to_f32(const double2 *__restrict__ x, int64_t n, float2 *y)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        y[i] = make_float2((float)x[i].x, (float)x[i].y);
}

__device__ __forceinline__ double2 zmul(double2 a, double2 b)
{
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Binning of the estimation hashes at B* in FP64, warp per (hash, bucket): bucket b
// collects the taps t = b + u B, |t| <= h, as A T_t exp(i pi t / n) x[(sigma t + tau) mod n]
// (T_t the unnormalised window tap), stored at the bucket's residue r = (sigma b + tau) mod B.
__global__ void k_bin64(const double2 *__restrict__ x, int logn, const HashParam *est, int L,
                        const WindowParam *win, const Job *job, double2 *out)
{
    if (!job->active) return;
    const int logB = job->logB;
    const uint64_t n = 1ull << logn, mask = n - 1, B = 1ull << logB;
    const WindowParam w = win[logB];
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t total = (int64_t)L << logB;
    for (int64_t wid = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); wid < total;
         wid += warps) {
        const int l = (int)(wid >> logB);
        const int64_t b = wid & (int64_t)(B - 1);
        const uint64_t sig = (uint64_t)est[l].sigma[0], tau = (uint64_t)est[l].tau[0];
        const int64_t u_lo = -((w.h + b) >> logB), u_hi = (w.h - b) >> logB;
        double2 acc = make_double2(0.0, 0.0);
        for (int64_t u = u_lo + lane; u <= u_hi; u += 32) {
            const int64_t t = b + u * (int64_t)B;
            const double g = w.A * window_term(t, (int64_t)n, logB, w.s);
            double sn, cs;
            sincospi((double)t / (double)n, &sn, &cs);
            const double2 v = x[(sig * (uint64_t)t + tau) & mask];
            const double2 tap = make_double2(g * cs, g * sn);
            const double2 p = zmul(tap, v);
            acc.x += p.x;
            acc.y += p.y;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
            acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
        }
        if (lane == 0) out[((int64_t)l << logB) + (int64_t)((sig * (uint64_t)b + tau) & (B - 1))] = acc;
    }
}

// 2D: the modulated window taps of the B* of the job, one axis (the window is the same on
// both): wt[t + h] = A T_t exp(i pi t / N) for |t| <= h (T_t the unnormalised tap).
__global__ void k_wtab64(int logn, const WindowParam *win, const Job *job, double2 *wt)
{
    if (!job->active) return;
    const int logB = job->logB;
    const int64_t n = (int64_t)1 << logn;
    const WindowParam w = win[logB];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= 2 * (int64_t)w.h;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = i - w.h;
        const double g = w.A * window_term(t, n, logB, w.s);
        double sn, cs;
        sincospi((double)t / (double)n, &sn, &cs);
        wt[i] = make_double2(g * cs, g * sn);
    }
}

// 2D binning in FP64, warp per (hash, bucket (b1, b2)): bucket (b1, b2) collects the tap
// pairs t1 = b1 + u1 B, t2 = b2 + u2 B (|t1|, |t2| <= h) as
// wt[t1] wt[t2] x[(sigma1 t1 + tau1) mod N][(sigma2 t2 + tau2) mod N], stored at the
// bucket's residues r = (sigma b + tau) mod B on each axis (row-major B x B per hash).
__global__ void k_bin64_2d(const double2 *__restrict__ x, int logn, const HashParam *est, int L,
                           const WindowParam *win, const Job *job, const double2 *__restrict__ wt,
                           double2 *out)
{
    if (!job->active) return;
    const int logB = job->logB;
    const uint64_t N = 1ull << logn, mask = N - 1, B = 1ull << logB;
    const int h = win[logB].h;
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t total = (int64_t)L << (2 * logB);
    for (int64_t wid = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); wid < total;
         wid += warps) {
        const int l = (int)(wid >> (2 * logB));
        const int64_t b1 = (wid >> logB) & (int64_t)(B - 1), b2 = wid & (int64_t)(B - 1);
        const HashParam hp = est[l];
        const int64_t lo1 = -((h + b1) >> logB), n1 = ((h - b1) >> logB) - lo1 + 1;
        const int64_t lo2 = -((h + b2) >> logB), n2 = ((h - b2) >> logB) - lo2 + 1;
        double2 acc = make_double2(0.0, 0.0);
        for (int64_t q = lane; q < n1 * n2; q += 32) {
            const int64_t t1 = b1 + (lo1 + q / n2) * (int64_t)B;
            const int64_t t2 = b2 + (lo2 + q % n2) * (int64_t)B;
            const uint64_t a1 = ((uint64_t)hp.sigma[0] * (uint64_t)t1 + hp.tau[0]) & mask;
            const uint64_t a2 = ((uint64_t)hp.sigma[1] * (uint64_t)t2 + hp.tau[1]) & mask;
            const double2 g = zmul(wt[t1 + h], wt[t2 + h]);
            const double2 p = zmul(g, x[a1 * N + a2]);
            acc.x += p.x;
            acc.y += p.y;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
            acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
        }
        if (lane == 0) {
            const uint64_t r1 = ((uint64_t)hp.sigma[0] * (uint64_t)b1 + hp.tau[0]) & (B - 1);
            const uint64_t r2 = ((uint64_t)hp.sigma[1] * (uint64_t)b2 + hp.tau[1]) & (B - 1);
            out[((int64_t)l << (2 * logB)) + (int64_t)((r1 << logB) | r2)] = acc;
        }
    }
}

// 2D: y[l][c][r] = x[l][r][c] for the L blocks of B* x B*; phase 0 reads the buffer that
// holds the row transforms (A for even log2 B*, B for odd) and writes the other, phase 1
// reads B and writes A (see launch_estimate_fp64).
__global__ void k_transpose64(const Job *job, int L, int phase, const double2 *bufA, double2 *bufB)
{
    if (!job->active) return;
    const int logB = job->logB;
    const bool even = (logB & 1) == 0;
    const double2 *x = phase == 0 ? (even ? bufA : bufB) : bufB;
    double2 *y = phase == 0 ? (double2 *)(even ? bufB : bufA) : (double2 *)bufA;
    const int64_t B = (int64_t)1 << logB, total = (int64_t)L << (2 * logB);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t l = i >> (2 * logB), r = (i >> logB) & (B - 1), c = i & (B - 1);
        y[(l << (2 * logB)) + (c << logB) + r] = x[i];
    }
}

// tw[m] = exp(-2 pi i m / B*), m < B*/2.
__global__ void k_tw64(const Job *job, double2 *tw)
{
    if (!job->active) return;
    const int logB = job->logB;
    const int64_t half = (int64_t)1 << (logB - 1);
    for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < half;
         m += (int64_t)gridDim.x * blockDim.x) {
        double sn, cs;
        sincospi(-2.0 * (double)m / (double)(2 * half), &sn, &cs);
        tw[m] = make_double2(cs, sn);
    }
}

// One radix-2 Stockham stage (sub-transform length 2 ns -> 4 ns... ns = 2^stage) of the
// L DFTs of length B* = 2^logB: y[(j / ns) 2 ns + j mod ns (+ ns)] = x[j] +/- w x[j + B/2],
// w = exp(-2 pi i (j mod ns) / (2 ns)).  After logB stages y = DFT(x) in natural order.
// The buffers: 1D (phase -1), and 2D phase 0 (the row transforms of the binned blocks),
// start from bufA; 2D phase 1 (the rows of the transposed blocks) starts from the buffer
// the first transpose wrote (B for even log2 B*, A for odd).  Stage s reads the start
// buffer for even s and the other for odd s.
__global__ void k_fft64_stage(const Job *job, int L, int stage, int phase,
                              const double2 *__restrict__ tw, double2 *bufA, double2 *bufB)
{
    if (!job->active || stage >= job->logB) return;
    const int logB = job->logB;
    double2 *start = phase == 1 && (logB & 1) == 0 ? bufB : bufA;
    double2 *other = start == bufA ? bufB : bufA;
    const double2 *x = (stage & 1) ? other : start;
    double2 *y = (stage & 1) ? start : other;
    const int64_t B = (int64_t)1 << logB, halfB = B >> 1, ns = (int64_t)1 << stage;
    const int64_t total = (int64_t)L * halfB * (phase >= 0 ? B : 1);   // 2D: L B rows
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t h = k >> (logB - 1), j = k & (halfB - 1);
        const double2 *xh = x + (h << logB);
        double2 *yh = y + (h << logB);
        const int64_t q = j & (ns - 1);
        const double2 a = xh[j], b = zmul(tw[q << (logB - 1 - stage)], xh[j + halfB]);
        const int64_t o = ((j - q) << 1) + q;
        yh[o] = make_double2(a.x + b.x, a.y + b.y);
        yh[o + ns] = make_double2(a.x - b.x, a.y - b.y);
    }
}

// Eq. (11) in FP64 for each kept coordinate and estimation hash (a group of grp lanes per
// coordinate, lane l = hash l), then the componentwise median (element floor(L/2),
// equal values ordered by hash index) into val[p].
__global__ void k_est64(const ExecState *state, const Job *job, const int64_t *loc,
                        int64_t capacity, const HashParam *est, int L, int grp, int ndim, int logn,
                        const double *resp, RespOffsets ro, const double2 *spec_even,
                        const double2 *spec_odd, double2 *val)
{
    if (!job->active || state->empty) return;
    const int b = job->logB;
    const int64_t cnt = state->count < capacity ? state->count : capacity;
    // the buffer that holds the DFT: 1D, the Stockham result (A for even log2 B*); 2D, A
    const double2 *Pz = (ndim == 1 && (b & 1)) ? spec_odd : spec_even;
    const uint64_t n = 1ull << logn, D = 1ull << (logn - b);
    const int lane = threadIdx.x & 31, gl = lane & (grp - 1);
    const int per_warp = 32 / grp;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t base = warp * per_warp; base < cnt; base += nwarps * per_warp) {
        const int64_t s = base + lane / grp;
        const bool valid = s < cnt;
        double2 v = make_double2(0.0, 0.0);
        if (valid && gl < L) {
            uint64_t jP, kph, m, kang;
            int64_t oi, idx;
            double g;
            if (ndim == 1) {
                axis_terms((uint64_t)loc[s], est[gl], 0, logn, b, jP, kph, oi, m);
                kang = (kph * D + n - m) & (n - 1);
                g = resp[ro.off[b] + oi];
                idx = ((int64_t)gl << b) + (int64_t)jP;
            } else {
                const uint64_t i = (uint64_t)loc[s] >> logn, j = (uint64_t)loc[s] & (n - 1);
                uint64_t jP2, kph2, m2;
                int64_t oi2;
                axis_terms(i, est[gl], 0, logn, b, jP, kph, oi, m);
                axis_terms(j, est[gl], 1, logn, b, jP2, kph2, oi2, m2);
                kang = ((kph + kph2) * D + 2 * n - m - m2) & (n - 1);
                g = resp[ro.off[b] + oi] * resp[ro.off[b] + oi2];
                idx = ((int64_t)gl << (2 * b)) + (int64_t)((jP << b) | jP2);
            }
            double sn, cs;
            sincospi(2.0 * (double)kang / (double)n, &sn, &cs);
            const double2 pv = Pz[idx];
            v = make_double2((pv.x * cs - pv.y * sn) / g, (pv.x * sn + pv.y * cs) / g);
        }
        int rr = 0, ri = 0;
        for (int c = 0; c < L; c++) {
            const double xr = __shfl_sync(0xffffffffu, v.x, c, grp);
            const double xi = __shfl_sync(0xffffffffu, v.y, c, grp);
            rr += xr < v.x || (xr == v.x && c < gl);
            ri += xi < v.y || (xi == v.y && c < gl);
        }
        if (valid && gl < L) {
            if (rr == L / 2) val[s].x = v.x;
            if (ri == L / 2) val[s].y = v.y;
        }
    }
}

void launch_to_f32(const atsfft_plan_s *P, const void *d_x, cudaStream_t s)
{
    k_to_f32<<<P->num_sms * 4, 256, 0, s>>>((const double2 *)d_x, P->ncoord, P->d_x32);
    count_launch(P);
}

void launch_estimate_fp64(const atsfft_plan_s *P, const void *d_x, const int64_t *d_loc,
                          void *d_val, int64_t capacity, cudaStream_t s)
{
    const Job *job = &P->d_state->job;
    const HashParam *est = P->d_le + P->est_base;
    const int L = P->L_est;
    double2 *bufA = P->d_f64a, *bufB = P->d_f64b;
    if (P->ndim == 1) {
        k_bin64<<<P->num_sms * 8, 256, 0, s>>>((const double2 *)d_x, P->logn, est, L, P->d_win,
                                               job, bufA);
        k_tw64<<<P->num_sms, 256, 0, s>>>(job, P->d_tw64);
        count_launch(P, 2);
        // stage p reads buffer p % 2 and writes the other; the result of logB stages is in
        // buffer logB % 2 (A for even, B for odd)
        for (int stage = 0; stage < P->b_hi; stage++) {
            k_fft64_stage<<<P->num_sms * 8, 256, 0, s>>>(job, L, stage, -1, P->d_tw64, bufA, bufB);
            count_launch(P);
        }
    } else {
        // taps, binning into A, rows (the result in A for even log2 B*, B for odd), transpose
        // into the other, rows again (the result in B either way), transpose back into A
        k_wtab64<<<P->num_sms, 256, 0, s>>>(P->logn, P->d_win, job, P->d_wtab64);
        k_bin64_2d<<<P->num_sms * 8, 256, 0, s>>>((const double2 *)d_x, P->logn, est, L, P->d_win,
                                                  job, P->d_wtab64, bufA);
        k_tw64<<<P->num_sms, 256, 0, s>>>(job, P->d_tw64);
        count_launch(P, 3);
        for (int phase = 0; phase < 2; phase++) {
            for (int stage = 0; stage < P->b_hi; stage++) {
                k_fft64_stage<<<P->num_sms * 8, 256, 0, s>>>(job, L, stage, phase, P->d_tw64, bufA,
                                                             bufB);
                count_launch(P);
            }
            k_transpose64<<<P->num_sms * 8, 256, 0, s>>>(job, L, phase, bufA, bufB);
            count_launch(P);
        }
    }
    if (capacity > 0) {
        RespOffsets ro;
        for (int b = 0; b < kMaxLogB; b++) ro.off[b] = P->resp_off[b];
        int grp = 1;
        while (grp < L) grp *= 2;
        k_est64<<<P->num_sms * 4, 256, 0, s>>>(P->d_state, job, d_loc, capacity, est, L, grp,
                                               P->ndim, P->logn, P->d_resp, ro, bufA, bufB,
                                               (double2 *)d_val);
        count_launch(P);
    }
}

}  // namespace atsfft
