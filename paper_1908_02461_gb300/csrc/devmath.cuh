// devmath.cuh -- device helpers shared by the forward estimate (tail.cu), the binning
// (bin.cu) and the adjoint (adjoint.cu), so that the forward map and its transpose use
// the same arithmetic.
#pragma once

#include "common.cuh"

namespace atsfft {

__device__ __forceinline__ float fast_exp2(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float fast_rcp(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// S_b = sin(pi b / B) exp(i pi b / n)
__device__ __forceinline__ float2 bucket_factor(uint32_t b, int logB, int logn)
{
    float s1 = sinpif(ldexpf((float)b, -logB));
    float sc, cc;
    sincospif(ldexpf((float)b, -logn), &sc, &cc);
    return make_float2(s1 * cc, s1 * sc);
}

// Eq. (11) index terms of coordinate i on one axis of a hash (Eq. (10) half-bin reading):
// P-index jP of its bucket, the bucket's phase term kph = jP sigma' tau mod B, the
// offset index into the Ghat' table and m = tau i mod n, all in exact integers.
__device__ __forceinline__ void axis_terms(uint64_t i, const HashParam &hp, int axis, int logn,
                                           int logB, uint64_t &jP, uint64_t &kph, int64_t &oidx,
                                           uint64_t &mtau)
{
    const uint64_t n = 1ull << logn, D = 1ull << (logn - logB), Bm = (1ull << logB) - 1;
    const uint64_t p = ((uint64_t)hp.sigma[axis] * i) & (n - 1);
    const uint64_t q = (2 * p + 1 + D) >> (logn - logB + 1);            // / (2 D)
    const int64_t o2 = (int64_t)(2 * p + 1) - (int64_t)(2 * q * D);   // odd, in (-D, D)
    const uint64_t h = q & Bm;
    const uint64_t sp = (uint64_t)hp.sinv[axis] & Bm;                   // sigma^{-1} mod B
    jP = (sp * h) & Bm;
    kph = (jP * ((uint64_t)hp.tau[axis] & Bm)) & Bm;                    // h sigma' tau mod B
    oidx = (o2 + (int64_t)D - 1) >> 1;                                  // >= 0
    mtau = ((uint64_t)hp.tau[axis] * i) & (n - 1);
}

// exp(2 pi i m / n) for an exact integer m in [0, n): product of the two table parts
// (entries m mod 2^s, then 2^s + m >> s).
__device__ __forceinline__ float2 phase_lookup(uint64_t m, const float2 *tab, int s)
{
    const float2 lo = __ldg(&tab[m & ((1ull << s) - 1)]);
    const float2 hi = __ldg(&tab[(1ull << s) + (m >> s)]);
    return make_float2(lo.x * hi.x - lo.y * hi.y, lo.x * hi.y + lo.y * hi.x);
}

// exp(2 pi i m / n) for m taken mod n (32-bit indices, n <= 2^32).
__device__ __forceinline__ float2 phase_lookup32(uint32_t m, uint32_t nmask, const float2 *tab,
                                                 int s)
{
    m &= nmask;
    const float2 lo = __ldg(&tab[m & ((1u << s) - 1)]);
    const float2 hi = __ldg(&tab[(1u << s) + (m >> s)]);
    return make_float2(lo.x * hi.x - lo.y * hi.y, lo.x * hi.y + lo.y * hi.x);
}

// R_u = (-1)^u exp(i pi u / D), D = n / B: exp(i pi u / D) = exp(2 pi i (u B / 2) / n).
__device__ __forceinline__ float2 rot_factor(int u, int logB, uint32_t nmask, const float2 *tab,
                                             int s)
{
    const float2 r = phase_lookup32((uint32_t)u << (logB - 1), nmask, tab, s);
    return (u & 1) ? make_float2(-r.x, -r.y) : r;
}

// S_b = sin(pi b / B) exp(i pi b / n) from the same table: sin(pi b' / B) is the imaginary
// part of exp(2 pi i (b' D / 2) / n) with b' = min(b, B - b) (an angle in [0, pi/2], so
// no cancellation), and exp(i pi b / n) = exp(2 pi i floor(b / 2) / n) times
// half = exp(i pi / n) when b is odd.
__device__ __forceinline__ float2 bucket_factor_tab(uint32_t b, int logB, int logn,
                                                    const float2 *tab, int s, float2 half)
{
    const uint32_t B = 1u << logB, nmask = (1u << logn) - 1;
    const uint32_t bp = b <= B / 2 ? b : B - b;
    const float s1 = phase_lookup32(bp << (logn - logB - 1), nmask, tab, s).y;
    float2 e = phase_lookup32(b >> 1, nmask, tab, s);
    if (b & 1) e = cmul(e, half);
    return make_float2(s1 * e.x, s1 * e.y);
}

// Eq. (11) as a linear functional of the hash's P-order spectrum: the estimate of
// coordinate `coord` (1D index, or i * N + j in 2D) is Pz[*idx] * C.
__device__ __forceinline__ float2 estimate_coef(uint64_t coord, const HashParam &hp, int ndim,
                                                int logn, int b, const float *rgain_b,
                                                const float2 *phase, int phase_s, int64_t *idx)
{
    const uint64_t n = 1ull << logn, D = 1ull << (logn - b);
    uint64_t jP, kph, m, kang;
    int64_t oi;
    float rg;
    if (ndim == 1) {
        axis_terms(coord, hp, 0, logn, b, jP, kph, oi, m);
        *idx = (int64_t)jP;
        rg = __ldg(&rgain_b[oi]);
        kang = (kph * D + n - m) & (n - 1);
    } else {
        const uint64_t i = coord >> logn, j = coord & (n - 1);
        uint64_t jP2, kph2, m2;
        int64_t oi2;
        axis_terms(i, hp, 0, logn, b, jP, kph, oi, m);
        axis_terms(j, hp, 1, logn, b, jP2, kph2, oi2, m2);
        *idx = (int64_t)((jP << b) | jP2);
        rg = __ldg(&rgain_b[oi]) * __ldg(&rgain_b[oi2]);
        kang = ((kph + kph2) * D + 2 * n - m - m2) & (n - 1);
    }
    const float2 w = phase_lookup(kang, phase, phase_s);
    return make_float2(w.x * rg, w.y * rg);
}

// Unnormalised tap T_t = exp(-t^2/(2 s^2)) * box(t), box(0) = D, box(t) = sin(pi t/B)/(pi t/n),
// with sin(pi t / B) reduced exactly in integers.
__device__ __forceinline__ double window_term(int64_t t, int64_t n, int logB, double s)
{
    int64_t B = (int64_t)1 << logB;
    double env = exp(-((double)t * (double)t) / (2.0 * s * s));
    if (t == 0) return env * (double)(n >> logB);
    int64_t r = t % (2 * B);
    if (r < 0) r += 2 * B;
    double sn = (r == 0 || r == B) ? 0.0 : sinpi((double)r / (double)B);
    return env * sn / (M_PI * (double)t / (double)n);
}

}  // namespace atsfft
