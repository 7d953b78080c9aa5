/*
 * atsfft_oracle.c -- plain FP64 CPU oracle for ATSFFT (arXiv 1908.02461).
 *
 * TEST INFRASTRUCTURE ONLY (see atsfft_oracle.h).  Deliberately simple:
 * explicit loops in the order the paper states the steps, library calls only
 * for exp/sin/cos/sqrt/qsort, no blocking or fusion.
 *
 * Readings of points the paper leaves open (each also noted where it is used):
 *  - 1D is one axis of the separable 2D method (Section II restricted to one index).
 *  - Hash parameters: fresh (sigma, tau) per hash from SplitMix64.
 *  - Flat window: continuous box of one bucket width D = n/B bins convolved with a
 *    Gaussian (Eqs. (8),(9)); time taps = Gaussian envelope x sampled sinc, applied
 *    with the modulation exp(i pi t/n) that moves the pass band by half a bin, so
 *    bucket c is centred at permuted frequency c*D - 1/2, the middle of the D
 *    frequencies it collects.
 *  - Hash h(i) = round((sigma*i mod n + 1/2) / D) mod B and offset
 *    o(i) = sigma*i mod n + 1/2 - h(i)*D in (-D/2, D/2) (Eq. (10) read per axis).
 *  - Local maximum: energy above max(thr_rel*maxE, thr_med*medianE) and dominating
 *    every cyclic neighbour (2 in 1D, 8 in 2D); energies within a relative band
 *    tie_eta count as tied and the tie goes to the cyclically later bucket.
 *  - Tuning: B doubles (Eq. (14) last branch) while r >= delta2; it stops at the
 *    first B with r < delta2 (keep branch, or halve branch whose B/2 was already
 *    evaluated); tuning hash at B uses index log2(B).
 *  - Location: L_loc hashes at B*, top num = k* local maxima, vote; keep
 *    coordinates with votes >= ceil(L_loc/2) (Section II-B).
 *  - Estimation: L_est fresh hashes at B*, Eq. (11), componentwise median.
 */
#include "atsfft_oracle.h"

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

typedef double complex cplx;

/* ------------------------------------------------------------------------- */
/* small helpers                                                              */
/* ------------------------------------------------------------------------- */

static int is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }

static int ilog2(int64_t v)
{
    int r = 0;
    while ((int64_t)1 << r < v) r++;
    return r;
}

static int64_t emod(int64_t a, int64_t m)
{
    int64_t r = a % m;
    return r < 0 ? r + m : r;
}

/* (a * b) mod n for 0 <= a, b < n <= 2^31, exact. */
static int64_t mulmod(int64_t a, int64_t b, int64_t n)
{
    return (int64_t)(((uint64_t)a * (uint64_t)b) % (uint64_t)n);
}

void orc_default_params(orc_params *p)
{
    p->delta1 = 0.02;  /* Eq. (14) */
    p->delta2 = 0.05;
    p->eps1 = 0.5;
    p->eps2 = 1.0;
    p->tune_max = 32;
    p->loops_loc = 7;
    p->loops_est = 7;
    p->filter_alpha = 0.5;
    p->filter_tol = 1e-6;
    p->thr_rel = 1e-3;
    p->thr_med = 20.0;
    p->tie_eta = 1e-2;
    p->b_min_log2 = 0;
    p->b_max_log2 = 0;
    p->fixed_k = 0;
    p->est_reuse_loc = 0;
}

/* ------------------------------------------------------------------------- */
/* Random spectrum permutation parameters (Def. 1)                            */
/* ------------------------------------------------------------------------- */

/* SplitMix64, as published by Steele, Lea and Flood (2014). */
uint64_t orc_splitmix64_next(uint64_t *state)
{
    uint64_t z = (*state += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Def. 1: sigma invertible mod n (odd, since n is a power of two), tau in [n].
 * Each hash draws its own pair from a SplitMix64 stream keyed by (seed, phase, index). */
void orc_hash_params(uint64_t seed, int phase, int index, int64_t n, int ndim, int64_t *out)
{
    uint64_t st = seed ^ ((uint64_t)(phase + 1) << 56) ^ ((uint64_t)(uint32_t)index << 32);
    uint64_t mask = (uint64_t)n - 1;
    for (int d = 0; d < ndim; d++) {
        out[2 * d + 0] = (int64_t)((orc_splitmix64_next(&st) & mask) | 1);
        out[2 * d + 1] = (int64_t)(orc_splitmix64_next(&st) & mask);
    }
}

/* sigma^{-1} mod n by the Newton (Hensel) step x <- x (2 - sigma x) mod 2^64, which
 * doubles the number of correct low bits each time; x = sigma is already correct to
 * 3 bits for odd sigma, so six steps cover 64 bits. */
int64_t orc_inv_mod(int64_t sigma, int64_t n)
{
    uint64_t s = (uint64_t)sigma, x = s;
    for (int it = 0; it < 6; it++) x = x * (2 - s * x);
    return (int64_t)(x & ((uint64_t)n - 1));
}

/* ------------------------------------------------------------------------- */
/* Flat window (Section II-A-2)                                               */
/* ------------------------------------------------------------------------- */

/* Window design for length n and B buckets (bucket width D = n/B bins):
 *   box car of width D in frequency (Eq. (8)) convolved with a Gaussian (Eq. (9))
 *   whose tail falls to `tol` at alpha*D/2 from the box edge.  In time this is
 *   G_t = A * exp(-t^2 / (2 s^2)) * sin(pi t / B) / (pi t / n),  G_0 = A * D,
 *   with s = B q / (pi alpha), q = sqrt(2 ln(1/tol)), support |t| <= h = ceil(s q).
 *   If h would exceed n/2 - 1 the support is clamped there and s shrunk to h/q so
 *   that the envelope still reaches `tol` at the support edge.
 *   A normalises sum_t G_t = n, so that Ghat'(0) = 1.  */
static void window_shape(int64_t n, int64_t B, double alpha, double tol, int64_t *h, double *s)
{
    double q = sqrt(2.0 * log(1.0 / tol));
    double ss = (double)B * q / (M_PI * alpha);
    double hh = ceil(ss * q);
    int64_t hmax = n / 2 - 1;
    if (hh > (double)hmax) {
        *h = hmax;
        *s = (double)hmax / q;
    } else {
        *h = (int64_t)hh;
        *s = ss;
    }
}

/* sin(pi t / B) with the argument reduced exactly in integers (period 2B). */
static double sin_pi_t_over_B(int64_t t, int64_t B)
{
    int64_t r = emod(t, 2 * B);
    if (r == 0 || r == B) return 0.0;
    return sin(M_PI * (double)r / (double)B);
}

int orc_filter_taps(int64_t n, int64_t B, double alpha, double tol,
                    int64_t *h_out, double *s_out, double *taps)
{
    if (!is_pow2(n) || !is_pow2(B) || B > n || alpha <= 0 || tol <= 0 || tol >= 1)
        return ORC_E_INVALID_ARG;
    int64_t h;
    double s;
    window_shape(n, B, alpha, tol, &h, &s);
    if (h_out) *h_out = h;
    if (s_out) *s_out = s;
    if (!taps) return ORC_OK;
    double D = (double)(n / B);
    double sum = 0.0;
    for (int64_t t = -h; t <= h; t++) {
        double env = exp(-((double)t * (double)t) / (2.0 * s * s));
        double box = (t == 0) ? D : sin_pi_t_over_B(t, B) / (M_PI * (double)t / (double)n);
        taps[t + h] = env * box;
        sum += taps[t + h];
    }
    double A = (double)n / sum;
    for (int64_t t = -h; t <= h; t++) taps[t + h] *= A;
    return ORC_OK;
}

/* Ghat'(o) = (1/n) sum_{t=-h}^{h} G_t cos(2 pi o t / n): the gain the filter applies
 * to a coefficient at offset o from its bucket centre (the divisor in Eq. (11)).
 * Offsets are half-integers o = j - D/2 + 1/2, j in [0, D); resp[j] = Ghat'(o). */
int orc_filter_response(int64_t n, int64_t B, double alpha, double tol, double *resp)
{
    int64_t h;
    double s;
    int st = orc_filter_taps(n, B, alpha, tol, &h, &s, NULL);
    if (st) return st;
    double *taps = (double *)malloc(sizeof(double) * (size_t)(2 * h + 1));
    if (!taps) return ORC_E_NOMEM;
    orc_filter_taps(n, B, alpha, tol, &h, &s, taps);
    int64_t D = n / B;
    for (int64_t j = 0; j < D; j++) {
        int64_t o2 = 2 * j - D + 1; /* 2*o, an odd integer */
        double acc = 0.0;
        for (int64_t t = -h; t <= h; t++) {
            int64_t m = emod(o2 * t, 2 * n); /* cos(2 pi o t/n) = cos(pi m/n) */
            acc += taps[t + h] * cos(M_PI * (double)m / (double)n);
        }
        resp[j] = acc / (double)n;
    }
    free(taps);
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* DFT                                                                        */
/* ------------------------------------------------------------------------- */

/* Iterative radix-2 decimation-in-time FFT of the unscaled forward DFT
 * Zhat_c = sum_b z_b exp(-2 pi i c b / len).  Twiddles are evaluated directly
 * (not by recurrence) from the exact fraction j/len. */
int orc_fft(double *a_, int64_t len)
{
    if (!is_pow2(len)) return ORC_E_INVALID_ARG;
    cplx *a = (cplx *)a_;
    int lg = ilog2(len);
    for (int64_t i = 0; i < len; i++) {
        int64_t r = 0;
        for (int b = 0; b < lg; b++)
            if (i & ((int64_t)1 << b)) r |= (int64_t)1 << (lg - 1 - b);
        if (r > i) {
            cplx t = a[i];
            a[i] = a[r];
            a[r] = t;
        }
    }
    for (int64_t m = 2; m <= len; m *= 2) {
        for (int64_t j = 0; j < m / 2; j++) {
            double ang = -2.0 * M_PI * (double)j / (double)m;
            cplx w = cos(ang) + I * sin(ang);
            for (int64_t k = j; k < len; k += m) {
                cplx u = a[k], v = w * a[k + m / 2];
                a[k] = u + v;
                a[k + m / 2] = u - v;
            }
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Hash function: permute, filter, subsample, B-point DFT (Section II-A)      */
/* ------------------------------------------------------------------------- */

typedef struct {
    int64_t h;
    double *taps; /* 2h+1 */
} window_t;

static int window_make(window_t *w, int64_t n, int64_t B, double alpha, double tol)
{
    double s;
    int st = orc_filter_taps(n, B, alpha, tol, &w->h, &s, NULL);
    if (st) return st;
    w->taps = (double *)malloc(sizeof(double) * (size_t)(2 * w->h + 1));
    if (!w->taps) return ORC_E_NOMEM;
    return orc_filter_taps(n, B, alpha, tol, &w->h, &s, w->taps);
}

/* Half-bin modulation exp(i pi t / n) of tap t (|t| < n/2): shifts the window's pass
 * band so that bucket c is centred at c*D - 1/2. */
static cplx half_bin(int64_t t, int64_t n)
{
    double ang = M_PI * (double)t / (double)n;
    return cos(ang) + I * sin(ang);
}

/* z_b = sum_{t in [-h,h], t = b mod B} G_t exp(i pi t/n) x[(sigma t + tau) mod n]
 * (Def. 1, window, Lemma 2 aliasing), then Zhat = DFT_B(z). */
static void hash_1d(const cplx *x, int64_t n, int64_t B, int64_t sigma, int64_t tau,
                    const window_t *w, cplx *Z)
{
    for (int64_t b = 0; b < B; b++) Z[b] = 0.0;
    for (int64_t t = -w->h; t <= w->h; t++) {
        int64_t a = (mulmod(sigma, emod(t, n), n) + tau) % n;
        Z[emod(t, B)] += w->taps[t + w->h] * half_bin(t, n) * x[a];
    }
    orc_fft((double *)Z, B);
}

/* 2D: z_{b1,b2} = sum G_{t1} G_{t2} exp(i pi (t1 + t2)/N) x[(s1 t1 + tau1) mod N, (s2 t2 + tau2) mod N] over the
 * separable window (Eq. (2), Lemma 2 in 2D), then the B x B DFT (rows, then columns). */
static void hash_2d(const cplx *x, int64_t N, int64_t B, const int64_t *hp,
                    const window_t *w, cplx *Z)
{
    int64_t s1 = hp[0], t1o = hp[1], s2 = hp[2], t2o = hp[3];
    for (int64_t b = 0; b < B * B; b++) Z[b] = 0.0;
    for (int64_t t1 = -w->h; t1 <= w->h; t1++) {
        int64_t a1 = (mulmod(s1, emod(t1, N), N) + t1o) % N;
        int64_t b1 = emod(t1, B);
        cplx g1 = w->taps[t1 + w->h] * half_bin(t1, N);
        for (int64_t t2 = -w->h; t2 <= w->h; t2++) {
            int64_t a2 = (mulmod(s2, emod(t2, N), N) + t2o) % N;
            int64_t b2 = emod(t2, B);
            Z[b1 * B + b2] += g1 * (w->taps[t2 + w->h] * half_bin(t2, N)) * x[a1 * N + a2];
        }
    }
    cplx *line = (cplx *)malloc(sizeof(cplx) * (size_t)B);
    for (int64_t r = 0; r < B; r++) orc_fft((double *)(Z + r * B), B);
    for (int64_t c = 0; c < B; c++) {
        for (int64_t r = 0; r < B; r++) line[r] = Z[r * B + c];
        orc_fft((double *)line, B);
        for (int64_t r = 0; r < B; r++) Z[r * B + c] = line[r];
    }
    free(line);
}

int orc_hash_spectrum_1d(const double *x, int64_t n, int64_t B, uint64_t seed, int phase,
                         int index, double alpha, double tol, double *Zhat)
{
    if (!is_pow2(n) || !is_pow2(B) || B > n) return ORC_E_INVALID_ARG;
    window_t w;
    int st = window_make(&w, n, B, alpha, tol);
    if (st) return st;
    int64_t hp[2];
    orc_hash_params(seed, phase, index, n, 1, hp);
    hash_1d((const cplx *)x, n, B, hp[0], hp[1], &w, (cplx *)Zhat);
    free(w.taps);
    return ORC_OK;
}

int orc_hash_spectrum_2d(const double *x, int64_t N, int64_t B, uint64_t seed, int phase,
                         int index, double alpha, double tol, double *Zhat)
{
    if (!is_pow2(N) || !is_pow2(B) || B > N) return ORC_E_INVALID_ARG;
    window_t w;
    int st = window_make(&w, N, B, alpha, tol);
    if (st) return st;
    int64_t hp[4];
    orc_hash_params(seed, phase, index, N, 2, hp);
    hash_2d((const cplx *)x, N, B, hp, &w, (cplx *)Zhat);
    free(w.taps);
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Local maxima (Section III-A) and decision margins                          */
/* ------------------------------------------------------------------------- */

static int cmp_double(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

static double rel_gap(double a, double b)
{
    double m = fmax(fabs(a), fabs(b));
    return m > 0.0 ? fabs(a - b) / m : INFINITY;
}

/* Log of the outcome-deciding comparisons whose relative margin lies below `band`
 * (see orc_decision): an FP32 implementation can only decide otherwise there. */
typedef struct {
    double band;
    orc_decision *rec;   /* may be NULL: count only */
    int64_t cap, n;      /* n counts every record, also those beyond cap */
    int phase, hash;     /* stamped on each record */
} declog_t;

static void log_decision(declog_t *lg, int kind, int64_t c, int64_t m, double margin)
{
    if (!lg || !(margin < lg->band)) return;
    if (lg->rec && lg->n < lg->cap) {
        orc_decision *d = &lg->rec[lg->n];
        d->phase = lg->phase;
        d->hash = lg->hash;
        d->kind = kind;
        d->pad = 0;
        d->c = c;
        d->m = m;
        d->margin = margin;
    }
    lg->n++;
}

/* Does bucket c dominate its neighbour at displacement (d1, d2) (energy Em)?
 * Strictly larger beyond the relative tie band eta wins.  Inside the band the tie
 * goes to the bucket that is later in cyclic order along the first axis that
 * differs, i.e. c wins iff the neighbour lies before it: d1 < 0, or d1 == 0 and
 * d2 < 0.  This matches the round-half-up hash (Eq. (10)): a coefficient exactly
 * midway between two bucket centres belongs to the later bucket, and there the
 * two energies are equal.  *margin gets the distance from the band edges. */
static int dominates(double Ec, double Em, int d1, int d2, double eta, double *margin)
{
    double g = fmin(rel_gap(Ec, (1.0 + eta) * Em), rel_gap(Em, (1.0 + eta) * Ec));
    if (margin && g < *margin) *margin = g;
    if (Ec > (1.0 + eta) * Em) return 1;
    if (Em > (1.0 + eta) * Ec) return 0;
    return d1 < 0 || (d1 == 0 && d2 < 0);
}

/* Threshold T = max(thr_rel * max E, thr_med * median E), the median being the
 * element of rank floor(nb/2) in ascending order. */
static double energy_threshold(const double *E, int64_t nb, double thr_rel, double thr_med,
                               double *maxE_out)
{
    double *tmp = (double *)malloc(sizeof(double) * (size_t)nb);
    memcpy(tmp, E, sizeof(double) * (size_t)nb);
    qsort(tmp, (size_t)nb, sizeof(double), cmp_double);
    double med = tmp[nb / 2], mx = tmp[nb - 1];
    free(tmp);
    if (maxE_out) *maxE_out = mx;
    return fmax(thr_rel * mx, thr_med * med);
}

/* Neighbours of bucket c on the cyclic grid: 2 in 1D, 8 in 2D (Fig. 5's local maxima
 * read as the cyclic neighbourhood).  Writes linear indices and displacements. */
static int neighbours(int64_t c, int64_t side, int ndim, int64_t *m, int *d1s, int *d2s)
{
    int64_t c1 = ndim == 1 ? 0 : c / side, c2 = ndim == 1 ? c : c % side;
    int cnt = 0;
    for (int d1 = (ndim == 1 ? 0 : -1); d1 <= (ndim == 1 ? 0 : 1); d1++) {
        for (int d2 = -1; d2 <= 1; d2++) {
            if (d1 == 0 && d2 == 0) continue;
            int64_t m1 = emod(c1 + d1, side), m2 = emod(c2 + d2, side);
            m[cnt] = ndim == 1 ? m2 : m1 * side + m2;
            d1s[cnt] = d1;
            d2s[cnt] = d2;
            cnt++;
        }
    }
    return cnt;
}

/* Counted iff above the threshold and dominating every neighbour, where the relation
 * with neighbour `flip_m` (if >= 0) is taken reversed. */
static int counted_with_flip(const double *E, int64_t c, int64_t side, int ndim, double T,
                             double eta, int64_t flip_m)
{
    if (!(E[c] > T)) return 0;
    int64_t m[8];
    int d1[8], d2[8];
    int nn = neighbours(c, side, ndim, m, d1, d2);
    for (int j = 0; j < nn; j++) {
        int d = dominates(E[c], E[m[j]], d1[j], d2[j], eta, NULL);
        if (m[j] == flip_m) d = !d;
        if (!d) return 0;
    }
    return 1;
}

/* mode 0: only the number of maxima matters (tuning); mode 1: which buckets are
 * maxima matters (location).  The margin records only comparisons whose reversal
 * would change that outcome. */
static int64_t local_maxima_mode(const double *E, int64_t side, int ndim, double thr_rel,
                                 double thr_med, double eta, int64_t *list, double *T_out,
                                 double *margin_out, int mode, declog_t *lg)
{
    int64_t nb = ndim == 1 ? side : side * side;
    double maxE;
    double T = energy_threshold(E, nb, thr_rel, thr_med, &maxE);
    double margin = INFINITY;
    int64_t cnt = 0;
    for (int64_t c = 0; c < nb; c++) {
        int64_t m[8];
        int d1[8], d2[8];
        int nn = neighbours(c, side, ndim, m, d1, d2);
        int dom = 1;
        for (int j = 0; j < nn; j++)
            if (!dominates(E[c], E[m[j]], d1[j], d2[j], eta, NULL)) dom = 0;
        int is_max = dom && E[c] > T;
        /* threshold comparison decides c's status when c dominates its neighbours */
        if (dom && T > 0.0) {
            double g = rel_gap(E[c], T);
            if (g < margin) margin = g;
            log_decision(lg, ORC_DEC_THRESHOLD, c, -1, g);
        }
        /* pair comparisons, each unordered pair once */
        for (int j = 0; j < nn; j++) {
            if (m[j] < c) continue;
            int before_c = is_max, before_m = counted_with_flip(E, m[j], side, ndim, T, eta, -1);
            int after_c = counted_with_flip(E, c, side, ndim, T, eta, m[j]);
            int after_m = counted_with_flip(E, m[j], side, ndim, T, eta, c);
            int changes = mode == 0 ? (before_c + before_m != after_c + after_m)
                                    : (before_c != after_c || before_m != after_m);
            if (changes) {
                double g = INFINITY;
                dominates(E[c], E[m[j]], d1[j], d2[j], eta, &g);
                if (g < margin) margin = g;
                log_decision(lg, ORC_DEC_DOMINANCE, c, m[j], g);
            }
        }
        if (is_max) {
            if (list) list[cnt] = c;
            cnt++;
        }
    }
    if (T_out) *T_out = T;
    if (margin_out) *margin_out = margin;
    return cnt;
}

int64_t orc_local_maxima(const double *E, int64_t side, int ndim, double thr_rel,
                         double thr_med, double eta, int64_t *list, double *T_out,
                         double *margin_out)
{
    return local_maxima_mode(E, side, ndim, thr_rel, thr_med, eta, list, T_out, margin_out, 1,
                             NULL);
}

int64_t orc_local_maxima_log(const double *E, int64_t side, int ndim, double thr_rel,
                             double thr_med, double eta, int mode, double band, int64_t *list,
                             double *T_out, double *margin_out, orc_decision *rec, int64_t cap,
                             int64_t *n_rec)
{
    declog_t lg = {band, rec, cap, 0, 0, 0};
    int64_t cnt = local_maxima_mode(E, side, ndim, thr_rel, thr_med, eta, list, T_out, margin_out,
                                    mode ? 1 : 0, &lg);
    if (n_rec) *n_rec = lg.n;
    return cnt;
}

/* ------------------------------------------------------------------------- */
/* Tuning controller (Eqs. (12)-(14), Algorithm 2)                            */
/* ------------------------------------------------------------------------- */

/* Eq. (12) r = |1 - k_cur/k_prev| and the branch of Eq. (14).  A zero count on
 * either side is read as an unbounded change (r = inf). */
static double change_ratio(int64_t k_prev, int64_t k_cur)
{
    if (k_prev == 0 || k_cur == 0) return INFINITY;
    return fabs(1.0 - (double)k_cur / (double)k_prev);
}

int orc_controller_branch(int64_t k_prev, int64_t k_cur, double delta1, double delta2)
{
    double r = change_ratio(k_prev, k_cur);
    if (r >= delta2) return 1;
    if (r >= delta1) return 0;
    return -1;
}

/* ------------------------------------------------------------------------- */
/* Cutoff: the num largest local maxima                                       */
/* ------------------------------------------------------------------------- */

typedef struct {
    double e;
    int64_t c;
} ec_t;

static int cmp_ec_desc(const void *a, const void *b)
{
    const ec_t *x = (const ec_t *)a, *y = (const ec_t *)b;
    if (x->e != y->e) return x->e < y->e ? 1 : -1;
    return (x->c > y->c) - (x->c < y->c);
}

static int cmp_i64(const void *a, const void *b)
{
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return (x > y) - (x < y);
}

/* Keep the num largest of the cnt local maxima (Algorithm 1 "find num largest",
 * Algorithm 2 "find num local maximum").  Pivot V = num-th largest energy; every
 * maximum above V(1+eta) is kept, and the rest are filled from those within
 * [V(1-eta), V(1+eta)] in ascending index order.  Result in sel (ascending). */
static int64_t top_num(const double *E, const int64_t *lm, int64_t cnt, int64_t num,
                       int64_t *sel, double eta, double *margin, declog_t *lg)
{
    if (cnt <= num) {
        memcpy(sel, lm, sizeof(int64_t) * (size_t)cnt);
        return cnt;
    }
    ec_t *v = (ec_t *)malloc(sizeof(ec_t) * (size_t)cnt);
    for (int64_t i = 0; i < cnt; i++) v[i] = (ec_t){E[lm[i]], lm[i]};
    qsort(v, (size_t)cnt, sizeof(ec_t), cmp_ec_desc);
    double V = v[num - 1].e, hi = V * (1.0 + eta), lo = V * (1.0 - eta);
    int64_t ns = 0;
    for (int64_t i = 0; i < cnt; i++) {
        double e = E[lm[i]];
        double g = fmin(rel_gap(e, hi), rel_gap(e, lo));
        if (g < *margin) *margin = g;
        log_decision(lg, ORC_DEC_TOPNUM, lm[i], -1, g);
        if (e > hi) sel[ns++] = lm[i];
    }
    for (int64_t i = 0; i < cnt && ns < num; i++) { /* lm is ascending */
        double e = E[lm[i]];
        if (e <= hi && e >= lo) sel[ns++] = lm[i];
    }
    free(v);
    qsort(sel, (size_t)ns, sizeof(int64_t), cmp_i64);
    return ns;
}

int64_t orc_top_num(const double *E, const int64_t *lm, int64_t cnt, int64_t num, double eta,
                    int64_t *sel)
{
    if (num < 1 || cnt < 0) return -1;
    double margin = INFINITY;
    return top_num(E, lm, cnt, num, sel, eta, &margin, NULL);
}

/* The location step of one hash on its energies (Algorithm 1: the local maxima, then the
 * num largest of them): the selected buckets, ascending, in sel and their number as the
 * return value; *margin is lowered to the smallest margin of a deciding comparison.
 * With a log, the near decisions are recorded, and for each recorded flip of a local
 * maximum (each alone, and all of them at once) the buckets whose selection that flip
 * would change: a maximum that enters or leaves the list moves the num-th largest
 * energy by one rank and the band fill by one place (ORC_DEC_PIVOT, m = the flipped
 * bucket, or -1 for all at once; margin = the flip's). */
static int64_t location_select(const double *E, int64_t side, int ndim, const orc_params *p,
                               int64_t num, int64_t *lm, int64_t *sel, double *margin,
                               declog_t *lg)
{
    int64_t nb = ndim == 1 ? side : side * side;
    double T = 0.0, marg = INFINITY;
    int64_t first = lg ? lg->n : 0;
    int64_t cnt = local_maxima_mode(E, side, ndim, p->thr_rel, p->thr_med, p->tie_eta, lm, &T,
                                    &marg, 1, lg);
    int64_t nflip = lg ? lg->n - first : 0;
    int64_t ns = top_num(E, lm, cnt, num, sel, p->tie_eta, &marg, lg);
    if (marg < *margin) *margin = marg;
    if (!lg || nflip == 0 || !lg->rec || first + nflip > lg->cap) return ns;

    unsigned char *base = (unsigned char *)calloc((size_t)nb, 1);
    unsigned char *alt = (unsigned char *)malloc((size_t)nb);
    int64_t *lm2 = (int64_t *)malloc(sizeof(int64_t) * (size_t)nb);
    int64_t *sel2 = (int64_t *)malloc(sizeof(int64_t) * (size_t)nb);
    orc_decision *fl = (orc_decision *)malloc(sizeof(orc_decision) * (size_t)nflip);
    memcpy(fl, lg->rec + first, sizeof(orc_decision) * (size_t)nflip);
    for (int64_t i = 0; i < cnt; i++) base[lm[i]] = 1;
    int64_t nalt = nflip > 1 ? nflip + 1 : nflip;
    for (int64_t a = 0; a < nalt; a++) {
        memcpy(alt, base, (size_t)nb);
        int64_t r0 = a < nflip ? a : 0, r1 = a < nflip ? a + 1 : nflip;
        double gmin = INFINITY;
        for (int64_t r = r0; r < r1; r++) {
            const orc_decision *d = &fl[r];
            if (d->margin < gmin) gmin = d->margin;
            if (d->kind == ORC_DEC_THRESHOLD) {
                alt[d->c] = !base[d->c];
            } else {
                alt[d->c] = (unsigned char)counted_with_flip(E, d->c, side, ndim, T, p->tie_eta, d->m);
                alt[d->m] = (unsigned char)counted_with_flip(E, d->m, side, ndim, T, p->tie_eta, d->c);
            }
        }
        int64_t cnt2 = 0;
        for (int64_t c = 0; c < nb; c++)
            if (alt[c]) lm2[cnt2++] = c;
        double dummy = INFINITY;
        int64_t ns2 = top_num(E, lm2, cnt2, num, sel2, p->tie_eta, &dummy, NULL);
        /* both selections are ascending: walk them together */
        int64_t i = 0, j = 0;
        while (i < ns || j < ns2) {
            if (j >= ns2 || (i < ns && sel[i] < sel2[j])) {
                log_decision(lg, ORC_DEC_PIVOT, sel[i++], a < nflip ? fl[a].c : -1, gmin);
            } else if (i >= ns || sel2[j] < sel[i]) {
                log_decision(lg, ORC_DEC_PIVOT, sel2[j++], a < nflip ? fl[a].c : -1, gmin);
            } else {
                i++;
                j++;
            }
        }
    }
    free(base);
    free(alt);
    free(lm2);
    free(sel2);
    free(fl);
    return ns;
}

int64_t orc_location_select_log(const double *E, int64_t side, int ndim, const orc_params *p,
                                int64_t num, double band, int64_t *sel, double *margin_out,
                                orc_decision *rec, int64_t cap, int64_t *n_rec)
{
    orc_params dp;
    if (!p) {
        orc_default_params(&dp);
        p = &dp;
    }
    if (!E || !sel || side < 1 || (ndim != 1 && ndim != 2) || num < 1) return -1;
    int64_t nb = ndim == 1 ? side : side * side;
    int64_t *lm = (int64_t *)malloc(sizeof(int64_t) * (size_t)nb);
    if (!lm) return -1;
    declog_t lg = {band, rec, cap, 0, 1, 0};
    double margin = INFINITY;
    int64_t ns = location_select(E, side, ndim, p, num, lm, sel, &margin, &lg);
    free(lm);
    if (margin_out) *margin_out = margin;
    if (n_rec) *n_rec = lg.n;
    return ns;
}

/* ------------------------------------------------------------------------- */
/* Hash index arithmetic (Eq. (10), offset of Eq. (11))                        */
/* ------------------------------------------------------------------------- */

/* h(i) = round((p + 1/2) / D) mod B with p = sigma i mod n, and twice the offset,
 * o2 = 2 (p + 1/2 - h D), an odd integer in (-D, D).  Bucket c collects exactly the
 * permuted positions p in [c D - D/2, c D + D/2 - 1]. */
static void bucket_of(int64_t i, int64_t sigma, int64_t n, int64_t B, int64_t *h, int64_t *o2)
{
    int64_t D = n / B;
    int64_t p = mulmod(sigma, i, n);
    int64_t q = (2 * p + 1 + D) / (2 * D);
    *o2 = 2 * p + 1 - 2 * q * D;
    *h = q % B;
}

int64_t orc_bucket_of(int64_t i, int64_t sigma, int64_t n, int64_t B)
{
    if (!is_pow2(n) || !is_pow2(B) || B > n || i < 0 || i >= n || sigma < 0 || sigma >= n)
        return -1;
    int64_t h, o2;
    bucket_of(i, sigma, n, B, &h, &o2);
    return h;
}

static int cmp_double_plain(const void *a, const void *b) { return cmp_double(a, b); }

/* Componentwise median over L values (Section II-B "median of the outputs of the L
 * rounds", read per real and imaginary part): element floor(L/2) of each sorted
 * component. */
static cplx median_c(const cplx *v, int L)
{
    double re[64], im[64];
    for (int l = 0; l < L; l++) {
        re[l] = creal(v[l]);
        im[l] = cimag(v[l]);
    }
    qsort(re, (size_t)L, sizeof(double), cmp_double_plain);
    qsort(im, (size_t)L, sizeof(double), cmp_double_plain);
    return re[L / 2] + I * im[L / 2];
}

int orc_median_componentwise(const double *v, int L, double *out)
{
    if (L < 1 || L > 64) return ORC_E_INVALID_ARG;
    cplx m = median_c((const cplx *)v, L);
    out[0] = creal(m);
    out[1] = cimag(m);
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Whole transform                                                            */
/* ------------------------------------------------------------------------- */

static int check_params(const orc_params *p)
{
    if (!(p->delta1 > 0 && p->delta1 < p->delta2 && p->delta2 < 1)) return 0;
    if (p->eps1 != 0.5 || p->eps2 != 1.0) return 0;
    if (p->tune_max < 1 || p->tune_max > ORC_MAX_TRIALS) return 0;
    if (p->loops_loc < 1 || p->loops_loc > 255 || p->loops_est < 1 || p->loops_est > 63) return 0;
    if (!(p->filter_alpha > 0 && p->filter_alpha <= 2)) return 0;
    if (!(p->filter_tol > 0 && p->filter_tol < 1)) return 0;
    if (!(p->thr_rel >= 0 && p->thr_med >= 0 && p->tie_eta >= 0 && p->tie_eta < 1)) return 0;
    if (p->fixed_k != 0 && p->fixed_k != 1) return 0;
    if (p->est_reuse_loc != 0 && p->est_reuse_loc != 1) return 0;
    if (p->est_reuse_loc && p->loops_est > p->loops_loc) return 0;
    return 1;
}

/* Energies |Zhat|^2 of a hash and the local-maximum count at side B. */
typedef struct {
    const cplx *x;
    int64_t n;      /* signal length (1D) or side N (2D) */
    int ndim;
    const orc_params *p;
    uint64_t seed;
} ctx_t;

static int hash_any(const ctx_t *cx, int64_t B, int phase, int index, const window_t *w, cplx *Z)
{
    int64_t hp[4];
    orc_hash_params(cx->seed, phase, index, cx->n, cx->ndim, hp);
    if (cx->ndim == 1)
        hash_1d(cx->x, cx->n, B, hp[0], hp[1], w, Z);
    else
        hash_2d(cx->x, cx->n, B, hp, w, Z);
    return ORC_OK;
}

/* Eq. (11) for estimation hash l (bucket-order spectrum Z at B, filter response resp;
 * with est_reuse_loc the l-th location hash, else the l-th estimation hash):
 * est[s * L + l] = Z[h(i)] omega^{tau i} / Ghat'(o(i)) for each kept coordinate keep[s]
 * (2D: i * N + j, per-axis buckets and gains multiplied). */
static void estimate_hash(const ctx_t *cx, int64_t B, int l, const cplx *Z, const double *resp,
                          const int64_t *keep, int64_t nkeep, cplx *est, int L)
{
    int64_t n = cx->n, D = n / B;
    int ndim = cx->ndim;
    int64_t hp[4];
    orc_hash_params(cx->seed, cx->p->est_reuse_loc ? 1 : 2, l, n, ndim, hp);
    for (int64_t s = 0; s < nkeep; s++) {
        int64_t i = ndim == 1 ? keep[s] : keep[s] / n;
        int64_t j = ndim == 1 ? 0 : keep[s] % n;
        int64_t h1, o1, h2 = 0, o2 = 0;
        bucket_of(i, hp[0], n, B, &h1, &o1);
        int64_t m = mulmod(hp[1], i, n);
        double gain = resp[(o1 + D - 1) / 2];
        int64_t bucket = h1;
        if (ndim == 2) {
            bucket_of(j, hp[2], n, B, &h2, &o2);
            m = (m + mulmod(hp[3], j, n)) % n;
            gain *= resp[(o2 + D - 1) / 2];
            bucket = h1 * B + h2;
        }
        double ang = -2.0 * M_PI * (double)m / (double)n; /* omega^{tau i} */
        cplx ph = cos(ang) + I * sin(ang);
        est[s * L + l] = Z[bucket] * ph / gain;
    }
}

static int atsfft_any(const ctx_t *cx, int64_t k_hint, int64_t *loc, double *val_,
                      int64_t capacity, orc_result *res, declog_t *lg)
{
    const orc_params *p = cx->p;
    int64_t n = cx->n;
    int ndim = cx->ndim;
    int lgn = ilog2(n);
    cplx *val = (cplx *)val_;
    memset(res, 0, sizeof(*res));
    res->min_margin = INFINITY;

    int b_lo = p->b_min_log2 ? p->b_min_log2 : (ndim == 1 ? 4 : 3);
    int b_hi = p->b_max_log2 ? p->b_max_log2 : (ndim == 1 ? lgn - 4 : lgn - 2);
    if (b_lo < 1 || b_hi > lgn - 1 || b_lo > b_hi) return res->status = ORC_E_INVALID_ARG;
    int b0 = b_lo;
    if (k_hint > 0) {
        /* R-INIT: B0 = smallest power of two >= 2 k_hint (1D) or >= sqrt(2 k_hint) per axis. */
        int want = ndim == 1 ? ilog2(2 * k_hint) : (ilog2(2 * k_hint) + 1) / 2;
        if (want > b0) b0 = want;
        if (b0 > b_hi) b0 = b_hi;
    }

    /* ---- tuning (Algorithm 2 loop) ---- */
    int64_t Bmax = (int64_t)1 << b_hi;
    int64_t nbmax = ndim == 1 ? Bmax : Bmax * Bmax;
    cplx *Z = (cplx *)malloc(sizeof(cplx) * (size_t)nbmax);
    double *E = (double *)malloc(sizeof(double) * (size_t)nbmax);
    int64_t *lm = (int64_t *)malloc(sizeof(int64_t) * (size_t)nbmax);
    if (!Z || !E || !lm) {
        free(Z); free(E); free(lm);
        return res->status = ORC_E_NOMEM;
    }

    int status = ORC_OK;
    int b = b0;
    int64_t k_prev = 0, k_cur = 0;
    int zero_signal = 0;
    if (p->fixed_k) {
        /* fixed-k mode (the SFFT setting the tuning replaces): no trials, B from k_hint */
        if (k_hint <= 0) {
            free(Z); free(E); free(lm);
            return res->status = ORC_E_INVALID_ARG;
        }
        int m = ilog2(ndim == 1 ? n * k_hint : n * n * k_hint);   /* ceil(log2) */
        int bf = ndim == 1 ? (m + 1) / 2 : (m + 3) / 4;
        if (bf < b_lo) bf = b_lo;
        if (bf > b_hi) bf = b_hi;
        res->B_star = (int64_t)1 << bf;
        res->k_star = k_hint;
        res->n_trials = 0;
    }
    for (int trial = 0; !p->fixed_k; trial++) {
        int64_t B = (int64_t)1 << b;
        int64_t nb = ndim == 1 ? B : B * B;
        window_t w;
        if (window_make(&w, n, B, p->filter_alpha, p->filter_tol)) {
            status = ORC_E_NOMEM;
            break;
        }
        hash_any(cx, B, 0, b, &w, Z); /* tuning hash at B uses index log2(B) */
        free(w.taps);
        double maxE = 0.0;
        for (int64_t c = 0; c < nb; c++) {
            E[c] = creal(Z[c]) * creal(Z[c]) + cimag(Z[c]) * cimag(Z[c]);
            if (E[c] > maxE) maxE = E[c];
        }
        double marg = INFINITY;
        if (lg) {
            lg->phase = 0;
            lg->hash = b;
        }
        k_cur = maxE > 0.0 ? local_maxima_mode(E, B, ndim, p->thr_rel, p->thr_med, p->tie_eta,
                                               NULL, NULL, &marg, 0, lg)
                           : 0;
        if (marg < res->min_margin) res->min_margin = marg;
        double r = trial == 0 ? NAN : change_ratio(k_prev, k_cur);
        res->trial_B[trial] = B;
        res->trial_k[trial] = k_cur;
        res->trial_r[trial] = r;
        res->n_trials = trial + 1;
        res->B_star = B;
        res->k_star = k_cur;
        if (maxE == 0.0) { /* nothing in the window: the signal is zero there */
            zero_signal = 1;
            break;
        }
        if (trial > 0 && r < p->delta2) break; /* keep branch, or halve onto a visited B */
        if (b == b_hi) {                       /* Eq. (14) asks to double past the limit */
            if (trial > 0) status = ORC_E_NOT_SPARSE;
            break;
        }
        if (trial + 1 >= p->tune_max) {
            status = ORC_E_NOT_CONVERGED;
            break;
        }
        k_prev = k_cur;
        b++;
    }
    if (status == ORC_E_NOMEM) {
        free(Z); free(E); free(lm);
        return res->status = status;
    }

    int64_t B = res->B_star, kstar = res->k_star;
    int64_t D = n / B;
    int64_t nb = ndim == 1 ? B : B * B;
    int64_t ncoord = ndim == 1 ? n : n * n;
    int64_t count = 0;

    if (!zero_signal && kstar > 0) {
        /* ---- location (Algorithm 1 lines "hash, DFT, num largest, reverse hash") ---- */
        window_t w;
        window_make(&w, n, B, p->filter_alpha, p->filter_tol);
        unsigned char *votes = (unsigned char *)calloc((size_t)ncoord, 1);
        int64_t *sel = (int64_t *)malloc(sizeof(int64_t) * (size_t)nb);
        for (int l = 0; l < p->loops_loc; l++) {
            hash_any(cx, B, 1, l, &w, Z);
            for (int64_t c = 0; c < nb; c++)
                E[c] = creal(Z[c]) * creal(Z[c]) + cimag(Z[c]) * cimag(Z[c]);
            if (lg) {
                lg->phase = 1;
                lg->hash = l;
            }
            int64_t ns = location_select(E, B, ndim, p, kstar, lm, sel, &res->min_margin, lg);
            int64_t hp[4];
            orc_hash_params(cx->seed, 1, l, n, ndim, hp);
            int64_t si1 = orc_inv_mod(hp[0], n);
            int64_t si2 = ndim == 2 ? orc_inv_mod(hp[2], n) : 0;
            /* reverse hash: every coordinate whose permuted position rounds to the bucket */
            for (int64_t s = 0; s < ns; s++) {
                int64_t c = sel[s];
                if (ndim == 1) {
                    for (int64_t q = 0; q < D; q++) {
                        int64_t pp = emod(c * D - D / 2 + q, n);
                        votes[mulmod(si1, pp, n)]++;
                    }
                } else {
                    int64_t c1 = c / B, c2 = c % B;
                    for (int64_t q1 = 0; q1 < D; q1++) {
                        int64_t i = mulmod(si1, emod(c1 * D - D / 2 + q1, n), n);
                        for (int64_t q2 = 0; q2 < D; q2++) {
                            int64_t j = mulmod(si2, emod(c2 * D - D / 2 + q2, n), n);
                            votes[i * n + j]++;
                        }
                    }
                }
            }
        }
        free(sel);
        /* keep coordinates that occurred in at least half of the location loops */
        int need = (p->loops_loc + 1) / 2;
        int64_t nkeep = 0;
        for (int64_t i = 0; i < ncoord; i++) nkeep += votes[i] >= need;
        int64_t *keep = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nkeep ? nkeep : 1));
        nkeep = 0;
        for (int64_t i = 0; i < ncoord; i++)
            if (votes[i] >= need) keep[nkeep++] = i;
        free(votes);

        /* ---- estimation (Eq. (11), median over loops) ---- */
        int L = p->loops_est;
        double *resp = (double *)malloc(sizeof(double) * (size_t)D);
        orc_filter_response(n, B, p->filter_alpha, p->filter_tol, resp);
        cplx *est = (cplx *)malloc(sizeof(cplx) * (size_t)(nkeep ? nkeep : 1) * (size_t)L);
        for (int l = 0; l < L; l++) {
            hash_any(cx, B, p->est_reuse_loc ? 1 : 2, l, &w, Z);
            estimate_hash(cx, B, l, Z, resp, keep, nkeep, est, L);
        }
        free(resp);
        free(w.taps);
        count = nkeep;
        for (int64_t s = 0; s < nkeep && s < capacity; s++) {
            loc[s] = keep[s];
            val[s] = median_c(est + s * L, L);
        }
        free(est);
        free(keep);
    }
    free(Z);
    free(E);
    free(lm);
    res->count = count;
    if (count > capacity && status == ORC_OK) status = ORC_E_CAPACITY;
    res->status = status;
    return status;
}

int orc_atsfft_1d(const double *x, int64_t n, int64_t k_hint, const orc_params *p,
                  uint64_t seed, int64_t *loc, double *val, int64_t capacity,
                  orc_result *res)
{
    orc_params dp;
    if (!p) {
        orc_default_params(&dp);
        p = &dp;
    }
    if (!x || !res || !is_pow2(n) || n < 256 || n > ((int64_t)1 << 31) || capacity < 0 ||
        !check_params(p)) {
        if (res) res->status = ORC_E_INVALID_ARG;
        return ORC_E_INVALID_ARG;
    }
    ctx_t cx = {(const cplx *)x, n, 1, p, seed};
    return atsfft_any(&cx, k_hint, loc, val, capacity, res, NULL);
}

int orc_atsfft_2d(const double *x, int64_t N, int64_t k_hint, const orc_params *p,
                  uint64_t seed, int64_t *loc, double *val, int64_t capacity,
                  orc_result *res)
{
    orc_params dp;
    if (!p) {
        orc_default_params(&dp);
        p = &dp;
    }
    if (!x || !res || !is_pow2(N) || N < 32 || N > ((int64_t)1 << 15) || capacity < 0 ||
        !check_params(p)) {
        if (res) res->status = ORC_E_INVALID_ARG;
        return ORC_E_INVALID_ARG;
    }
    ctx_t cx = {(const cplx *)x, N, 2, p, seed};
    return atsfft_any(&cx, k_hint, loc, val, capacity, res, NULL);
}

int orc_atsfft_log(const double *x, int ndim, int64_t side, int64_t k_hint, const orc_params *p,
                   uint64_t seed, int64_t *loc, double *val, int64_t capacity, orc_result *res,
                   double band, orc_decision *rec, int64_t cap, int64_t *n_rec)
{
    orc_params dp;
    if (!p) {
        orc_default_params(&dp);
        p = &dp;
    }
    int64_t lo = ndim == 1 ? 256 : 32, hi = ndim == 1 ? ((int64_t)1 << 31) : ((int64_t)1 << 15);
    if (!x || !res || (ndim != 1 && ndim != 2) || !is_pow2(side) || side < lo || side > hi ||
        capacity < 0 || cap < 0 || !check_params(p)) {
        if (res) res->status = ORC_E_INVALID_ARG;
        return ORC_E_INVALID_ARG;
    }
    ctx_t cx = {(const cplx *)x, side, ndim, p, seed};
    declog_t lg = {band, rec, cap, 0, 0, 0};
    int st = atsfft_any(&cx, k_hint, loc, val, capacity, res, &lg);
    if (n_rec) *n_rec = lg.n;
    return st;
}

/* The L_est estimates of Eq. (11) of each coordinate loc[0..count) of a 1D signal at B
 * buckets, without the median: out[s * L_est + l] (complex, interleaved) is estimation
 * hash l's value (the support is given, nothing is located). */
int orc_estimates_1d(const double *x, int64_t n, int64_t B, const orc_params *p, uint64_t seed,
                     const int64_t *loc, int64_t count, double *out)
{
    orc_params dp;
    if (!p) {
        orc_default_params(&dp);
        p = &dp;
    }
    if (!x || !out || (count > 0 && !loc) || !is_pow2(n) || !is_pow2(B) || B > n / 2 ||
        count < 0 || !check_params(p))
        return ORC_E_INVALID_ARG;
    for (int64_t s = 0; s < count; s++)
        if (loc[s] < 0 || loc[s] >= n) return ORC_E_INVALID_ARG;
    ctx_t cx = {(const cplx *)x, n, 1, p, seed};
    window_t w;
    if (window_make(&w, n, B, p->filter_alpha, p->filter_tol) != ORC_OK) return ORC_E_NOMEM;
    int64_t D = n / B;
    double *resp = (double *)malloc(sizeof(double) * (size_t)D);
    cplx *Z = (cplx *)malloc(sizeof(cplx) * (size_t)B);
    if (!resp || !Z) {
        free(resp);
        free(Z);
        free(w.taps);
        return ORC_E_NOMEM;
    }
    orc_filter_response(n, B, p->filter_alpha, p->filter_tol, resp);
    for (int l = 0; l < p->loops_est; l++) {
        hash_any(&cx, B, p->est_reuse_loc ? 1 : 2, l, &w, Z);
        estimate_hash(&cx, B, l, Z, resp, loc, count, (cplx *)out, p->loops_est);
    }
    free(resp);
    free(Z);
    free(w.taps);
    return ORC_OK;
}
