/*
 * atsfft_oracle.h -- plain, slow, FP64 CPU oracle for ATSFFT (arXiv 1908.02461).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls, links or
 * includes this code; only tests/, the smoke check and the benchmark's CPU
 * baseline leg may load it.  It shares no code with the CUDA path: the two
 * implement the same readings of the paper independently.
 *
 * Everything is computed in FP64 (complex double) from the complex64 input
 * values widened to FP64.  Each function cites the passage of the paper it
 * follows; where the paper is silent the reading used is stated in place.
 *
 * Conventions (Section II): omega = exp(-2*pi*i/n), unscaled forward DFT,
 * indices mod n, n and B powers of two with B | n.
 */
#ifndef ATSFFT_ORACLE_H
#define ATSFFT_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    ORC_OK = 0,
    ORC_E_INVALID_ARG = 1,
    ORC_E_NOMEM = 2,
    ORC_E_NOT_CONVERGED = 4, /* tuning hit its trial cap; best result returned */
    ORC_E_NOT_SPARSE = 5,    /* B reached its upper limit; result at that B returned */
    ORC_E_CAPACITY = 6       /* output arrays too small; count holds the size needed */
};

/* Parameters of Algorithm 2 plus the readings of what the paper leaves open. */
typedef struct {
    double delta1, delta2;      /* Eq. (14): 0.02, 0.05 */
    double eps1, eps2;          /* Eq. (13)/(14): 0.5, 1.0 (only these keep B a power of 2) */
    int tune_max;               /* cap on tuning trials */
    int loops_loc, loops_est;   /* location / estimation loops (7, 7) */
    double filter_alpha;        /* transition width as a fraction of a half bucket (0.5) */
    double filter_tol;          /* Gaussian tail tolerance (1e-6) */
    double thr_rel, thr_med;    /* local-maximum threshold: max(thr_rel*maxE, thr_med*medianE) */
    double tie_eta;             /* relative band inside which two energies count as tied */
    int b_min_log2, b_max_log2; /* tuning range of B (per axis in 2D); 0 = default */
    int fixed_k;                /* 1: no tuning; B = the smallest power of two with B >= sqrt(n k)
                                   (2D: B^2 >= N sqrt(k)) for k = k_hint, k* = k_hint      */
    int est_reuse_loc;          /* 1: the estimation loops reuse the location hashes
                                   (loops_est <= loops_loc) instead of fresh ones          */
} orc_params;

#define ORC_MAX_TRIALS 64

/* A discrete decision close to its boundary.  An implementation that computes the
 * energies in lower precision (FP32) can only decide differently from this FP64 oracle
 * where a deciding comparison has a relative margin within its rounding error, so a
 * transform can log every such comparison below a chosen band; a test then demands that
 * each difference between the two traces back to a logged one.  Kinds:
 *   THRESHOLD  E_c against the threshold T, for a bucket c that dominates its
 *              neighbours (Section III-A local maxima);
 *   DOMINANCE  the pair (c, m) against the edges of the tie band, where reversing it
 *              changes the outcome (tuning: the count; location: the maxima set);
 *   TOPNUM     a local maximum c against the cutoff band edges V(1 +- eta)
 *              (Algorithm 1 "find num largest");
 *   PIVOT      a bucket c whose selection changes if the logged local-maximum flip of
 *              bucket m (-1: all of the hash's flips at once) happened: the num-th
 *              largest energy moves by a rank and the band fill by a place. */
enum { ORC_DEC_THRESHOLD = 1, ORC_DEC_DOMINANCE = 2, ORC_DEC_TOPNUM = 3, ORC_DEC_PIVOT = 4 };

typedef struct {
    int32_t phase;    /* 0: a tuning trial, 1: a location hash */
    int32_t hash;     /* tuning: log2 B (per axis) of the trial; location: hash index l */
    int32_t kind;     /* ORC_DEC_* */
    int32_t pad;
    int64_t c, m;     /* bucket indices (linear c1 * B + c2 in 2D); m = -1 if unused */
    double margin;    /* relative margin of the comparison (PIVOT: of the flip) */
} orc_decision;

typedef struct {
    int status;
    int64_t B_star;             /* bucket count chosen by the tuning (per axis in 2D) */
    int64_t k_star;             /* detected sparsity: local maxima at B_star */
    int64_t count;              /* number of output coordinates (|I'|) */
    int n_trials;
    int64_t trial_B[ORC_MAX_TRIALS];
    int64_t trial_k[ORC_MAX_TRIALS];
    double trial_r[ORC_MAX_TRIALS];
    double min_margin;          /* smallest relative margin of any outcome-deciding comparison */
} orc_result;

void orc_default_params(orc_params *p);

/* SplitMix64 (Steele, Lea, Flood, OOPSLA 2014): advances *state, returns next word. */
uint64_t orc_splitmix64_next(uint64_t *state);

/* Hash parameters (Def. 1) for hash `index` of `phase` (0 tune, 1 locate, 2 estimate).
 * out = {sigma, tau} (ndim 1) or {sigma1, tau1, sigma2, tau2} (ndim 2); sigma odd. */
void orc_hash_params(uint64_t seed, int phase, int index, int64_t n, int ndim, int64_t *out);

/* Inverse of an odd sigma modulo n (n a power of two). */
int64_t orc_inv_mod(int64_t sigma, int64_t n);

/* Flat window (Section II-A-2, Eqs. (8),(9)) for length n and B buckets.
 * Writes h (support half-width) and s (time-domain Gaussian std); if taps is
 * non-NULL it receives the 2h+1 taps G_{-h..h} (index t+h). */
int orc_filter_taps(int64_t n, int64_t B, double alpha, double tol,
                    int64_t *h_out, double *s_out, double *taps);

/* Frequency response Ghat'(o) = (1/n) sum_t G_t cos(2 pi o t / n) at the half-integer
 * bucket offsets o = j - D/2 + 1/2 (D = n/B), written to resp[j], j in [0, D). */
int orc_filter_response(int64_t n, int64_t B, double alpha, double tol, double *resp);

/* Own radix-2 FFT, forward, unscaled, in place on len complex values (interleaved re,im). */
int orc_fft(double *a, int64_t len);

/* One hash (permute, filter, subsample, B-point DFT) of a 1D signal x (n complex,
 * interleaved FP64) with the hash parameters of (seed, phase, index).
 * Zhat receives B complex values. */
int orc_hash_spectrum_1d(const double *x, int64_t n, int64_t B, uint64_t seed, int phase,
                         int index, double alpha, double tol, double *Zhat);

/* 2D analogue on an N x N row-major image; Zhat receives B*B complex (row-major). */
int orc_hash_spectrum_2d(const double *x, int64_t N, int64_t B, uint64_t seed, int phase,
                         int index, double alpha, double tol, double *Zhat);

/* Local maxima of the bucket energies E (1D: ndim=1, nb=B; 2D: ndim=2, nb=B*B with
 * side B).  Writes ascending bucket indices to list (capacity nb), returns the count.
 * T_out and margin_out (may be NULL) receive the threshold and the smallest margin. */
int64_t orc_local_maxima(const double *E, int64_t side, int ndim, double thr_rel,
                         double thr_med, double eta, int64_t *list, double *T_out,
                         double *margin_out);

/* orc_local_maxima with a choice of what counts as the outcome (mode 0: the number of
 * maxima, as in a tuning trial; 1: which buckets are maxima, as in a location hash) and
 * a log: the comparisons deciding it with a margin below `band` go to rec (capacity
 * cap); *n_rec receives their number (which may exceed cap: then only cap are stored). */
int64_t orc_local_maxima_log(const double *E, int64_t side, int ndim, double thr_rel,
                             double thr_med, double eta, int mode, double band, int64_t *list,
                             double *T_out, double *margin_out, orc_decision *rec, int64_t cap,
                             int64_t *n_rec);

/* The location step of one hash on its energies E, exactly as the transform takes it
 * (local maxima, then the num largest of them, parameters from p, NULL = defaults):
 * the selected buckets (ascending) in sel (capacity: the number of buckets), their
 * number returned (-1 on bad arguments); *margin_out the smallest margin; the near
 * decisions, including the PIVOT consequences of each local-maximum flip, logged as in
 * orc_local_maxima_log (records stamped phase 1, hash 0). */
int64_t orc_location_select_log(const double *E, int64_t side, int ndim, const orc_params *p,
                                int64_t num, double band, int64_t *sel, double *margin_out,
                                orc_decision *rec, int64_t cap, int64_t *n_rec);

/* Bucket h(i) of coordinate i under a hash with this sigma, one axis (Eq. (10) as read
 * here); -1 on bad arguments. */
int64_t orc_bucket_of(int64_t i, int64_t sigma, int64_t n, int64_t B);

/* The "num largest" cutoff of the location step (Algorithm 1) on a list of local maxima:
 * lm holds cnt bucket indices in ascending order, E the energies by bucket.  Writes the
 * kept buckets (ascending) to sel (capacity cnt) and returns how many; -1 for num < 1
 * or cnt < 0. */
int64_t orc_top_num(const double *E, const int64_t *lm, int64_t cnt, int64_t num, double eta,
                    int64_t *sel);

/* Componentwise median of L complex values (interleaved); out = {re, im}. */
int orc_median_componentwise(const double *v, int L, double *out);

/* Eq. (14) branch for counts k_prev -> k_cur: -1 halve, 0 keep, +1 double. */
int orc_controller_branch(int64_t k_prev, int64_t k_cur, double delta1, double delta2);

/* Whole ATSFFT (Algorithm 2 with Algorithm 1's location and estimation steps).
 * x: n complex (interleaved FP64).  loc/val receive up to `capacity` outputs in
 * ascending location order; res receives the tuning trace and status. */
int orc_atsfft_1d(const double *x, int64_t n, int64_t k_hint, const orc_params *p,
                  uint64_t seed, int64_t *loc, double *val, int64_t capacity,
                  orc_result *res);

/* 2D-SFFT/ATSFFT on an N x N image; loc holds linear indices i*N + j. */
int orc_atsfft_2d(const double *x, int64_t N, int64_t k_hint, const orc_params *p,
                  uint64_t seed, int64_t *loc, double *val, int64_t capacity,
                  orc_result *res);

/* orc_atsfft_1d (ndim 1, side = n) or orc_atsfft_2d (ndim 2, side = N) that also logs
 * every outcome-deciding comparison of the tuning trials and the location hashes whose
 * margin lies below `band` (see orc_decision) into rec (capacity cap); *n_rec receives
 * the number of records (only cap are stored when it is larger). */
int orc_atsfft_log(const double *x, int ndim, int64_t side, int64_t k_hint, const orc_params *p,
                   uint64_t seed, int64_t *loc, double *val, int64_t capacity, orc_result *res,
                   double band, orc_decision *rec, int64_t cap, int64_t *n_rec);

/* The loops_est estimates of Eq. (11) (no median) of coordinates loc[0..count) of a 1D
 * signal at B buckets; out: count x loops_est complex values, interleaved (re, im). */
int orc_estimates_1d(const double *x, int64_t n, int64_t B, const orc_params *p, uint64_t seed,
                     const int64_t *loc, int64_t count, double *out);

#ifdef __cplusplus
}
#endif
#endif
