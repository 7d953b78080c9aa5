// plan.cu -- plan creation: hash permutations (Def. 1), window shapes and tables
// (Section II-A-2), scratch allocation.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <new>

#include "devmath.cuh"

namespace atsfft {

atsfft_status cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return ATSFFT_OK;
    if (e == cudaErrorMemoryAllocation) return ATSFFT_E_NOMEM;
    return ATSFFT_E_CUDA;
}

// SplitMix64 (Steele, Lea and Flood, 2014).
uint64_t splitmix64_next(uint64_t *state)
{
    uint64_t z = (*state += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// Inverse of odd sigma modulo the power of two n: Newton steps y <- y (2 - sigma y)
// each double the number of correct low bits (y = sigma is right to 3 bits).
uint32_t inv_mod_pow2(uint32_t sigma, int64_t n)
{
    uint64_t y = sigma;
    for (int i = 0; i < 6; i++) y = y * (2 - (uint64_t)sigma * y);
    return (uint32_t)(y & (uint64_t)(n - 1));
}

// Hash `index` of `phase` (0 tuning, 1 location, 2 estimation): one SplitMix64 stream
// keyed by (seed, phase, index) draws sigma (odd) and tau per axis.
void hash_params_for(uint64_t seed, int phase, int index, int64_t n, int ndim, HashParam *out)
{
    uint64_t st = seed ^ ((uint64_t)(phase + 1) << 56) ^ ((uint64_t)(uint32_t)index << 32);
    uint64_t mask = (uint64_t)n - 1;
    memset(out, 0, sizeof(*out));
    for (int d = 0; d < ndim; d++) {
        out->sigma[d] = (uint32_t)((splitmix64_next(&st) & mask) | 1u);
        out->tau[d] = (uint32_t)(splitmix64_next(&st) & mask);
        out->sinv[d] = inv_mod_pow2(out->sigma[d], n);
    }
}

// Window of B = 2^logB buckets over length n: box car of one bucket width convolved
// with a Gaussian reaching `tol` at alpha * D / 2 beyond the box edge.  Time-domain
// std s = B q / (pi alpha), q = sqrt(2 ln(1/tol)), support h = ceil(s q); when that
// exceeds n/2 - 1 the support is clamped and s shrunk to h / q.
WindowParam window_shape(int64_t n, int logB, double alpha, double tol)
{
    WindowParam w;
    double B = ldexp(1.0, logB);
    double q = sqrt(2.0 * log(1.0 / tol));
    double s = B * q / (M_PI * alpha);
    double hh = ceil(s * q);
    int64_t hmax = n / 2 - 1;
    if (hh > (double)hmax) {
        w.h = (int32_t)hmax;
        w.s = (double)hmax / q;
    } else {
        w.h = (int32_t)hh;
        w.s = s;
    }
    w.k2 = (float)(1.4426950408889634 / (2.0 * w.s * w.s));
    w.A = 0.0;
    w.log2c = 0.0f;
    w.cA_D = 0.0f;
    return w;
}

// Residue-stream binning when the window covers at least a fifth of the signal and
// the per-bucket rotation table fits in shared memory; the gather form (a group of
// lanes per bucket walking its taps) otherwise.
Job make_job(const atsfft_plan_s *P, int logB, int nh)
{
    Job j;
    memset(&j, 0, sizeof(j));
    j.logB = logB;
    j.nh = nh;
    j.active = 1;
    int64_t w = 2 * (int64_t)P->h_win[logB].h + 1;
    int64_t D = P->n >> logB;
    if (P->ndim == 1) {
        j.stream = (5 * w >= P->n && D <= 4096) ? 1 : 0;
        if (j.stream) {
            // at least 2^16 items (residues x row chunks), spread evenly over the SMs; every
            // further chunk adds B partial sums per hash for the bucket FFT to read
            int64_t B = (int64_t)1 << logB;
            int64_t rows = P->n >> logB;
            int64_t chunks = ((int64_t)1 << 16) / B;
            if (chunks < 1) chunks = 1;
            if (chunks > rows) chunks = rows;
            j.chunks = (int32_t)chunks;
        } else {
            j.chunks = 1;
        }
    } else {
        // 2D: residue-stream over (r1, r2) once the window covers a fifth of each axis
        j.stream = (5 * w >= P->n) ? 1 : 0;
        int64_t B2 = (int64_t)1 << (2 * logB);
        int64_t rows = D;  // row blocks per residue pair along axis 1
        int64_t chunks = j.stream ? ((int64_t)1 << 18) / B2 : 1;
        if (chunks < 1) chunks = 1;
        if (chunks > rows) chunks = rows;
        j.chunks = (int32_t)chunks;
    }
    return j;
}

// ---- plan-time window tables (FP64) ---------------------------------------------


// Partial sums over a chunk of t in [0, h] of w_t T_t cos(pi o2 t / n) (w_0 = 1, else 2)
// for every half-integer offset o2 = 2j - D + 1, j in [0, D), and o2 = 0 (j = D, the
// normalising sum).  The cosine advances by an exact FP64 rotation from an exactly
// reduced start.
constexpr int kRespThreads = 128;
constexpr int kRespTile = 128;
constexpr int64_t kRespChunk = 8192;

__global__ void k_window_partial(int64_t n, int logB, double s, int h, double *partial,
                                 int nchunks)
{
    __shared__ double terms[kRespTile];
    int64_t D = n >> logB;
    int64_t j = (int64_t)blockIdx.x * kRespThreads + threadIdx.x;
    int chunk = blockIdx.y;
    int64_t t0 = (int64_t)chunk * kRespChunk;
    int64_t t1 = t0 + kRespChunk - 1;
    if (t1 > h) t1 = h;
    int64_t o2 = (j < D) ? 2 * j - D + 1 : 0;
    // start angle pi * o2 * t0 / n, reduced mod 2n exactly
    int64_t m = (o2 * t0) % (2 * n);
    if (m < 0) m += 2 * n;
    double c, sn;
    sincospi((double)m / (double)n, &sn, &c);
    double cr, sr;
    sincospi((double)o2 / (double)n, &sr, &cr);
    double acc = 0.0;
    for (int64_t tb = t0; tb <= t1; tb += kRespTile) {
        __syncthreads();
        int64_t tt = tb + threadIdx.x;
        terms[threadIdx.x] = (tt <= t1) ? window_term(tt, n, logB, s) * (tt == 0 ? 1.0 : 2.0) : 0.0;
        __syncthreads();
        int cnt = (int)((t1 - tb + 1) < kRespTile ? (t1 - tb + 1) : kRespTile);
        for (int k = 0; k < cnt; k++) {
            acc += terms[k] * c;
            double c2 = c * cr - sn * sr;
            sn = sn * cr + c * sr;
            c = c2;
        }
    }
    if (j <= D) partial[j * nchunks + chunk] = acc;
}

// Sums the chunk partials in order; resp[j] = S(o2_j) / S(0).
__global__ void k_window_finish(int64_t D, const double *partial, int nchunks, double *resp,
                                double *S0_out)
{
    __shared__ double S0;
    if (threadIdx.x == 0) {
        double s0 = 0.0;
        for (int c = 0; c < nchunks; c++) s0 += partial[D * nchunks + c];
        S0 = s0;
        *S0_out = s0;
    }
    __syncthreads();
    for (int64_t j = threadIdx.x; j < D; j += blockDim.x) {
        double acc = 0.0;
        for (int c = 0; c < nchunks; c++) acc += partial[j * nchunks + c];
        resp[j] = acc / S0;
    }
}

// Reciprocal gains 1 / Ghat'(o) in FP32 for the estimates of Eq. (11).
__global__ void k_recip_gain(const double *resp, int64_t count, float *rgain)
{
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < count;
         j += (int64_t)gridDim.x * blockDim.x)
        rgain[j] = (float)(1.0 / resp[j]);
}

// Phase factors exp(2 pi i m / n) for an exact integer m in [0, n): m = hi 2^s + lo,
// table entries lo < 2^s, then 2^s + hi for hi < n / 2^s, each from an exact fraction
// in FP64 and rounded to FP32; the product of the two is within 2 FP32 ulps.
__global__ void k_phase_table(int logn, int s_bits, float2 *tab)
{
    const int64_t nlo = (int64_t)1 << s_bits, nhi = ((int64_t)1 << logn) >> s_bits;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nlo + nhi;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t m = j < nlo ? j : (j - nlo) << s_bits;
        double sn, cs;
        sincospi(ldexp(2.0 * (double)m, -logn), &sn, &cs);
        tab[j] = make_float2((float)cs, (float)sn);
    }
}

// Twiddles from exact fractions, for the shared-memory FFT: entry j < 4096 is
// exp(-2 pi i j / 4096); entry 4096 + j is exp(-2 pi i j / 2^24), the fine factor of
// the four-step twiddle exp(-2 pi i m / B) = coarse(m >> (b - 12)) fine(low bits of m).
__global__ void k_twiddles(float2 *tw)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < kTwEntries) {
        double s, c;
        if (j < kSmallFFT)
            sincospi(-2.0 * (double)j / (double)kSmallFFT, &s, &c);
        else
            sincospi(-2.0 * (double)(j - kSmallFFT) / 16777216.0, &s, &c);
        tw[j] = make_float2((float)c, (float)s);
    }
}

}  // namespace atsfft

using namespace atsfft;

extern "C" void atsfft_default_params(atsfft_params *p)
{
    if (!p) return;
    p->delta1 = 0.02;
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
    p->coop_blocks_per_sm = 0;
    p->tune_stages = 3;
    p->fixed_k = 0;
    p->est_reuse_loc = 0;
    p->precision = 0;
    p->coop_sms = 0;
}

extern "C" const char *atsfft_status_string(atsfft_status s)
{
    switch (s) {
    case ATSFFT_OK: return "ok";
    case ATSFFT_E_INVALID_ARG: return "invalid argument";
    case ATSFFT_E_NOMEM: return "out of memory";
    case ATSFFT_E_CUDA: return "CUDA error";
    case ATSFFT_E_NOT_CONVERGED: return "tuning did not converge within tune_max trials";
    case ATSFFT_E_NOT_SPARSE: return "signal not sparse enough for the largest B";
    case ATSFFT_E_CAPACITY: return "output capacity too small";
    }
    return "unknown status";
}

static bool params_ok(const atsfft_params *p)
{
    if (!(p->delta1 > 0 && p->delta1 < p->delta2 && p->delta2 < 1)) return false;
    if (p->eps1 != 0.5 || p->eps2 != 1.0) return false;
    if (p->tune_max < 1 || p->tune_max > kMaxTrialsTrace) return false;
    if (p->loops_loc < 1 || p->loops_loc > kMaxLoops || p->loops_est < 1 ||
        p->loops_est > kMaxLoops)
        return false;
    if (!(p->filter_alpha > 0 && p->filter_alpha <= 2)) return false;
    if (!(p->filter_tol > 0 && p->filter_tol < 1)) return false;
    if (!(p->thr_rel >= 0 && p->thr_med >= 0 && p->tie_eta >= 0 && p->tie_eta < 1)) return false;
    if (p->coop_blocks_per_sm < 0 || p->coop_blocks_per_sm > 8) return false;
    if (p->tune_stages < 1 || p->tune_stages > 3) return false;
    if (p->fixed_k != 0 && p->fixed_k != 1) return false;
    if (p->est_reuse_loc != 0 && p->est_reuse_loc != 1) return false;
    if (p->est_reuse_loc && p->loops_est > p->loops_loc) return false;
    if (p->precision != 0 && p->precision != 1) return false;
    if (p->coop_sms < 0) return false;
    return true;
}

static void plan_free(atsfft_plan_s *P)
{
    void *ptrs[] = {P->d_tune, P->d_le, P->d_win, P->d_resp, P->d_rgain, P->d_phase, P->d_tw, P->d_part, P->d_tz,
                    P->d_z, P->d_fft_tmp, P->d_energy, P->d_stats, P->d_lmax, P->d_lmax_e,
                    P->d_sel, P->d_bucketbits, P->d_kept, P->d_coordbits, P->d_blk, P->d_x32, P->d_f64a,
                    P->d_f64b, P->d_tw64, P->d_wtab64, P->d_state, P->d_tjob, P->d_tstat,
                    P->d_lstat, P->d_taps_tune, P->d_taps_le};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    if (P->prof)
        for (int i = 0; i <= kPhases; i++) cudaEventDestroy(P->ev[i]);
    delete P;
}

static int ilog2_ceil(int64_t v)
{
    int r = 0;
    while (((int64_t)1 << r) < v) r++;
    return r;
}

// Plan creation; with `tmpl` (a plan of the same shape, parameters, hint and seed) the
// window, phase and twiddle tables are copied from it instead of being computed.
static atsfft_status plan_create(atsfft_plan_t *out, int ndim, const int64_t *shape,
                                 int64_t k_hint, const atsfft_params *pp, uint64_t seed,
                                 const atsfft_plan_s *tmpl)
{
    if (!out) return ATSFFT_E_INVALID_ARG;
    *out = nullptr;
    if (!shape || (ndim != 1 && ndim != 2) || k_hint < 0) return ATSFFT_E_INVALID_ARG;
    if (shape[0] > 0 && k_hint > (ndim == 1 ? shape[0] : shape[0] * shape[0])) return ATSFFT_E_INVALID_ARG;
    atsfft_params p;
    if (pp)
        p = *pp;
    else
        atsfft_default_params(&p);
    if (!params_ok(&p)) return ATSFFT_E_INVALID_ARG;
    int64_t n = shape[0];
    if (n <= 0 || (n & (n - 1))) return ATSFFT_E_INVALID_ARG;
    if (ndim == 1 && (n < 256 || n > ((int64_t)1 << 28))) return ATSFFT_E_INVALID_ARG;
    if (ndim == 2 && (shape[1] != n || n < 32 || n > ((int64_t)1 << 14))) return ATSFFT_E_INVALID_ARG;

    atsfft_plan_s *P = new (std::nothrow) atsfft_plan_s;
    if (!P) return ATSFFT_E_NOMEM;
    memset(P, 0, sizeof(*P));
    P->ndim = ndim;
    P->n = n;
    P->logn = ilog2_ceil(n);
    P->ncoord = ndim == 1 ? n : n * n;
    P->p = p;
    P->seed = seed;
    P->L_loc = p.loops_loc;
    P->L_est = p.loops_est;
    P->b_lo = p.b_min_log2 ? p.b_min_log2 : (ndim == 1 ? 4 : 3);
    P->b_hi = p.b_max_log2 ? p.b_max_log2 : (ndim == 1 ? P->logn - 4 : P->logn - 2);
    if (P->b_lo < 1 || P->b_hi > P->logn - 1 || P->b_lo > P->b_hi ||
        (ndim == 1 && P->b_hi > 24) || (ndim == 2 && P->b_hi > 12)) {
        delete P;
        return ATSFFT_E_INVALID_ARG;
    }
    P->b0 = P->b_lo;
    P->k_hint = k_hint;
    if (k_hint > 0) {
        int want = ndim == 1 ? ilog2_ceil(2 * k_hint) : (ilog2_ceil(2 * k_hint) + 1) / 2;
        if (want > P->b0) P->b0 = want;
        if (P->b0 > P->b_hi) P->b0 = P->b_hi;
    }
    if (cudaGetDevice(&P->device) != cudaSuccess) {
        delete P;
        return ATSFFT_E_CUDA;
    }
    cudaDeviceGetAttribute(&P->num_sms, cudaDevAttrMultiProcessorCount, P->device);

    for (int b = P->b0; b <= P->b_hi; b++) hash_params_for(seed, 0, b, n, ndim, &P->h_tune[b]);
    for (int l = 0; l < P->L_loc; l++) hash_params_for(seed, 1, l, n, ndim, &P->h_le[l]);
    P->est_base = p.est_reuse_loc ? 0 : P->L_loc;
    P->nh_le = p.est_reuse_loc ? P->L_loc : P->L_loc + P->L_est;
    if (!p.est_reuse_loc)
        for (int l = 0; l < P->L_est; l++) hash_params_for(seed, 2, l, n, ndim, &P->h_le[P->L_loc + l]);
    if (p.fixed_k) {
        // B^2 >= n k (1D) or B^4 >= N^2 k (2D), clamped to the range
        if (k_hint <= 0) {
            delete P;
            return ATSFFT_E_INVALID_ARG;
        }
        const int m = ilog2_ceil(ndim == 1 ? n * k_hint : n * n * k_hint);
        int bf = ndim == 1 ? (m + 1) / 2 : (m + 3) / 4;
        if (bf < P->b_lo) bf = P->b_lo;
        if (bf > P->b_hi) bf = P->b_hi;
        P->b_fixed = bf;
    }

    // ---- allocations ----
    atsfft_status st = ATSFFT_OK;
    auto A = [&](void **ptr, size_t bytes) {
        if (st != ATSFFT_OK) return;
        cudaError_t e = cudaMalloc(ptr, bytes ? bytes : 16);
        if (e != cudaSuccess) st = cuda_status(e);
    };
    int64_t resp_total = 0;
    int64_t tz_total = 0;
    for (int b = P->b0; b <= P->b_hi; b++) {
        P->h_win[b] = window_shape(n, b, p.filter_alpha, p.filter_tol);
        P->resp_off[b] = resp_total;
        resp_total += n >> b;
        P->tz_off[b] = tz_total;
        tz_total += ndim == 1 ? ((int64_t)1 << b) : ((int64_t)1 << (2 * b));
    }
    for (int b = P->b0; b <= P->b_hi; b++) P->h_tjob[b] = make_job(P, b, 1);
    int64_t nb_max = ndim == 1 ? ((int64_t)1 << P->b_hi) : ((int64_t)1 << (2 * P->b_hi));
    int nh_le = P->nh_le;
    // partials: largest of (tuning single hash, location + estimation) x chunks
    size_t part = 0;
    for (int b = P->b0; b <= P->b_hi; b++) {
        int64_t nb = ndim == 1 ? ((int64_t)1 << b) : ((int64_t)1 << (2 * b));
        Job j = make_job(P, b, nh_le);
        size_t need = (size_t)j.chunks * (size_t)nh_le * (size_t)nb;
        if (need > part) part = need;
    }
    // tuning partials: every B of the range gets its own region so all bins run before
    // one batched FFT.  1D large-window B's share one residue-stream pass with modulus
    // R = the largest of them; B's hash writes chunks(R) * R / B blocks of B values.
    {
        int64_t off = 0;
        // tuning stages in 1D: the leading gather-form trials; then the residue-stream
        // trials; with three stages the largest trial alone last (rarely needed: it only
        // runs when the controller walks past the one before it)
        int s1 = P->b_hi, s2 = P->b_hi;
        if (ndim == 1 && p.tune_stages >= 2) {
            s1 = P->b0 - 1;
            for (int b = P->b0; b <= P->b_hi && !P->h_tjob[b].stream; b++) s1 = b;
            if (p.tune_stages == 3 && P->b_hi - 1 > s1) s2 = P->b_hi - 1;
        }
        P->tune_hi[0] = P->b0 - 1;
        P->tune_hi[1] = s1;
        P->tune_hi[2] = s2;
        P->tune_hi[3] = P->b_hi;
        int stage_of[kMaxLogB];
        for (int st = 1; st <= 3; st++) {
            P->tstream_logR[st] = -1;
            for (int b = P->tune_hi[st - 1] + 1; b <= P->tune_hi[st]; b++) {
                stage_of[b] = st;
                if (ndim == 1 && P->h_tjob[b].stream) P->tstream_logR[st] = b;
            }
            P->tstream_chunks[st] =
                P->tstream_logR[st] >= 0 ? P->h_tjob[P->tstream_logR[st]].chunks : 1;
        }
        P->tstream_logR[0] = -1;
        P->tstream_chunks[0] = 1;
        for (int b = P->b0; b <= P->b_hi; b++) {
            int64_t nb = ndim == 1 ? ((int64_t)1 << b) : ((int64_t)1 << (2 * b));
            P->tpart_off[b] = off;
            if (ndim == 1 && P->h_tjob[b].stream) {
                const int st = stage_of[b];
                P->tchunks[b] = P->tstream_chunks[st] << (P->tstream_logR[st] - b);
            } else if (ndim == 1) {
                P->tchunks[b] = 1;
            } else {
                P->tchunks[b] = P->h_tjob[b].chunks;
            }
            off += nb * P->tchunks[b];
        }
        if ((size_t)off > part) part = (size_t)off;
    }
    P->part_elems = part;
    P->lmax_cap = ndim == 1 ? nb_max / 2 + 1 : nb_max / 4 + 1;
    P->bucket_words = (nb_max + 31) / 32;
    P->kept_cap = kKeptCap;
    P->coord_words = (P->ncoord + 31) / 32;
    P->e_loc_off = tz_total;

    A((void **)&P->d_tune, sizeof(HashParam) * kMaxLogB);
    A((void **)&P->d_le, sizeof(HashParam) * (2 * kMaxLoops + 1));
    A((void **)&P->d_win, sizeof(WindowParam) * kMaxLogB);
    A((void **)&P->d_resp, sizeof(double) * resp_total);
    A((void **)&P->d_rgain, sizeof(float) * resp_total);
    P->phase_s = (P->logn + 1) / 2;
    A((void **)&P->d_phase, sizeof(float2) * (((size_t)1 << P->phase_s) + ((size_t)P->n >> P->phase_s)));
    A((void **)&P->d_tw, sizeof(float2) * kTwEntries);
    A((void **)&P->d_part, sizeof(float2) * part);
    A((void **)&P->d_tz, sizeof(float2) * tz_total);
    A((void **)&P->d_z, sizeof(float2) * nh_le * nb_max);
    // four-step intermediate (1D: the location pass's nh x B*, or every tuning trial's
    // spectrum size at its tz offset) or per-axis tap tables, nh x 2 x N (2D)
    size_t tmp_elems = (size_t)nh_le * (size_t)nb_max;
    if ((size_t)tz_total > tmp_elems) tmp_elems = (size_t)tz_total;
    if (ndim == 2 && (size_t)nh_le * 2 * (size_t)n > tmp_elems) tmp_elems = (size_t)nh_le * 2 * (size_t)n;
    A((void **)&P->d_fft_tmp, sizeof(float2) * tmp_elems);
    A((void **)&P->d_energy, sizeof(float) * (tz_total + P->L_loc * nb_max));
    A((void **)&P->d_stats, sizeof(HashStats) * (kMaxLogB + kMaxLoops));
    A((void **)&P->d_lmax, sizeof(int32_t) * P->L_loc * P->lmax_cap);
    A((void **)&P->d_lmax_e, sizeof(float) * P->L_loc * P->lmax_cap);
    A((void **)&P->d_sel, sizeof(int32_t) * P->L_loc * P->lmax_cap);
    A((void **)&P->d_bucketbits, sizeof(uint32_t) * (size_t)P->L_loc * (size_t)P->bucket_words);
    A((void **)&P->d_kept, sizeof(uint32_t) * (size_t)P->kept_cap);
    A((void **)&P->d_coordbits, sizeof(uint32_t) * (size_t)P->coord_words);
    // kept coordinates per chunk of the coordinate bitmap (the ordered compaction beyond
    // kKeptCap kept coordinates), zeroed at the start of every exec
    P->nchunks = (P->coord_words + kChunkWords - 1) / kChunkWords;
    A((void **)&P->d_blk, sizeof(uint32_t) * (size_t)P->nchunks);
    if (p.precision == 1) {
        A((void **)&P->d_x32, sizeof(float2) * (size_t)P->ncoord);
        A((void **)&P->d_f64a, sizeof(double2) * (size_t)P->L_est * (size_t)nb_max);
        A((void **)&P->d_f64b, sizeof(double2) * (size_t)P->L_est * (size_t)nb_max);
        A((void **)&P->d_tw64, sizeof(double2) * (size_t)(((int64_t)1 << P->b_hi) / 2 + 1));
        if (ndim == 2) A((void **)&P->d_wtab64, sizeof(double2) * (size_t)n);   // 2h + 1 <= N - 1
    }
    if (ndim == 2) {
        // per-axis tap tables of every B of the range (tuning hash; location and estimation
        // hashes), built once below
        A((void **)&P->d_taps_tune, sizeof(float2) * (size_t)(P->b_hi + 1) * 2 * (size_t)n);
        A((void **)&P->d_taps_le, sizeof(float2) * (size_t)(P->b_hi + 1) * (size_t)nh_le * 2 * (size_t)n);
    }
    A((void **)&P->d_state, sizeof(ExecState));
    A((void **)&P->d_tjob, sizeof(Job) * kMaxLogB);
    A((void **)&P->d_tstat, sizeof(StatJob) * kMaxLogB);
    A((void **)&P->d_lstat, sizeof(StatJob) * kMaxLoops);
    if (st != ATSFFT_OK) {
        plan_free(P);
        return st;
    }

    // ---- window tables (plan time, synchronous) ----
    cudaError_t e = cudaSuccess;
    double *d_partial = nullptr, *d_S0 = nullptr;
    // one B at a time uses (D + 1) offsets x its chunks of taps; the largest such product
    // (the largest D and the most chunks belong to opposite ends of the B range, so their
    // product would be far larger: terabytes at n = 2^28)
    int64_t partial_elems = 1;
    for (int b = P->b0; b <= P->b_hi && !tmpl; b++) {
        const int64_t nch = (P->h_win[b].h + kRespChunk) / kRespChunk;
        const int64_t need = ((n >> b) + 1) * nch;
        if (need > partial_elems) partial_elems = need;
    }
    e = cudaMalloc(&d_partial, sizeof(double) * (size_t)partial_elems);
    if (e == cudaSuccess) e = cudaMalloc(&d_S0, sizeof(double) * kMaxLogB);
    for (int b = P->b0; b <= P->b_hi && e == cudaSuccess && !tmpl; b++) {
        WindowParam &w = P->h_win[b];
        int64_t D = n >> b;
        int nch = (int)((w.h + kRespChunk) / kRespChunk);
        dim3 grid((unsigned)((D + 1 + kRespThreads - 1) / kRespThreads), (unsigned)nch);
        k_window_partial<<<grid, kRespThreads>>>(n, b, w.s, w.h, d_partial, nch);
        k_window_finish<<<1, 256>>>(D, d_partial, nch, P->d_resp + P->resp_off[b], d_S0 + b);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && !tmpl) {
        k_twiddles<<<kTwEntries / 256, 256>>>(P->d_tw);
        k_recip_gain<<<P->num_sms * 4, 256>>>(P->d_resp, resp_total, P->d_rgain);
        k_phase_table<<<P->num_sms, 256>>>(P->logn, P->phase_s, P->d_phase);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && tmpl) {
        const size_t nphase = ((size_t)1 << P->phase_s) + ((size_t)n >> P->phase_s);
        e = cudaMemcpy(P->d_tw, tmpl->d_tw, sizeof(float2) * kTwEntries, cudaMemcpyDeviceToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(P->d_resp, tmpl->d_resp, sizeof(double) * resp_total, cudaMemcpyDeviceToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(P->d_rgain, tmpl->d_rgain, sizeof(float) * resp_total, cudaMemcpyDeviceToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(P->d_phase, tmpl->d_phase, sizeof(float2) * nphase, cudaMemcpyDeviceToDevice);
        memcpy(P->h_win, tmpl->h_win, sizeof(P->h_win));
    }
    double S0[kMaxLogB];
    if (e == cudaSuccess && !tmpl)
        e = cudaMemcpy(S0, d_S0, sizeof(double) * kMaxLogB, cudaMemcpyDeviceToHost);
    if (d_partial) cudaFree(d_partial);
    if (d_S0) cudaFree(d_S0);
    if (e == cudaSuccess) {
        if (!tmpl)
            for (int b = P->b0; b <= P->b_hi; b++) {
                WindowParam &w = P->h_win[b];
                w.A = (double)n / S0[b];
                w.log2c = (float)log2(w.A * (double)n / M_PI);
                w.cA_D = (float)(w.A * (double)(n >> b));
            }
        e = cudaMemcpy(P->d_win, P->h_win, sizeof(P->h_win), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaMemcpy(P->d_tune, P->h_tune, sizeof(P->h_tune), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(P->d_le, P->h_le, sizeof(P->h_le), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && ndim == 2) {
        for (int b = P->b0; b <= P->b_hi; b++) {
            k_taps_2d<<<P->num_sms * 2, 256>>>(P->logn, P->d_tune + b, 1, P->d_win, nullptr, b,
                                               P->d_taps_tune + (size_t)b * 2 * (size_t)n);
            k_taps_2d<<<P->num_sms * 2, 256>>>(P->logn, P->d_le, nh_le, P->d_win, nullptr, b,
                                               P->d_taps_le + (size_t)b * (size_t)nh_le * 2 * (size_t)n);
        }
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(P->d_tjob, P->h_tjob, sizeof(P->h_tjob), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        // tuning stat jobs: one per B of the range, spectra and energies at tz_off[b]
        StatJob ts[kMaxLogB];
        P->ntstat = 0;
        for (int b = P->b0; b <= P->b_hi; b++) {
            StatJob &j = ts[P->ntstat++];
            j.spec = P->d_tz + P->tz_off[b];
            j.energy = P->d_energy + P->tz_off[b];
            j.hash = P->d_tune + b;
            j.logB = b;
            j.slot = b;
            j.list = -1;
            j.active = 1;
        }
        e = cudaMemcpy(P->d_tstat, ts, sizeof(StatJob) * P->ntstat, cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaMemset(P->d_coordbits, 0, sizeof(uint32_t) * P->coord_words);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        plan_free(P);
        return cuda_status(e);
    }
    *out = P;
    return ATSFFT_OK;
}

extern "C" atsfft_status atsfft_plan(atsfft_plan_t *out, int ndim, const int64_t *shape,
                                     int64_t k_hint, const atsfft_params *pp, uint64_t seed)
{
    return plan_create(out, ndim, shape, k_hint, pp, seed, nullptr);
}

extern "C" atsfft_status atsfft_plan_clone(atsfft_plan_t src, atsfft_plan_t *out)
{
    if (!out) return ATSFFT_E_INVALID_ARG;
    *out = nullptr;
    if (!src) return ATSFFT_E_INVALID_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return ATSFFT_E_CUDA;
    if (dev != src->device) return ATSFFT_E_INVALID_ARG;
    const int64_t shape[2] = {src->n, src->n};
    return plan_create(out, src->ndim, shape, src->k_hint, &src->p, src->seed, src);
}

extern "C" atsfft_status atsfft_destroy(atsfft_plan_t P)
{
    if (!P) return ATSFFT_E_INVALID_ARG;
    cudaDeviceSynchronize();
    plan_free(P);
    return ATSFFT_OK;
}

extern "C" atsfft_status atsfft_window_response(atsfft_plan_t P, int64_t B, double *h_resp)
{
    if (!P || !h_resp || B <= 0 || (B & (B - 1))) return ATSFFT_E_INVALID_ARG;
    int b = ilog2_ceil(B);
    if (b < P->b0 || b > P->b_hi) return ATSFFT_E_INVALID_ARG;
    cudaError_t e = cudaMemcpy(h_resp, P->d_resp + P->resp_off[b], sizeof(double) * (P->n >> b),
                               cudaMemcpyDeviceToHost);
    return cuda_status(e);
}
