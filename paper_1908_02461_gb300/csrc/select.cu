// select.cu -- bucket energies, threshold, local maxima and their count (Section III-A,
// Fig. 5), the tuning controller (Eqs. (12)-(14), Algorithm 2), the top-num cutoff
// (Algorithm 1 "find num largest indices") and the location votes (Section II-B).
//
// Threshold T = max(thr_rel * maxE, thr_med * medianE), median = element floor(nb/2) of the
// ascending energies.  The median is needed only if it can exceed X = (thr_rel/thr_med)
// maxE: with #{E > X'} <= nb - floor(nb/2) - 1 for X' = X (1 - 2^-20) the median is <= X'
// and thr_med * median < thr_rel * maxE, so T = thr_rel * maxE exactly.  Otherwise the
// median is found exactly by a three-digit radix select on the energies' bit patterns.
#include <math.h>

#include "common.cuh"

namespace atsfft {

__device__ __forceinline__ int64_t nb_of(int ndim, int logB)
{
    return ndim == 1 ? ((int64_t)1 << logB) : ((int64_t)1 << (2 * logB));
}

template <typename T, typename Op>
__device__ T block_reduce(T v, Op op)
{
    __shared__ T red[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    if (w == 0) {
        v = lane < (int)(blockDim.x >> 5) ? red[lane] : red[0];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_xor_sync(0xffffffffu, v, o));
    }
    return v;   // valid in thread 0
}

struct MaxF { __device__ float operator()(float a, float b) const { return fmaxf(a, b); } };
struct SumU { __device__ uint32_t operator()(uint32_t a, uint32_t b) const { return a + b; } };

__global__ void k_stats_energy(const StatJob *jobs, int ndim, HashStats *stats)
{
    const StatJob J = jobs[blockIdx.y];
    if (!J.active) return;
    const int64_t nb = nb_of(ndim, J.logB);
    float m = 0.f;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nb;
         j += (int64_t)gridDim.x * blockDim.x) {
        const float2 v = J.spec[j];
        const float e = v.x * v.x + v.y * v.y;
        J.energy[j] = e;
        m = fmaxf(m, e);
    }
    m = block_reduce(m, MaxF());
    if (threadIdx.x == 0 && m > 0.f) atomicMax(&stats[J.slot].max_bits, __float_as_uint(m));
}

__global__ void k_stats_above(const StatJob *jobs, int ndim, HashStats *stats, float ratio)
{
    const StatJob J = jobs[blockIdx.y];
    if (!J.active) return;
    const int64_t nb = nb_of(ndim, J.logB);
    const float X = __uint_as_float(stats[J.slot].max_bits) * ratio;
    uint32_t c = 0;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nb;
         j += (int64_t)gridDim.x * blockDim.x)
        c += J.energy[j] > X;
    c = block_reduce(c, SumU());
    if (threadIdx.x == 0 && c) atomicAdd(&stats[J.slot].above, c);
}

__global__ void k_stats_decide(const StatJob *jobs, int ndim, HashStats *stats, uint32_t *hist,
                               int use_median)
{
    const StatJob J = jobs[blockIdx.x];
    if (!J.active) return;
    const int64_t nb = nb_of(ndim, J.logB);
    const int64_t m = nb / 2;
    HashStats &st = stats[J.slot];
    const bool need = use_median && (int64_t)st.above > nb - m - 1;
    if (threadIdx.x == 0) {
        st.need_median = need;
        st.prefix = 0;
        st.rank = (uint32_t)m;
    }
    if (need)
        for (int b = threadIdx.x; b < kHistBins; b += blockDim.x) hist[(int64_t)J.slot * kHistBins + b] = 0;
}

// digit 0: bits [20, 32), digit 1: [8, 20), digit 2: [0, 8)
__device__ __forceinline__ void digit_range(int digit, int &lo, int &width)
{
    lo = digit == 0 ? 20 : (digit == 1 ? 8 : 0);
    width = digit == 2 ? 8 : 12;
}

__global__ void k_radix_hist(const StatJob *jobs, int ndim, HashStats *stats, uint32_t *hist,
                             int digit)
{
    __shared__ uint32_t h[kHistBins];
    const StatJob J = jobs[blockIdx.y];
    if (!J.active || !stats[J.slot].need_median) return;
    int lo, width;
    digit_range(digit, lo, width);
    const int hi = lo + width;
    const uint32_t prefix = stats[J.slot].prefix;
    for (int b = threadIdx.x; b < kHistBins; b += blockDim.x) h[b] = 0;
    __syncthreads();
    const int64_t nb = nb_of(ndim, J.logB);
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nb;
         j += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t bits = __float_as_uint(J.energy[j]);
        if (digit == 0 || (bits >> hi) == prefix) atomicAdd(&h[(bits >> lo) & ((1u << width) - 1)], 1u);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < (1 << width); b += blockDim.x)
        if (h[b]) atomicAdd(&hist[(int64_t)J.slot * kHistBins + b], h[b]);
}

// One block (256 threads) per job: find the bin holding the wanted rank.
__global__ void k_radix_pick(const StatJob *jobs, HashStats *stats, uint32_t *hist, int digit)
{
    __shared__ uint32_t part[256];
    const StatJob J = jobs[blockIdx.x];
    if (!J.active || !stats[J.slot].need_median) return;
    int lo, width;
    digit_range(digit, lo, width);
    (void)lo;
    const int nbins = 1 << width;
    const int per = nbins / 256;
    uint32_t *hh = hist + (int64_t)J.slot * kHistBins;
    HashStats &st = stats[J.slot];
    const uint32_t rank = st.rank;
    uint32_t sum = 0;
    for (int k = 0; k < per; k++) sum += hh[threadIdx.x * per + k];
    part[threadIdx.x] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t acc = 0;
        for (int t = 0; t < 256; t++) {
            const uint32_t v = part[t];
            part[t] = acc;
            acc += v;
        }
    }
    __syncthreads();
    const uint32_t before = part[threadIdx.x];
    if (rank >= before && rank < before + sum) {
        uint32_t cum = before;
        for (int k = 0; k < per; k++) {
            const uint32_t v = hh[threadIdx.x * per + k];
            if (rank < cum + v) {
                const uint32_t bin = threadIdx.x * per + k;
                st.prefix = (st.prefix << width) | bin;
                st.rank = rank - cum;
                if (digit == 2) st.med_bits = st.prefix;
                break;
            }
            cum += v;
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < kHistBins; b += blockDim.x) hh[b] = 0;
}

// Does a bucket of energy ec dominate its neighbour (displacement d1, d2) of energy em?
// Beyond the relative tie band the larger wins; inside it the neighbour loses iff it
// lies before the bucket in cyclic order (d1 < 0, or d1 == 0 and d2 < 0).
__device__ __forceinline__ bool dominates(float ec, float em, float up, int d1, int d2)
{
    if (ec > up * em) return true;
    if (em > up * ec) return false;
    return d1 < 0 || (d1 == 0 && d2 < 0);
}

__global__ void k_stats_localmax(const StatJob *jobs, int ndim, HashStats *stats, float thr_rel,
                                 float thr_med, float up, int32_t *lists, int64_t cap)
{
    const StatJob J = jobs[blockIdx.y];
    if (!J.active) return;
    HashStats &st = stats[J.slot];
    const float M = __uint_as_float(st.max_bits);
    float T = thr_rel * M;
    if (st.need_median) T = fmaxf(T, thr_med * __uint_as_float(st.med_bits));
    if (blockIdx.x == 0 && threadIdx.x == 0) st.T = T;
    const int logB = J.logB;
    const uint32_t B = 1u << logB, mask = B - 1;
    const float *E = J.energy;
    const int64_t nb = nb_of(ndim, logB);
    const uint32_t s1 = J.hash->sigma[0] & mask, p1 = J.hash->sinv[0] & mask;
    const uint32_t s2 = J.hash->sigma[1] & mask, p2 = J.hash->sinv[1] & mask;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nb;
         j += (int64_t)gridDim.x * blockDim.x) {
        const float e = E[j];
        if (!(e > T)) continue;
        bool ok = true;
        int32_t c;
        if (ndim == 1) {
            const uint32_t jj = (uint32_t)j;
            c = (int32_t)((s1 * jj) & mask);
            ok = dominates(e, E[(jj - p1) & mask], up, 0, -1) &&
                 dominates(e, E[(jj + p1) & mask], up, 0, 1);
        } else {
            const uint32_t j1 = (uint32_t)(j >> logB), j2 = (uint32_t)(j & mask);
            c = (int32_t)((((s1 * j1) & mask) << logB) | ((s2 * j2) & mask));
            for (int d1 = -1; d1 <= 1 && ok; d1++)
                for (int d2 = -1; d2 <= 1 && ok; d2++) {
                    if (d1 == 0 && d2 == 0) continue;
                    const uint32_t m1 = (j1 + (uint32_t)d1 * p1) & mask;
                    const uint32_t m2 = (j2 + (uint32_t)d2 * p2) & mask;
                    ok = dominates(e, E[((int64_t)m1 << logB) | m2], up, d1, d2);
                }
        }
        if (ok) {
            const uint32_t pos = atomicAdd(&st.nmax, 1u);
            if (J.list >= 0 && pos < cap) lists[(int64_t)J.list * cap + pos] = c;
        }
    }
}

void launch_stats(const atsfft_plan_s *P, const StatJob *jobs, int njobs, int64_t max_nb,
                  cudaStream_t s)
{
    const int ndim = P->ndim;
    const atsfft_params &p = P->p;
    int64_t blocks = (max_nb + 255) / 256;
    if (blocks > (int64_t)P->num_sms * 4) blocks = (int64_t)P->num_sms * 4;
    if (blocks < 1) blocks = 1;
    const dim3 grid((unsigned)blocks, (unsigned)njobs);
    const bool use_median = p.thr_med > 0;
    const float ratio = use_median ? (float)(p.thr_rel / p.thr_med * (1.0 - 1.0 / 1048576.0)) : 0.f;
    k_stats_energy<<<grid, 256, 0, s>>>(jobs, ndim, P->d_stats);
    count_launch(P, use_median ? 10 : 2);
    if (use_median) {
        k_stats_above<<<grid, 256, 0, s>>>(jobs, ndim, P->d_stats, ratio);
        k_stats_decide<<<njobs, 256, 0, s>>>(jobs, ndim, P->d_stats, P->d_hist, 1);
        for (int d = 0; d < 3; d++) {
            k_radix_hist<<<grid, 256, 0, s>>>(jobs, ndim, P->d_stats, P->d_hist, d);
            k_radix_pick<<<njobs, 256, 0, s>>>(jobs, P->d_stats, P->d_hist, d);
        }
    }
    k_stats_localmax<<<grid, 256, 0, s>>>(jobs, ndim, P->d_stats, (float)p.thr_rel,
                                          (float)p.thr_med, (float)(1.0 + p.tie_eta), P->d_lmax,
                                          P->lmax_cap);
}

// ---------------------------------------------------------------------------------
// Controller: one thread walks the tuning trials B0, 2 B0, ... (each B's count was
// computed speculatively by the kernels above) through Eq. (12) and Eq. (14) until
// the stop reading: stop at the first trial with r < delta2 (keep branch, or halve
// branch onto the already evaluated B/2); r = inf when either count is 0; a trial
// whose energies are all 0 ends with k* = 0.  Then it writes the job at B*.
// ---------------------------------------------------------------------------------
__global__ void k_controller(int ndim, int b0, int b_hi, int tune_max, double delta1,
                             double delta2, const HashStats *stats, const Job *tjob, int nh_le,
                             int L_loc, ExecState *state, StatJob *lstat, const float2 *z,
                             float *e_loc, const HashParam *le)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    (void)delta1;
    int b = b0, trial = 0;
    int64_t kprev = 0, k = 0;
    int status = ATSFFT_OK, empty = 0;
    for (;; trial++) {
        k = stats[b].nmax;
        if (trial < kMaxTrialsTrace) {
            state->trial_B[trial] = (int64_t)1 << b;
            state->trial_k[trial] = k;
        }
        if (stats[b].max_bits == 0) {   // every energy exactly 0
            empty = 1;
            k = 0;
            break;
        }
        double r = NAN;
        if (trial > 0) r = (kprev == 0 || k == 0) ? INFINITY : fabs(1.0 - (double)k / (double)kprev);
        if (trial > 0 && r < delta2) break;
        if (b == b_hi) {
            if (trial > 0) status = ATSFFT_E_NOT_SPARSE;
            break;
        }
        if (trial + 1 >= tune_max) {
            status = ATSFFT_E_NOT_CONVERGED;
            break;
        }
        kprev = k;
        b++;
    }
    if (k == 0) empty = 1;
    state->ntrials = trial + 1;
    state->b_star = b;
    state->k_star = k;
    state->status = status;
    state->empty = empty;
    Job j = tjob[b];
    j.nh = nh_le;
    j.active = !empty;
    state->job = j;
    const int64_t nb = nb_of(ndim, b);
    for (int l = 0; l < L_loc; l++) {
        StatJob s;
        s.spec = z + (int64_t)l * nb;
        s.energy = e_loc + (int64_t)l * nb;
        s.hash = le + l;
        s.logB = b;
        s.slot = kMaxLogB + l;
        s.list = l;
        s.active = !empty;
        lstat[l] = s;
    }
}

void launch_controller(const atsfft_plan_s *P, cudaStream_t s)
{
    count_launch(P);
    k_controller<<<1, 32, 0, s>>>(P->ndim, P->b0, P->b_hi, P->p.tune_max, P->p.delta1,
                                  P->p.delta2, P->d_stats, P->d_tjob, P->L_loc + P->L_est,
                                  P->L_loc, P->d_state, P->d_lstat, P->d_z,
                                  P->d_energy + P->e_loc_off, P->d_le);
}

// ---------------------------------------------------------------------------------
// Top-num cutoff and votes
// ---------------------------------------------------------------------------------

// k-th smallest (0-based) key among the entries i < cnt with pred(i): four 8-bit radix
// passes over the list with a shared histogram.  Whole block must call.
template <class KeyF, class PredF>
__device__ uint32_t block_kth(int64_t cnt, uint32_t k, KeyF key, PredF pred)
{
    __shared__ uint32_t hist[256];
    __shared__ uint32_t sh_prefix, sh_k;
    if (threadIdx.x == 0) {
        sh_prefix = 0;
        sh_k = k;
    }
    for (int pass = 0; pass < 4; pass++) {
        const int shift = 24 - 8 * pass;
        for (int b = threadIdx.x; b < 256; b += blockDim.x) hist[b] = 0;
        __syncthreads();
        const uint32_t prefix = sh_prefix;
        for (int64_t i = threadIdx.x; i < cnt; i += blockDim.x) {
            if (!pred(i)) continue;
            const uint32_t kk = key(i);
            if (pass == 0 || (kk >> (shift + 8)) == prefix) atomicAdd(&hist[(kk >> shift) & 255u], 1u);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t cum = 0, want = sh_k;
            for (int b = 0; b < 256; b++) {
                if (want < cum + hist[b]) {
                    sh_prefix = (prefix << 8) | (uint32_t)b;
                    sh_k = want - cum;
                    break;
                }
                cum += hist[b];
            }
        }
        __syncthreads();
    }
    return sh_prefix;
}

__global__ void k_topnum(const StatJob *lstat, HashStats *stats, const int32_t *lists,
                         int32_t *sel, int64_t cap, ExecState *state, float eta_up, float eta_dn,
                         int ndim)
{
    __shared__ uint32_t n_sel, n_hi;
    const StatJob J = lstat[blockIdx.x];
    HashStats &st = stats[J.slot];
    if (!J.active) {
        if (threadIdx.x == 0) st.nsel = 0;
        return;
    }
    const int logB = J.logB;
    const uint32_t mask = (1u << logB) - 1;
    const uint32_t p1 = J.hash->sinv[0] & mask, p2 = J.hash->sinv[1] & mask;
    const int64_t cnt = min((int64_t)st.nmax, cap);
    const int64_t num = state->k_star;
    const int32_t *list = lists + (int64_t)J.list * cap;
    int32_t *out = sel + (int64_t)J.list * cap;
    const float *E = J.energy;
    auto energy_of = [&](int64_t i) -> float {
        const uint32_t c = (uint32_t)list[i];
        if (ndim == 1) return E[(p1 * c) & mask];
        const uint32_t c1 = c >> logB, c2 = c & mask;
        return E[((int64_t)((p1 * c1) & mask) << logB) | ((p2 * c2) & mask)];
    };
    if (threadIdx.x == 0) {
        n_sel = 0;
        n_hi = 0;
    }
    __syncthreads();
    if (cnt <= num) {
        for (int64_t i = threadIdx.x; i < cnt; i += blockDim.x) out[i] = list[i];
        if (threadIdx.x == 0) n_sel = (uint32_t)cnt;
    } else {
        // pivot: the num-th largest energy (bit patterns of E >= 0 order like the values)
        const uint32_t vb = ~block_kth(
            cnt, (uint32_t)(num - 1), [&](int64_t i) { return ~__float_as_uint(energy_of(i)); },
            [&](int64_t) { return true; });
        const float V = __uint_as_float(vb);
        const float hi = V * eta_up, lo = V * eta_dn;
        for (int64_t i = threadIdx.x; i < cnt; i += blockDim.x)
            if (energy_of(i) > hi) atomicAdd(&n_hi, 1u);
        __syncthreads();
        const uint32_t need = (uint32_t)num - n_hi;
        const uint32_t cthr = block_kth(
            cnt, need - 1, [&](int64_t i) { return (uint32_t)list[i]; },
            [&](int64_t i) {
                const float e = energy_of(i);
                return e >= lo && e <= hi;
            });
        for (int64_t i = threadIdx.x; i < cnt; i += blockDim.x) {
            const float e = energy_of(i);
            if (e > hi || (e >= lo && e <= hi && (uint32_t)list[i] <= cthr)) {
                const uint32_t pos = atomicAdd(&n_sel, 1u);
                out[pos] = list[i];
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) st.nsel = n_sel;
}

__global__ void k_vote(const HashStats *stats, const int32_t *sel, int64_t cap,
                       const ExecState *state, const HashParam *le, uint32_t *votes, int ndim,
                       int logn, int L_loc)
{
    __shared__ int64_t off[kMaxLoops + 1];
    if (state->empty) return;
    const int b = state->b_star;
    const int logD = logn - b;
    const int64_t D = (int64_t)1 << logD;
    const int64_t Dd = ndim == 1 ? D : D * D;
    if (threadIdx.x == 0) {
        int64_t acc = 0;
        for (int l = 0; l < L_loc; l++) {
            off[l] = acc;
            acc += (int64_t)stats[kMaxLogB + l].nsel * Dd;
        }
        off[L_loc] = acc;
    }
    __syncthreads();
    const int64_t items = off[L_loc];
    const uint32_t n = 1u << logn, nmask = n - 1, Bm = (1u << b) - 1;
    for (int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; it < items;
         it += (int64_t)gridDim.x * blockDim.x) {
        int l = 0;
        while (it >= off[l + 1]) l++;
        const int64_t rem = it - off[l];
        const int64_t sidx = rem >> (ndim == 1 ? logD : 2 * logD);
        const uint32_t q = (uint32_t)(rem & (Dd - 1));
        const uint32_t c = (uint32_t)sel[(int64_t)l * cap + sidx];
        const HashParam hp = le[l];
        int64_t coord;
        if (ndim == 1) {
            // bucket c collects permuted positions p in [c D - D/2, c D + D/2 - 1]
            const uint32_t pp = ((c << logD) - (uint32_t)(D >> 1) + q) & nmask;
            coord = (hp.sinv[0] * pp) & nmask;
        } else {
            const uint32_t c1 = c >> b, c2 = c & Bm;
            const uint32_t q1 = q >> logD, q2 = q & (uint32_t)(D - 1);
            const uint32_t pp1 = ((c1 << logD) - (uint32_t)(D >> 1) + q1) & nmask;
            const uint32_t pp2 = ((c2 << logD) - (uint32_t)(D >> 1) + q2) & nmask;
            coord = ((int64_t)((hp.sinv[0] * pp1) & nmask) << logn) | ((hp.sinv[1] * pp2) & nmask);
        }
        atomicAdd(&votes[coord >> 2], 1u << (8 * (coord & 3)));
    }
}

void launch_topnum_vote(const atsfft_plan_s *P, cudaStream_t s)
{
    count_launch(P, 2);
    k_topnum<<<P->L_loc, 256, 0, s>>>(P->d_lstat, P->d_stats, P->d_lmax, P->d_sel, P->lmax_cap,
                                      P->d_state, (float)(1.0 + P->p.tie_eta),
                                      (float)(1.0 - P->p.tie_eta), P->ndim);
    k_vote<<<P->num_sms * kPersistCtas, 256, 0, s>>>(P->d_stats, P->d_sel, P->lmax_cap, P->d_state,
                                                     P->d_le, P->d_votes, P->ndim, P->logn,
                                                     P->L_loc);
}

void launch_reset(const atsfft_plan_s *P, cudaStream_t s)
{
    cudaMemsetAsync(P->d_stats, 0, sizeof(HashStats) * (kMaxLogB + kMaxLoops), s);
    cudaMemsetAsync(P->d_state, 0, sizeof(ExecState), s);
}

}  // namespace atsfft
