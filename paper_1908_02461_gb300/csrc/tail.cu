// tail.cu -- everything after the bucket FFTs, with no grid-wide barrier: every step
// that needs all the results of the previous one is either a new kernel (chained with
// programmatic dependent launch, so its blocks are scheduled while the previous kernel
// finishes), or is run by the block that completes the last unit of work it depends on
// (a completion counter per hash and per launch: the block whose count is the last one
// goes on, nobody waits), or stays inside one thread-block cluster (whose CTAs are
// scheduled together: a hardware cluster barrier).
//
//   k_tune_tail  : threshold and local-maximum counts of the trials of one tuning stage
//                  (Section III-A; the energies and their maxima come from the bucket
//                  FFTs); the last block of a trial settles its median where it can matter;
//                  the last block of the launch walks the controller over Eqs. (12)/(14)
//                  (Algorithm 2), which fixes B*, k* and the jobs at B* (or leaves the walk
//                  to the next stage).
//   k_loc_select : the same statistics for the location hashes at B*, one thread-block
//                  cluster per hash: its CTAs gather the maxima in the shared memory of the
//                  first one (distributed shared memory), which makes the top-num cutoff
//                  (Algorithm 1 "find num largest") and the bitmap of selected buckets.
//   k_loc_votes  : votes (reverse hash): the preimages of the selected buckets that lie in
//                  >= ceil(L_loc/2) selected buckets are kept (Section II-B); one CTA per
//                  SM with the bitmaps in shared memory.
//   k_loc_finish : the kept coordinates in ascending order, the estimates of Eq. (11) with
//                  their componentwise median, and the caller's status words.
//
// Threshold T = max(thr_rel * maxE, thr_med * medianE), median = element floor(nb/2) of
// the ascending energies.  With #{E > X'} <= nb - floor(nb/2) - 1 for
// X' = (thr_rel/thr_med) maxE (1 - 2^-20) the median is <= X' and T = thr_rel * maxE
// exactly, so the local maxima are found with that T at once; only when the count says
// the median could matter is it found exactly (radix select on the energy bit patterns)
// and the maxima recounted (tuning) or the listed ones above the raised threshold kept
// (location: dominance does not depend on T).
#include <math.h>
#include <string.h>

#include "devmath.cuh"

namespace atsfft {

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Diagnostic time stamp (kernel start or end of a phase), kept in the exec state.
__device__ __forceinline__ void stamp(TailStamps *ts)
{
    const unsigned i = atomicAdd(&ts->nstamp, 1u);
    if (i < 32) ts->stamp[i] = global_ns();
}

// Programmatic dependent launch: wait until the previous kernel of the stream has
// completed and its writes are visible (returns at once for a kernel launched without
// the dependency); let the next kernel's blocks be scheduled.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_next()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Whole block, after it finished one unit of a group of `units`: counts it, and returns
// true (in every thread) in the block that counted the group's last unit.  The writes
// and atomics of every counted unit are then visible to that block: the block barrier
// orders every thread's writes before thread 0's release fence and count, and in the
// last block thread 0's acquire fence after the count comes before the barrier that
// releases its threads, which read the others' results through L2 (__ldcg).
__device__ bool finished_last(uint32_t *counter, uint32_t units)
{
    __shared__ int last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const bool l = atomicAdd(counter, 1u) == units - 1;
        if (l) __threadfence();
        last = l;
    }
    __syncthreads();
    return last != 0;
}


__device__ __forceinline__ int64_t nb_of(int ndim, int logB)
{
    return ndim == 1 ? ((int64_t)1 << logB) : ((int64_t)1 << (2 * logB));
}

__device__ __forceinline__ uint32_t warp_sum(uint32_t v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

constexpr int64_t kTask = 4096;   // buckets per statistics task

// Whole block (blockDim.x <= 1024, a multiple of 32): the sum of one value per thread.
__device__ uint32_t block_sum(uint32_t v)
{
    __shared__ uint32_t red[32];
    const int lane = threadIdx.x & 31;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    return warp_sum(lane < (int)(blockDim.x >> 5) ? red[lane] : 0u);
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

struct StatsParams {
    int ndim;
    float thr_rel, thr_med, up, ratio;   // up = 1 + eta; ratio = X' / maxE
    int use_median;
    HashStats *stats;
    int32_t *lists;
    float *list_e;         // the listed maxima's energies (same layout)
    int64_t cap;
};

__device__ float threshold_of(const HashStats &st, const StatsParams &S)
{
    float T = S.thr_rel * __uint_as_float(st.max_bits);
    if (st.need_median) T = fmaxf(T, S.thr_med * __uint_as_float(st.med_bits));
    return T;
}

// hist[bin] += 1 for every calling lane, one shared atomic per distinct bin in the warp
// (radix digits of nearly equal energies share a few bins).
__device__ __forceinline__ void hist_add(uint32_t *hist, uint32_t bin)
{
    const unsigned am = __activemask();
    const unsigned peers = __match_any_sync(am, bin);
    if ((int)(threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&hist[bin], (uint32_t)__popc(peers));
}

// Inclusive prefix sum over the lanes of a warp.
__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// Whole block (blockDim.x <= 1024, a multiple of 32): exclusive prefix sum of one value
// per thread and the block total, with one barrier (the warp totals are scanned by every
// warp at once, a lane per warp total).  The caller synchronises before the next call.
__device__ __forceinline__ uint32_t block_scan_core(uint32_t v, uint32_t &all)
{
    __shared__ uint32_t wtot[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t incl = warp_incl_scan(v);
    if (lane == 31) wtot[w] = incl;
    __syncthreads();
    const uint32_t t = lane < (int)(blockDim.x >> 5) ? wtot[lane] : 0u;
    const uint32_t tincl = warp_incl_scan(t);
    all = __shfl_sync(0xffffffffu, tincl, 31);
    return incl - v + __shfl_sync(0xffffffffu, tincl - t, w);
}

// Whole block: exclusive prefix sum of one value per thread; *total (shared) receives the
// block sum.
__device__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *total)
{
    uint32_t all;
    const uint32_t before = block_scan_core(v, all);
    if (total && threadIdx.x == 0) *total = all;
    __syncthreads();
    return before;
}

// Whole block (blockDim.x <= 1024, a multiple of 32; nbins a power of two): find the
// bin b of hist[0..nbins) (shared or global) with cum(b) <= rank < cum(b) + hist[b],
// where cum is the exclusive prefix sum.  The block's thread t sums bins
// [t*per, (t+1)*per); a block scan gives each thread its offset; the owner walks its few
// bins.  Result in *bin, *rem (shared), after a sync.
__device__ void block_find_rank(const uint32_t *hist, int nbins, uint32_t rank, uint32_t *bin,
                                uint32_t *rem)
{
    const int per = nbins >= (int)blockDim.x ? nbins / (int)blockDim.x : 1;
    const int t = threadIdx.x;
    uint32_t sum = 0;
    if (t * per < nbins)
        for (int k = 0; k < per; k++) sum += hist[t * per + k];
    uint32_t all;
    const uint32_t before = block_scan_core(sum, all);
    if (sum && rank >= before && rank < before + sum) {
        uint32_t cum = before;
        for (int k = 0; k < per; k++) {
            const uint32_t v = hist[t * per + k];
            if (rank < cum + v) {
                *bin = (uint32_t)(t * per + k);
                *rem = rank - cum;
                break;
            }
            cum += v;
        }
    }
    __syncthreads();
}

constexpr int kSmallMedian = 8192;

// Exact median (element floor(nb/2) of the ascending energies, as bits) of nb <= 8192
// energies by one block: the values are staged in shared memory and selected by rank
// comparison when there are at most blockDim of them, else with three radix digits
// (11, 11, 10 bits) over their bit patterns (E >= 0: bit order = value order).
__device__ __noinline__ uint32_t block_median(const float *E, int nb)
{
    extern __shared__ __align__(16) uint32_t dsm[];   // phase scratch shared by the tail's phases
    uint32_t *vals = dsm;               // kSmallMedian entries
    uint32_t *hist = dsm + kSmallMedian; // 2048 entries
    __shared__ uint32_t sh_prefix, sh_rank;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) vals[i] = __float_as_uint(E[i]);
    if (nb <= (int)blockDim.x) {
        // few values: the element whose rank (ties by index) is floor(nb/2), one per thread
        if (threadIdx.x == 0) sh_prefix = 0;
        __syncthreads();
        const int i = threadIdx.x;
        if (i < nb) {
            const uint32_t v = vals[i];
            int r = 0;
            for (int j = 0; j < nb; j++) {
                const uint32_t u = vals[j];
                r += u < v || (u == v && j < i);
            }
            if (r == nb / 2) sh_prefix = v;
        }
        __syncthreads();
        return sh_prefix;
    }
    if (threadIdx.x == 0) {
        sh_prefix = 0;
        sh_rank = (uint32_t)(nb / 2);
    }
    __syncthreads();
    const int los[3] = {21, 10, 0}, widths[3] = {11, 11, 10};
    for (int d = 0; d < 3; d++) {
        const int lo = los[d], width = widths[d], hi = lo + width;
        for (int b = threadIdx.x; b < (1 << width); b += blockDim.x) hist[b] = 0;
        __syncthreads();
        const uint32_t prefix = sh_prefix;
        for (int i = threadIdx.x; i < nb; i += blockDim.x) {
            const uint32_t v = vals[i];
            if (d == 0 || (v >> hi) == prefix) hist_add(hist, (v >> lo) & ((1u << width) - 1));
        }
        __syncthreads();
        __shared__ uint32_t fb, fr;
        block_find_rank(hist, 1 << width, sh_rank, &fb, &fr);
        if (threadIdx.x == 0) {
            sh_prefix = (prefix << width) | fb;
            sh_rank = fr;
        }
        __syncthreads();
    }
    return sh_prefix;
}

// One statistics job as the phases use it, staged in shared memory (all fields loaded
// in parallel at the start of the phases).
struct JobView {
    const float *E;        // energies (P-index order)
    HashStats *st;
    int32_t logB, list, active, pad;
    uint32_t s1, p1, s2, p2;   // sigma and sigma^{-1} mod B per axis
};

constexpr int kPerTask = (int)(kTask / 256);   // buckets per thread of a statistics task

// The local-maximum test of P-indices [e0, e1) of one job by a block of NT threads
// (e1 - e0 <= 16 NT): thread t tests e0 + t + NT u, u < 16, from energies loaded up front
// (ev[u]); bit u of `found` marks a maximum above T, `above` counts the thread's energies
// above X.
template <int NT>
__device__ __forceinline__ void localmax_scan(const JobView &J, const StatsParams &S, float T,
                                              int64_t e0, int64_t e1, float X,
                                              float (&ev)[kPerTask], uint32_t &found,
                                              uint32_t &above)
{
    const int logB = J.logB;
    const uint32_t mask = (1u << logB) - 1;
    const float *__restrict__ E = J.E;
    const uint32_t p1 = J.p1, p2 = J.p2;
#pragma unroll
    for (int u = 0; u < kPerTask; u++) {
        const int64_t j = e0 + threadIdx.x + NT * u;
        ev[u] = j < e1 ? __ldg(&E[j]) : 0.f;
    }
    above = 0;
    found = 0;
    if (S.ndim == 1) {
        // both neighbours of every element requested at once (coalesced: consecutive
        // threads hold consecutive P-indices)
        float el[kPerTask], er[kPerTask];
#pragma unroll
        for (int u = 0; u < kPerTask; u++) {
            const int64_t j = e0 + threadIdx.x + NT * u;
            const uint32_t jj = (uint32_t)j;
            el[u] = j < e1 ? __ldg(&E[(jj - p1) & mask]) : 0.f;
            er[u] = j < e1 ? __ldg(&E[(jj + p1) & mask]) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < kPerTask; u++) {
            const int64_t j = e0 + threadIdx.x + NT * u;
            const float e = ev[u];
            above += j < e1 && e > X;
            if (j < e1 && e > T && dominates(e, el[u], S.up, 0, -1) && dominates(e, er[u], S.up, 0, 1))
                found |= 1u << u;
        }
    } else {
        // eight neighbours, four elements at a time
#pragma unroll
        for (int u0 = 0; u0 < kPerTask; u0 += 4) {
            float nbv[4][8];
#pragma unroll
            for (int v = 0; v < 4; v++) {
                const int64_t j = e0 + threadIdx.x + NT * (u0 + v);
                const uint32_t jA = (uint32_t)(j >> logB) & mask, jB = (uint32_t)(j & mask);
                int q = 0;
#pragma unroll
                for (int d1 = -1; d1 <= 1; d1++)
#pragma unroll
                    for (int d2 = -1; d2 <= 1; d2++) {
                        if (d1 == 0 && d2 == 0) continue;
                        const uint32_t m1 = (jA + (uint32_t)d1 * p1) & mask;
                        const uint32_t m2 = (jB + (uint32_t)d2 * p2) & mask;
                        nbv[v][q++] = j < e1 ? __ldg(&E[((int64_t)m1 << logB) | m2]) : 0.f;
                    }
            }
#pragma unroll
            for (int v = 0; v < 4; v++) {
                const int u = u0 + v;
                const int64_t j = e0 + threadIdx.x + NT * u;
                const float e = ev[u];
                above += j < e1 && e > X;
                if (!(j < e1 && e > T)) continue;
                bool ok = true;
                int q = 0;
#pragma unroll
                for (int d1 = -1; d1 <= 1; d1++)
#pragma unroll
                    for (int d2 = -1; d2 <= 1; d2++) {
                        if (d1 == 0 && d2 == 0) continue;
                        ok = ok && dominates(e, nbv[v][q], S.up, d1, d2);
                        q++;
                    }
                if (ok) found |= 1u << u;
            }
        }
    }
}

// Bucket index of P-index j of a job (c = sigma j mod B, per axis).
__device__ __forceinline__ int32_t bucket_of_pindex(const JobView &J, int ndim, int64_t j)
{
    const uint32_t mask = (1u << J.logB) - 1;
    if (ndim == 1) return (int32_t)((J.s1 * (uint32_t)j) & mask);
    const uint32_t jA = (uint32_t)(j >> J.logB), jB = (uint32_t)(j & mask);
    return (int32_t)((((J.s1 * jA) & mask) << J.logB) | ((J.s2 * jB) & mask));
}

// Local maxima of buckets [e0, e1) of one job by a block of 256 threads
// (e1 - e0 <= kTask): the block's maxima are appended to the job's list with one atomic,
// and the count of energies above X with another.
__device__ void localmax_task(const JobView &J, const StatsParams &S, float T, int64_t e0,
                              int64_t e1, float X)
{
    HashStats &st = *J.st;
    float ev[kPerTask];
    uint32_t found, above;
    localmax_scan<256>(J, S, T, e0, e1, X, ev, found, above);
    __shared__ uint32_t base_sh;
    uint32_t total;
    const uint32_t before = block_exclusive_scan((uint32_t)__popc(found), &total);
    const uint32_t nabove = block_sum(above);
    if (threadIdx.x == 0) {
        base_sh = total ? atomicAdd(&st.nmax, total) : 0u;
        if (nabove) atomicAdd(&st.above, nabove);
    }
    __syncthreads();
    if (found && J.list >= 0) {
        uint32_t pos = base_sh + before;
        int32_t *lst = S.lists + (int64_t)J.list * S.cap;
#pragma unroll
        for (int u = 0; u < kPerTask; u++) {
            if (!(found & (1u << u))) continue;
            const int64_t j = e0 + threadIdx.x + 256 * u;
            const int32_t c = bucket_of_pindex(J, S.ndim, j);
            if (pos < S.cap) {
                lst[pos] = c;
                S.list_e[(int64_t)J.list * S.cap + pos] = ev[u];
            }
            pos++;
        }
    }
    __syncthreads();
}

// The recount after an exact median (rare): one out-of-line copy.
__device__ __noinline__ void localmax_task_cold(const JobView &J, const StatsParams &S, float T,
                                                int64_t e0, int64_t e1)
{
    localmax_task(J, S, T, e0, e1, INFINITY);
}

// A hash that is one task (nb <= kTask) by the whole block: decide here whether the
// median can exceed X (then compute it exactly) and count the local maxima with the final
// threshold, so that such hashes need no median phase after the barrier.  Used by the
// tuning tail, whose small-B trials often need the median (measured slower in the
// location tail, where it rarely does).
__device__ __noinline__ void localmax_whole_hash(const JobView &J, const StatsParams &S, float M,
                                                 float X, int64_t nb)
{
    uint32_t above = 0;
    for (int64_t j = threadIdx.x; j < nb; j += blockDim.x) above += __ldg(&J.E[j]) > X;
    above = block_sum(above);
    float T = S.thr_rel * M;
    if ((int64_t)above > nb - nb / 2 - 1) {
        const uint32_t m = block_median(J.E, (int)nb);
        if (threadIdx.x == 0) {
            J.st->need_median = 1;
            J.st->med_bits = m;
        }
        T = fmaxf(T, S.thr_med * __uint_as_float(m));
    }
    localmax_task(J, S, T, 0, nb, INFINITY);
}

// Exact median (element floor(nb/2) of the ascending energies, as bits) of nb energies
// in global memory by one block: three radix digits (11, 11, 10 bits) over their bit
// patterns, each pass streaming the energies.  The rare path (the median can only matter
// when more than half of the buckets exceed X'); nb <= kSmallMedian goes through
// block_median in shared memory.
__device__ __noinline__ uint32_t block_median_global(const float *E, int64_t nb)
{
    if (nb <= kSmallMedian) return block_median(E, (int)nb);
    extern __shared__ __align__(16) uint32_t dsm[];
    uint32_t *hist = dsm;   // 2048 entries
    __shared__ uint32_t sh_prefix, sh_rank;
    if (threadIdx.x == 0) {
        sh_prefix = 0;
        sh_rank = (uint32_t)(nb / 2);
    }
    __syncthreads();
    const int los[3] = {21, 10, 0}, widths[3] = {11, 11, 10};
    for (int d = 0; d < 3; d++) {
        const int lo = los[d], width = widths[d], hi = lo + width;
        for (int b = threadIdx.x; b < (1 << width); b += blockDim.x) hist[b] = 0;
        __syncthreads();
        const uint32_t prefix = sh_prefix;
        for (int64_t i = threadIdx.x; i < nb; i += blockDim.x) {
            const uint32_t v = __float_as_uint(__ldg(&E[i]));
            if (d == 0 || (v >> hi) == prefix) hist_add(hist, (v >> lo) & ((1u << width) - 1));
        }
        __syncthreads();
        __shared__ uint32_t fb, fr;
        block_find_rank(hist, 1 << width, sh_rank, &fb, &fr);
        if (threadIdx.x == 0) {
            sh_prefix = (prefix << width) | fb;
            sh_rank = fr;
        }
        __syncthreads();
    }
    return sh_prefix;
}

// ---------------------------------------------------------------------------------
// Tuning tail: statistics of every trial of a stage, then the controller.
// ---------------------------------------------------------------------------------

// One trial as the tail kernels see it (passed by value: no dependent loads).
struct TrialView {
    int64_t e_off;         // its energies in the plan's energy buffer
    int32_t logB, slot;
    uint32_t s1, p1, s2, p2;   // sigma and sigma^{-1} mod B per axis
};

struct TuneTailArgs {
    StatsParams S;
    TrialView trial[kMaxLogB];   // this stage's trials, ascending B
    int njobs;
    int stage;             // >= 2: return at once if an earlier stage settled the controller
    int limit_b;           // the controller may visit trials up to this log2 B
    int b0, b_hi, tune_max;
    double delta2;
    const Job *tjob;
    int nh_le, L_loc;
    StatJob *lstat;
    const float2 *z;
    float *energy;         // the plan's energy buffer (tuning region first)
    float *e_loc;
    const HashParam *le;
    ExecState *state;
};

__device__ __forceinline__ JobView trial_view(const TrialView &t, const StatsParams &S,
                                              const float *energy)
{
    JobView v;
    v.E = energy + t.e_off;
    v.st = S.stats + t.slot;
    v.logB = t.logB;
    v.list = -1;
    v.active = 1;
    v.pad = 0;
    v.s1 = t.s1;
    v.p1 = t.p1;
    v.s2 = t.s2;
    v.p2 = t.p2;
    return v;
}

// Records B* = 2^b and k* for the location stage: the state words, the job at B* (all
// nh_le hashes) and the statistics jobs of the location hashes.
__device__ void publish_bstar(const TuneTailArgs &A, int b, int64_t k, int status, int empty,
                              int ntrials)
{
    ExecState *state = A.state;
    state->ntrials = ntrials;
    state->b_star = b;
    state->k_star = k;
    state->status = status;
    state->empty = empty;
    state->tune_done = 1;
    Job j = A.tjob[b];
    j.nh = A.nh_le;
    j.active = !empty;
    state->job = j;
    const int64_t nb = nb_of(A.S.ndim, b);
    for (int l = 0; l < A.L_loc; l++) {
        StatJob s;
        s.spec = A.z + (int64_t)l * nb;
        s.energy = A.e_loc + (int64_t)l * nb;
        s.hash = A.le + l;
        s.logB = b;
        s.slot = kMaxLogB + l;
        s.list = l;
        s.active = !empty;
        A.lstat[l] = s;
    }
}

// One thread walks the trials B0, 2 B0, ... through Eq. (12) and Eq. (14) until the
// stop reading: the first trial with r < delta2 (keep branch, or halve branch onto the
// already evaluated B/2); r = inf when either count is 0; a trial whose energies are
// all exactly 0 ends with k* = 0.  Then it writes the jobs at B*.  A walk that would
// step past limit_b (the trials evaluated so far) writes nothing and leaves tune_done
// at 0 for the next stage, which walks again from B0 over all trials.  Called by the
// first warp of a block: lane t stages trial B0 2^t's counts and its Eq. (12) ratio
// r = |1 - k_t / k_(t-1)| (FP64, slow on this GPU: all trials' divisions at once instead
// of one per step of the walk), then lane 0 walks.
__device__ void controller(const TuneTailArgs &A)
{
    __shared__ uint32_t s_nmax[32], s_maxb[32];
    __shared__ double s_r[32];
    static_assert(kMaxLogB <= 32, "one lane per trial");
    const int lane = threadIdx.x & 31;
    const HashStats *stats = A.S.stats;
    const bool have = lane <= A.b_hi - A.b0;
    const uint32_t kl = have ? __ldcg(&stats[A.b0 + lane].nmax) : 0u;
    const uint32_t kp = __shfl_up_sync(0xffffffffu, kl, 1);
    if (have) {
        s_nmax[lane] = kl;
        s_maxb[lane] = __ldcg(&stats[A.b0 + lane].max_bits);
        s_r[lane] = (kp == 0 || kl == 0) ? INFINITY : fabs(1.0 - (double)kl / (double)kp);
    }
    __syncwarp();
    if (lane != 0) return;
    ExecState *state = A.state;
    int b = A.b0, trial = 0;
    int64_t k = 0;
    int status = state->status, empty = 0;
    for (;; trial++) {
        k = s_nmax[b - A.b0];
        if (trial < kMaxTrialsTrace) {
            state->trial_B[trial] = (int64_t)1 << b;
            state->trial_k[trial] = k;
        }
        if (s_maxb[b - A.b0] == 0) {
            empty = 1;
            k = 0;
            break;
        }
        if (trial > 0 && s_r[b - A.b0] < A.delta2) break;   // r of this trial vs the previous
        if (b == A.b_hi) {
            if (trial > 0 && status == ATSFFT_OK) status = ATSFFT_E_NOT_SPARSE;
            break;
        }
        if (trial + 1 >= A.tune_max) {
            if (status == ATSFFT_OK) status = ATSFFT_E_NOT_CONVERGED;
            break;
        }
        if (b == A.limit_b) return;   // needs the trials of a later stage
        b++;
    }
    if (k == 0) empty = 1;
    publish_bstar(A, b, k, status, empty, trial + 1);
}

// Fixed-k mode: B* and k* come from the plan (no trials); one thread.
__global__ void k_fixed_setup(const TuneTailArgs A, int b, int64_t k)
{
    chain_wait();
    chain_next();
    if (blockIdx.x == 0 && threadIdx.x == 0) publish_bstar(A, b, k, A.state->status, 0, 0);
}

// A trial of more than one statistics task, after all its tasks counted (its last block):
// where the median can matter, the exact median, and the maxima recounted with the
// threshold it gives (the rare path, by this block alone).
__device__ __noinline__ void settle_trial_median(const JobView &J, const StatsParams &S, int64_t nb)
{
    HashStats &st = *J.st;
    if (!(S.use_median && (int64_t)__ldcg(&st.above) > nb - nb / 2 - 1)) return;
    const uint32_t m = block_median_global(J.E, nb);
    if (threadIdx.x == 0) {
        st.need_median = 1;
        st.med_bits = m;
        st.nmax = 0;   // recounted below with the exact threshold
    }
    __threadfence_block();
    __syncthreads();
    const float T = fmaxf(S.thr_rel * __uint_as_float(__ldcg(&st.max_bits)),
                          S.thr_med * __uint_as_float(m));
    for (int64_t e0 = 0; e0 < nb; e0 += kTask) localmax_task_cold(J, S, T, e0, min(e0 + kTask, nb));
}

// Tasks: every trial of at most kTask buckets is one task (settled in one block, median
// included); larger trials are split into tasks of kTask buckets.
__global__ void __launch_bounds__(256) k_tune_tail(const TuneTailArgs A)
{
    pdl_wait();
    pdl_launch_next();
    ExecState *state = A.state;
    if (A.stage >= 2 && state->tune_done) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) stamp(&state->bar);
    __shared__ int64_t tstart[kMaxLogB + 1];
    if (threadIdx.x == 0) {
        int64_t acc = 0;
        for (int jb = 0; jb < A.njobs; jb++) {
            tstart[jb] = acc;
            acc += (nb_of(A.S.ndim, A.trial[jb].logB) + kTask - 1) / kTask;
        }
        tstart[A.njobs] = acc;
    }
    __syncthreads();
    const int64_t ntasks = tstart[A.njobs];
    for (int64_t task = blockIdx.x; task < ntasks; task += gridDim.x) {
        int jb = 0;
        while (task >= tstart[jb + 1]) jb++;
        const JobView J = trial_view(A.trial[jb], A.S, A.energy);
        const int64_t nb = nb_of(A.S.ndim, J.logB);
        const float M = __uint_as_float(J.st->max_bits);
        const float X = A.S.use_median ? M * A.S.ratio : INFINITY;
        if (nb <= kTask) {
            localmax_whole_hash(J, A.S, M, X, nb);
        } else {
            const int64_t e0 = (task - tstart[jb]) * kTask;
            localmax_task(J, A.S, A.S.thr_rel * M, e0, min(e0 + kTask, nb), X);
            const uint32_t units = (uint32_t)(tstart[jb + 1] - tstart[jb]);
            if (finished_last(&state->done[A.trial[jb].slot], units)) settle_trial_median(J, A.S, nb);
        }
        if (finished_last(&state->done_all[A.stage - 1], (uint32_t)ntasks)) {
            if (threadIdx.x < 32) controller(A);
            if (threadIdx.x == 0) stamp(&state->bar);
        }
    }
}

// ---------------------------------------------------------------------------------
// Location tail
// ---------------------------------------------------------------------------------

struct LocTailArgs {
    StatsParams S;
    int L_loc, L_est;
    int est_base;           // first estimation hash in le / z (0 when they reuse location's)
    int est_group;          // lanes per coordinate in the estimates: power of two >= L_est
    float eta_up, eta_dn;
    uint32_t sig[kMaxLoops][2], sinv[kMaxLoops][2];   // the location hashes (by value)
    const float *e_loc;     // location energies at B*: [L_loc][B*] (P-index order)
    int32_t *sel;           // [L_loc][S.cap] selected buckets per location hash
    uint32_t need;          // votes needed: ceil(L_loc / 2)
    uint32_t *bucketbits;   // [L_loc][bucket_words] selected-bucket bitmaps
    int64_t bucket_words;
    uint32_t *kept;         // kept coordinates, unordered (kept_cap entries)
    int64_t kept_cap;
    uint32_t *coordbits;    // one bit per coordinate (all zero between transforms)
    int64_t coord_words;
    uint32_t *chunkcnt;     // kept coordinates per kChunkWords-word chunk of coordbits
    int64_t nchunks;
    int64_t vote_words;     // bitmap words k_loc_votes stages in shared memory (0: none)
    HashParam est[kMaxLoops];   // the estimation hashes (by value)
    const float2 *z;        // spectra at B*: location then estimation hashes
    const float *rgain;     // 1 / Ghat' per B (offsets ro)
    RespOffsets ro;
    const float2 *phase;    // exp(2 pi i m / n) tables, split at phase_s bits
    int phase_s;
    int logn;
    int64_t *loc;
    float2 *val;
    uint8_t *msel;          // optional: median hash indices (real, imaginary) per output
    int skip_est;           // 1: locations only (the FP64 path estimates afterwards)
    int64_t capacity;
    int64_t *d_count, *d_k;
    int32_t *d_status;
    ExecState *state;
};

// k-th smallest (0-based) key among entries i < cnt with pred(i): four 8-bit radix
// passes with a shared histogram.  Whole block must call.
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
            if (pass == 0 || (kk >> (shift + 8)) == prefix) hist_add(hist, (kk >> shift) & 255u);
        }
        __syncthreads();
        __shared__ uint32_t fb, fr;
        block_find_rank(hist, 256, sh_k, &fb, &fr);
        if (threadIdx.x == 0) {
            sh_prefix = (prefix << 8) | fb;
            sh_k = fr;
        }
        __syncthreads();
    }
    return sh_prefix;
}

// k-th smallest (0-based) of the cnt keys key(i) < 2^bits (bits <= 22) in two radix
// passes of up to 11 bits each (2048-bin shared histogram).  Whole block must call.
template <class KeyF>
__device__ uint32_t block_kth_narrow(int cnt, uint32_t k, int bits, KeyF key)
{
    __shared__ uint32_t hist[2048];
    __shared__ uint32_t sh_prefix, sh_k;
    const int lo_bits = bits / 2, hi_bits = bits - lo_bits;
    if (threadIdx.x == 0) {
        sh_prefix = 0;
        sh_k = k;
    }
    for (int pass = 0; pass < 2; pass++) {
        const int shift = pass == 0 ? lo_bits : 0;
        const int width = pass == 0 ? hi_bits : lo_bits;
        for (int b = threadIdx.x; b < 2048; b += blockDim.x) hist[b] = 0;
        __syncthreads();
        const uint32_t prefix = sh_prefix;
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
            const uint32_t kk = key(i);
            if (pass == 0 || (kk >> lo_bits) == prefix) hist_add(hist, (kk >> shift) & ((1u << width) - 1));
        }
        __syncthreads();
        __shared__ uint32_t fb, fr;
        block_find_rank(hist, 1 << width, sh_k, &fb, &fr);
        if (threadIdx.x == 0) {
            sh_prefix = pass == 0 ? fb : ((prefix << lo_bits) | fb);
            sh_k = fr;
        }
        __syncthreads();
    }
    return sh_prefix;
}

constexpr int kTopStage = 4096;

// Top-num cutoff of one location hash by one block: keep every maximum above
// V(1+eta) (V = the num-th largest energy) and fill up from [V(1-eta), V(1+eta)] in
// ascending bucket order.
// The maxima were listed by other blocks: read through L2.
__device__ void topnum_block(int l, int logB, int64_t cnt, const LocTailArgs &A, int64_t num)
{
    __shared__ uint32_t n_sel;
    HashStats &st = A.S.stats[kMaxLogB + l];
    const int ndim = A.S.ndim;
    const uint32_t mask = (1u << logB) - 1;
    const uint32_t p1 = A.sinv[l][0] & mask, p2 = A.sinv[l][1] & mask;
    const int32_t *list = A.S.lists + (int64_t)l * A.S.cap;
    int32_t *out = A.sel + (int64_t)l * A.S.cap;
    const float *E = A.e_loc + ((int64_t)l << (ndim == 1 ? logB : 2 * logB));
    auto energy_global = [&](int64_t i) -> float {
        const uint32_t c = (uint32_t)__ldcg(&list[i]);
        if (ndim == 1) return E[(p1 * c) & mask];
        const uint32_t c1 = c >> logB, c2 = c & mask;
        return E[((int64_t)((p1 * c1) & mask) << logB) | ((p2 * c2) & mask)];
    };
    // the candidates' energies, staged once when they fit
    extern __shared__ __align__(16) uint32_t dsm[];
    float *es = reinterpret_cast<float *>(dsm);   // kTopStage entries
    const bool staged = cnt <= kTopStage;
    if (staged)
        for (int64_t i = threadIdx.x; i < cnt; i += blockDim.x) es[i] = energy_global(i);
    auto energy_of = [&](int64_t i) -> float { return staged ? es[i] : energy_global(i); };
    if (threadIdx.x == 0) n_sel = 0;
    __syncthreads();
    if (cnt <= num) {
        for (int64_t i = threadIdx.x; i < cnt; i += blockDim.x) out[i] = __ldcg(&list[i]);
        if (threadIdx.x == 0) n_sel = (uint32_t)cnt;
    } else {
        const uint32_t vb = ~block_kth(
            cnt, (uint32_t)(num - 1), [&](int64_t i) { return ~__float_as_uint(energy_of(i)); },
            [&](int64_t) { return true; });
        const float V = __uint_as_float(vb);
        const float hi = V * A.eta_up, lo = V * A.eta_dn;
        uint32_t mine = 0;
        for (int64_t i = threadIdx.x; i < cnt; i += blockDim.x) mine += energy_of(i) > hi;
        const uint32_t nhi = block_sum(mine);
        const uint32_t need = (uint32_t)num - nhi;
        const uint32_t cthr = block_kth(
            cnt, need - 1, [&](int64_t i) { return (uint32_t)__ldcg(&list[i]); },
            [&](int64_t i) {
                const float e = energy_of(i);
                return e >= lo && e <= hi;
            });
        // the kept maxima, appended with one shared atomic per warp and round
        const int lane = threadIdx.x & 31;
        for (int64_t i0 = 0; i0 < cnt; i0 += blockDim.x) {
            const int64_t i = i0 + threadIdx.x;
            bool keep = false;
            if (i < cnt) {
                const float e = energy_of(i);
                keep = e > hi || (e >= lo && e <= hi && (uint32_t)__ldcg(&list[i]) <= cthr);
            }
            const unsigned bal = __ballot_sync(0xffffffffu, keep);
            uint32_t base = 0;
            if (lane == 0 && bal) base = atomicAdd(&n_sel, (uint32_t)__popc(bal));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (keep) out[base + __popc(bal & ((1u << lane) - 1))] = __ldcg(&list[i]);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) st.nsel = n_sel;
    __syncthreads();
}

// Eq. (11) for coordinate `coord` and estimation hash l: the bucket value times the
// phase exp(2 pi i m / n) (m from exact integer index arithmetic) divided by the window
// gain Ghat'(o) (as a reciprocal from the plan's FP64 table).
__device__ float2 estimate_term(uint64_t coord, const LocTailArgs &A, int b, int l)
{
    const int64_t nb = nb_of(A.S.ndim, b);
    const float2 *Pz = A.z + (int64_t)(A.est_base + l) * nb;
    int64_t idx;
    const float2 c = estimate_coef(coord, A.est[l], A.S.ndim, A.logn, b,
                                   A.rgain + A.ro.off[b], A.phase, A.phase_s, &idx);
    return cmul(Pz[idx], c);
}

// Componentwise median (element floor(L/2) of each sorted component; equal values
// ordered by hash index) of the values v held by lanes 0..L-1 of a group of grp lanes:
// each lane ranks its own value against the group's by shuffles, and the lane of rank
// floor(L/2) stores that component to *out (and, with sel != nullptr, its hash index to
// sel[0] for the real part, sel[1] for the imaginary part).  All lanes of the warp must
// call.
__device__ __forceinline__ void group_median(float2 v, int L, int grp, bool valid, float2 *out,
                                             uint8_t *sel)
{
    const int gl = (int)(threadIdx.x & 31) & (grp - 1);
    int rr = 0, ri = 0;
    for (int c = 0; c < L; c++) {
        const float xr = __shfl_sync(0xffffffffu, v.x, c, grp);
        const float xi = __shfl_sync(0xffffffffu, v.y, c, grp);
        rr += xr < v.x || (xr == v.x && c < gl);
        ri += xi < v.y || (xi == v.y && c < gl);
    }
    if (valid && gl < L) {
        if (rr == L / 2) {
            out->x = v.x;
            if (sel) sel[0] = (uint8_t)gl;
        }
        if (ri == L / 2) {
            out->y = v.y;
            if (sel) sel[1] = (uint8_t)gl;
        }
    }
}

// Bucket of coordinate i under hash hp on one axis (Eq. (10) with the half-bin reading):
// round((sigma i mod n + 1/2) / D) mod B.
__device__ __forceinline__ uint32_t bucket_of(uint32_t i, uint32_t sigma, int logn, int logB)
{
    const uint32_t nmask = (1u << logn) - 1, D = 1u << (logn - logB);
    const uint32_t p = (sigma * i) & nmask;   // 2p + 1 + D < 2^30 for n <= 2^28
    return ((2u * p + 1u + D) >> (logn - logB + 1)) & ((1u << logB) - 1);
}

constexpr int kRankStage = 4096;   // top-num by ranking: candidates staged in shared memory
constexpr int kPivots = 32;   // one warp: lane p holds pivot p
constexpr int kSelCluster = 8;     // CTAs per location hash in k_loc_select (one cluster)
constexpr int kSelThreads = 512;   // threads per CTA of k_loc_select
constexpr int64_t kSelTask = kTask * kSelThreads / 256;   // buckets per task of k_loc_select
constexpr int kVoteThreads = 1024; // k_loc_votes: one CTA per SM
constexpr int kVoteIlp = 2;        // candidates per thread per round of the votes
constexpr int kVoteSmem = 96 * 1024;   // largest bitmap staging of k_loc_votes (bytes)
constexpr int kVoteKeep = 2048;    // kept coordinates a CTA of k_loc_votes collects before
                                   // reserving their places in the kept list at once

// Value of descending rank r (0-based; equal values ordered by index) among es[0..cnt),
// by the whole block.  kPivots sampled values are counted against all elements (every
// thread against all pivots); only the elements between the two pivots that bracket
// rank r are then ranked exactly, one thread per element.  scratch: cnt entries of
// shared memory.
__device__ __noinline__ float block_select_desc(const float *es, int cnt, uint32_t r, uint32_t *scratch)
{
    __shared__ float pv[kPivots];
    __shared__ uint32_t pg[kPivots];
    __shared__ float lo_sh, hi_sh, v_sh;
    __shared__ uint32_t nbr;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    static_assert(kPivots == 32, "the reduce-scatter leaves pivot p in lane p");
    if (threadIdx.x < kPivots) {
        pv[threadIdx.x] = es[(int64_t)threadIdx.x * cnt / kPivots];
        pg[threadIdx.x] = 0;
    }
    if (threadIdx.x == 0) nbr = 0;
    __syncthreads();
    // g[p] = #{e > pv[p]}: every thread counts its elements against all pivots (held in
    // registers), a reduce-scatter over the warp leaves pivot p's warp total in lane p
    {
        float pr[kPivots];
        uint32_t c[kPivots];
#pragma unroll
        for (int p = 0; p < kPivots; p++) {
            pr[p] = pv[p];
            c[p] = 0;
        }
        for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
            const float e = es[j];
#pragma unroll
            for (int p = 0; p < kPivots; p++) c[p] += e > pr[p];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const bool upper = (lane & o) != 0;
#pragma unroll
            for (int i = 0; i < o; i++) {
                const uint32_t send = upper ? c[i] : c[i + o];
                const uint32_t keep = upper ? c[i + o] : c[i];
                c[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
            }
        }
        atomicAdd(&pg[lane], c[0]);
    }
    __syncthreads();
    __shared__ uint32_t above_u;
    if (warp == 0) {
        // V lies in (L, U]: L the largest pivot with >= r + 1 elements above it, U the
        // smallest pivot with <= r elements above it (lane p holds pivot p)
        const float v = pv[lane];
        const uint32_t g = pg[lane];
        float L = g >= r + 1 ? v : -INFINITY, U = g >= r + 1 ? INFINITY : v;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            L = fmaxf(L, __shfl_xor_sync(0xffffffffu, L, o));
            U = fminf(U, __shfl_xor_sync(0xffffffffu, U, o));
        }
        // every element outside (L, U] is either above U (g(U) of them) or at most L, so
        // a bracket member's rank is g(U) plus its rank inside the bracket
        const unsigned at_u = __ballot_sync(0xffffffffu, v == U);
        const uint32_t gu = __shfl_sync(0xffffffffu, g, at_u ? __ffs(at_u) - 1 : 0);
        if (lane == 0) {
            lo_sh = L;
            hi_sh = U;
            above_u = U == INFINITY ? 0u : gu;
        }
    }
    __syncthreads();
    const float L = lo_sh, U = hi_sh;
    for (int i0 = 0; i0 < cnt; i0 += blockDim.x) {
        const int i = i0 + threadIdx.x;
        const bool in = i < cnt && es[i] > L && es[i] <= U;
        const unsigned bal = __ballot_sync(0xffffffffu, in);
        uint32_t base = 0;
        if (lane == 0 && bal) base = atomicAdd(&nbr, (uint32_t)__popc(bal));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (in) scratch[base + __popc(bal & ((1u << lane) - 1))] = (uint32_t)i;
    }
    __syncthreads();
    const int nb = (int)nbr;
    for (int m = threadIdx.x; m < nb; m += blockDim.x) {
        const int i = (int)scratch[m];
        const float e = es[i];
        uint32_t rk = above_u;
        for (int q = 0; q < nb; q++) {
            const int j = (int)scratch[q];
            const float f = es[j];
            rk += f > e || (f == e && j < i);
        }
        if (rk == r) v_sh = e;
    }
    __syncthreads();
    return v_sh;
}

// Keeps, in place and in order, the listed maxima (bucket, energy) of one hash whose
// energy exceeds T; returns how many.  Whole block; the entries were written by other
// blocks (read through L2).
__device__ int64_t filter_list(int32_t *list, float *list_e, int64_t cnt, float T)
{
    __shared__ uint32_t tot;
    int64_t base = 0;
    for (int64_t i0 = 0; i0 < cnt; i0 += blockDim.x) {
        const int64_t i = i0 + threadIdx.x;
        int32_t c = 0;
        float e = 0.f;
        if (i < cnt) {
            c = __ldcg(&list[i]);
            e = __ldcg(&list_e[i]);
        }
        const bool keep = i < cnt && e > T;
        // (the scan synchronises: every read of this chunk precedes every write, and a
        // kept entry only moves down)
        const uint32_t ex = block_exclusive_scan(keep ? 1u : 0u, &tot);
        if (keep) {
            list[base + ex] = c;
            list_e[base + ex] = e;
        }
        base += tot;
        __syncthreads();
    }
    return base;
}

// Thread-block clusters: rank and size of the calling CTA's cluster, shared-memory
// addresses in another CTA of the cluster (distributed shared memory) and the cluster
// barrier, split into arrive and wait.
__device__ __forceinline__ uint32_t cluster_ctarank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_nctarank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_addr(const void *p, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;"
                 : "=r"(r)
                 : "r"((uint32_t)__cvta_generic_to_shared(p)), "r"(rank));
    return r;
}
__device__ __forceinline__ void st_cluster(uint32_t addr, uint32_t v)
{
    asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t atom_add_cluster(uint32_t addr, uint32_t v)
{
    uint32_t old;
    asm volatile("atom.shared::cluster.add.u32 %0, [%1], %2;" : "=r"(old) : "r"(addr), "r"(v) : "memory");
    return old;
}
__device__ __forceinline__ void red_add_cluster(uint32_t addr, uint32_t v)
{
    asm volatile("red.shared::cluster.add.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
// (release: this thread's earlier memory operations, shared, distributed shared and
// global, are visible to the cluster's threads after their matching wait)
__device__ __forceinline__ void cluster_arrive()
{
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait()
{
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Layout of the dynamic shared memory of k_loc_select (words): the gathered maxima, energy
// bits es[0, kRankStage) and buckets cs[kRankStage, 2 kRankStage); an auxiliary region
// aux[2 kRankStage, 3 kRankStage): the coarse and the fine energy histograms (kDigitBins
// words each), later the band list; and the band bitmap [3 kRankStage, 4 kRankStage).
constexpr int kDigitBins = 2048;
static_assert(2 * kDigitBins <= kRankStage, "both histograms fit the auxiliary region");
constexpr size_t kSelSmem = sizeof(uint32_t) * 4 * kRankStage;

// Selection key of a maximum of energy e below the hash's maximum energy maxE (both > 0:
// their bit patterns order like their values): key = bits(maxE) - bits(e), ascending
// with descending energy; its coarse digit is key >> 16, clamped to the last bin.
__device__ __forceinline__ uint32_t coarse_digit(uint32_t key)
{
    return min(key >> 16, (uint32_t)kDigitBins - 1);
}

// Top-num cutoff of location hash l (Algorithm 1 "find num largest") from its cnt local
// maxima staged in shared memory (cnt <= kRankStage, cnt > num), by one block: V = the
// num-th largest energy; every maximum above V(1+eta) is kept and the band
// [V(1-eta), V(1+eta)] fills up in ascending bucket order.  The kept buckets go to the
// hash's selection list and bitmap (cleared before).  V is found from the coarse digit
// histogram (have_hist: summed by the cluster while the maxima were gathered, and the
// fine histograms and band bitmap already zero; else built here), one fine pass over the
// 11 digits below the coarse one and a 32-bin pass over the last 5 bits; the band's
// cutoff bucket from a bitmap of the band buckets by a block prefix popcount.
__device__ __noinline__ void cutoff_staged(const LocTailArgs &A, int l, int b, int64_t num, int cnt,
                                           uint32_t mbits, bool have_hist)
{
    extern __shared__ __align__(16) uint32_t dsm[];
    const int ndim = A.S.ndim;
    const int lane = threadIdx.x & 31;
    HashStats &st = A.S.stats[kMaxLogB + l];
    uint32_t *bits = A.bucketbits + (int64_t)l * A.bucket_words;
    int32_t *out = A.sel + (int64_t)l * A.S.cap;
    const uint32_t *eb = dsm;   // energy bits
    const float *es = reinterpret_cast<const float *>(dsm);
    const uint32_t *cs = dsm + kRankStage;   // buckets
    uint32_t *aux = dsm + 2 * kRankStage;
    uint32_t *h1 = aux, *h2 = aux + kDigitBins;
    uint32_t *bandbits = dsm + 3 * kRankStage;
    const int64_t words = (nb_of(ndim, b) + 31) >> 5;
    const bool use_bitmap = words <= kRankStage;
    __shared__ uint32_t n_sel, nband, fb, fr, cthr;
    __shared__ uint32_t h3[32];
    if (threadIdx.x == 0) {
        n_sel = 0;
        nband = 0;
    }
    if (threadIdx.x < 32) h3[threadIdx.x] = 0;
    if (!have_hist) {
        for (int i = threadIdx.x; i < 2 * kDigitBins; i += blockDim.x) h1[i] = 0;   // h1, h2
        if (use_bitmap)
            for (int64_t w = threadIdx.x; w < words; w += blockDim.x) bandbits[w] = 0u;
        __syncthreads();
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) hist_add(h1, coarse_digit(mbits - eb[i]));
        __syncthreads();
    }
    // V: the key of ascending rank num - 1
    const uint32_t r = (uint32_t)(num - 1);
    block_find_rank(h1, kDigitBins, r, &fb, &fr);
    const uint32_t beta = fb, r1 = fr;
    float V;
    if (beta == (uint32_t)kDigitBins - 1) {
        // (V more than 2^-16 below maxE: the clamped bin, only with a threshold far below
        // the default) the generic selection
        V = block_select_desc(es, cnt, r, aux);
    } else {
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
            const uint32_t key = mbits - eb[i];
            if ((key >> 16) == beta) hist_add(h2, (key >> 5) & (kDigitBins - 1));
        }
        __syncthreads();
        block_find_rank(h2, kDigitBins, r1, &fb, &fr);
        const uint32_t pre = (beta << 11) | fb, r2 = fr;
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
            const uint32_t key = mbits - eb[i];
            if ((key >> 5) == pre) hist_add(h3, key & 31u);
        }
        __syncthreads();
        // every warp reads the 32 bins and finds the one of rank r2
        const uint32_t v = h3[lane];
        const uint32_t incl = warp_incl_scan(v);
        const unsigned at = __ballot_sync(0xffffffffu, v && r2 >= incl - v && r2 < incl);
        V = __uint_as_float(mbits - ((pre << 5) | (uint32_t)(__ffs(at) - 1)));
    }
    const float hi = V * A.eta_up, lo = V * A.eta_dn;
    uint32_t mine = 0;
    for (int i0 = 0; i0 < cnt; i0 += blockDim.x) {
        const int i = i0 + threadIdx.x;
        const float e = i < cnt ? es[i] : 0.f;
        mine += i < cnt && e > hi;
        const bool in = i < cnt && e >= lo && e <= hi;
        if (use_bitmap) {
            if (in) atomicOr(&bandbits[cs[i] >> 5], 1u << (cs[i] & 31));
        } else {
            // the band's buckets listed (one shared atomic per warp)
            const unsigned bal = __ballot_sync(0xffffffffu, in);
            uint32_t base = 0;
            if (lane == 0 && bal) base = atomicAdd(&nband, (uint32_t)__popc(bal));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (in) aux[base + __popc(bal & ((1u << lane) - 1))] = cs[i];
        }
    }
    const uint32_t nhi = block_sum(mine);   // (synchronises: the band complete)
    const uint32_t need_band = (uint32_t)num - nhi;   // >= 1: V itself is in the band
    // the need_band-th smallest band bucket
    uint32_t ct;
    if (use_bitmap) {
        const int64_t per = words >= (int64_t)blockDim.x ? words / blockDim.x : 1;
        const int64_t w0 = (int64_t)threadIdx.x * per;
        uint32_t sum = 0;
        if (w0 < words)
            for (int64_t k = 0; k < per; k++) sum += __popc(bandbits[w0 + k]);
        uint32_t all;
        const uint32_t before = block_scan_core(sum, all);
        const uint32_t rk = need_band - 1;
        if (sum && rk >= before && rk < before + sum) {
            uint32_t cum = before;
            for (int64_t k = 0; k < per; k++) {
                const uint32_t w = bandbits[w0 + k], pc = (uint32_t)__popc(w);
                if (rk < cum + pc) {
                    cthr = (uint32_t)(w0 + k) * 32u + __fns(w, 0, (int)(rk - cum) + 1);
                    break;
                }
                cum += pc;
            }
        }
        __syncthreads();
        ct = cthr;
    } else {
        const uint32_t nbd = nband;
        const int kbits = ndim == 1 ? b : 2 * b;   // bucket indices < B (B^2 in 2D)
        if (kbits <= 22)
            ct = block_kth_narrow((int)nbd, need_band - 1, kbits, [&](int i) { return aux[i]; });
        else
            ct = block_kth((int64_t)nbd, need_band - 1, [&](int64_t i) { return aux[i]; },
                           [](int64_t) { return true; });
    }
    for (int i0 = 0; i0 < cnt; i0 += blockDim.x) {
        const int i = i0 + threadIdx.x;
        bool keep = false;
        uint32_t c = 0;
        if (i < cnt) {
            const float e = es[i];
            c = cs[i];
            keep = e > hi || (e >= lo && e <= hi && c <= ct);
        }
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        uint32_t base = 0;
        if (lane == 0 && bal) base = atomicAdd(&n_sel, (uint32_t)__popc(bal));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (keep) {
            out[base + __popc(bal & ((1u << lane) - 1))] = (int32_t)c;
            atomicOr(&bits[c >> 5], 1u << (c & 31));
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) st.nsel = n_sel;
}

// The cutoff of hash l from its maxima list in global memory (cnt entries), by one
// block: the rare paths of k_loc_select.  With `median` the exact median first (it can
// only matter when more than half of the energies exceed X: it may raise the threshold,
// and the listed maxima below the new one drop out); more maxima than kRankStage go to
// the radix selection over the list; otherwise the list is staged and cut as usual.
__device__ __noinline__ void cutoff_global(const LocTailArgs &A, int l, int b, int64_t num,
                                           int64_t cnt, bool median)
{
    extern __shared__ __align__(16) uint32_t dsm[];
    const int ndim = A.S.ndim;
    const int64_t nb = nb_of(ndim, b);
    HashStats &st = A.S.stats[kMaxLogB + l];
    int32_t *list = A.S.lists + (int64_t)l * A.S.cap;
    float *list_e = A.S.list_e + (int64_t)l * A.S.cap;
    uint32_t *bits = A.bucketbits + (int64_t)l * A.bucket_words;
    int32_t *out = A.sel + (int64_t)l * A.S.cap;
    cnt = min(cnt, A.S.cap);
    if (median) {
        const uint32_t m = block_median_global(A.e_loc + (int64_t)l * nb, nb);
        const float T = fmaxf(A.S.thr_rel * __uint_as_float(__ldcg(&st.max_bits)),
                              A.S.thr_med * __uint_as_float(m));
        cnt = filter_list(list, list_e, cnt, T);
        if (threadIdx.x == 0) {
            st.need_median = 1;
            st.med_bits = m;
            st.nmax = (uint32_t)cnt;
        }
        __syncthreads();
    }
    if (cnt <= num) {
        // every maximum is kept: the list is the selection
        for (int64_t i = threadIdx.x; i < cnt; i += blockDim.x) {
            const uint32_t c = (uint32_t)__ldcg(&list[i]);
            out[i] = (int32_t)c;
            atomicOr(&bits[c >> 5], 1u << (c & 31));
        }
        if (threadIdx.x == 0) st.nsel = (uint32_t)cnt;
        return;
    }
    if (cnt > kRankStage) {
        // more maxima than stage: radix selection, then the bitmap
        topnum_block(l, b, cnt, A, num);
        const int64_t ns = st.nsel;
        for (int64_t i = threadIdx.x; i < ns; i += blockDim.x) {
            const uint32_t c = (uint32_t)out[i];
            atomicOr(&bits[c >> 5], 1u << (c & 31));
        }
        return;
    }
    for (int64_t i = threadIdx.x; i < cnt; i += blockDim.x) {
        dsm[kRankStage + i] = (uint32_t)__ldcg(&list[i]);
        dsm[i] = __float_as_uint(__ldcg(&list_e[i]));
    }
    __syncthreads();
    cutoff_staged(A, l, b, num, (int)cnt, __ldcg(&st.max_bits), false);
}

__device__ __forceinline__ JobView loc_view(const LocTailArgs &A, int l, int b)
{
    const uint32_t mask = (1u << b) - 1;
    JobView v;
    v.E = A.e_loc + ((int64_t)l << (A.S.ndim == 1 ? b : 2 * b));
    v.st = A.S.stats + kMaxLogB + l;
    v.logB = b;
    v.list = l;
    v.active = 1;
    v.pad = 0;
    v.s1 = A.sig[l][0] & mask;
    v.p1 = A.sinv[l][0] & mask;
    v.s2 = A.sig[l][1] & mask;
    v.p2 = A.sinv[l][1] & mask;
    return v;
}

// Thresholds, local maxima and top-num cutoff of the L_loc location hashes at B*: one
// thread-block cluster per hash.  Every CTA of the cluster takes a contiguous range of
// P-indices (tasks of kSelTask buckets) and clears its share of the hash's bucket bitmap;
// the maxima it finds go straight into the shared memory of the cluster's first CTA, at
// positions taken from a counter there (distributed shared memory; positions beyond
// kRankStage go to the hash's list in global memory, at the same positions), and the
// coarse digits of their selection keys into a histogram, summed into the first CTA's.
// After the cluster barrier the first CTA holds them all and makes the cutoff.
__global__ void __launch_bounds__(kSelThreads) k_loc_select(const LocTailArgs A)
{
    pdl_wait();
    pdl_launch_next();
    __shared__ uint32_t sh_cnt, sh_above, sh_base, sh_tot;
    extern __shared__ __align__(16) uint32_t dsm[];
    uint32_t *hist = dsm + 2 * kRankStage;   // coarse digits of this CTA's maxima
    const uint32_t rank = cluster_ctarank(), csize = cluster_nctarank();
    const int l = (int)(blockIdx.x / csize);
    if (l >= A.L_loc) return;   // (whole clusters: the grid is L_loc clusters)
    ExecState *state = A.state;
    if (blockIdx.x == 0 && threadIdx.x == 0) stamp(&state->bar);
    // zero: every CTA its coarse histogram; the first CTA also its fine histogram and band
    // bitmap (used by its cutoff)
    for (int i = threadIdx.x; i < (rank == 0 ? 2 * kRankStage : kDigitBins); i += blockDim.x) hist[i] = 0;
    if (threadIdx.x == 0) {
        sh_cnt = 0;
        sh_above = 0;
    }
    cluster_arrive();   // the first CTA's counters and histogram are zero before any adds
    const int empty = state->empty;
    const int b = state->b_star;
    const int64_t num = state->k_star;
    const JobView J = loc_view(A, l, b);
    const uint32_t mbits = J.st->max_bits;
    cluster_wait();
    if (empty) return;   // (the same in every CTA: nothing else touches the cluster)
    const int ndim = A.S.ndim;
    const int64_t nb = nb_of(ndim, b);
    uint32_t *bits = A.bucketbits + (int64_t)l * A.bucket_words;
    const int64_t words = (nb + 31) >> 5;
    for (int64_t w = words * rank / csize + threadIdx.x; w < words * (rank + 1) / csize; w += blockDim.x)
        bits[w] = 0u;
    int32_t *list = A.S.lists + (int64_t)l * A.S.cap;
    float *list_e = A.S.list_e + (int64_t)l * A.S.cap;
    const uint32_t es_r = cluster_addr(dsm, 0), cs_r = cluster_addr(dsm + kRankStage, 0);
    const float M = __uint_as_float(mbits);
    const float X = A.S.use_median ? M * A.S.ratio : INFINITY;
    const float T = A.S.thr_rel * M;
    uint32_t above_all = 0;
    for (int64_t e0 = nb * rank / csize, r1 = nb * (rank + 1) / csize; e0 < r1; e0 += kSelTask) {
        float ev[kPerTask];
        uint32_t found, above;
        localmax_scan<kSelThreads>(J, A.S, T, e0, min(e0 + kSelTask, r1), X, ev, found, above);
        above_all += above;
        const uint32_t before = block_exclusive_scan((uint32_t)__popc(found), &sh_tot);
        if (threadIdx.x == 0) sh_base = sh_tot ? atom_add_cluster(cluster_addr(&sh_cnt, 0), sh_tot) : 0u;
        __syncthreads();
        uint32_t pos = sh_base + before;
#pragma unroll
        for (int u = 0; u < kPerTask; u++) {
            if (!(found & (1u << u))) continue;
            const int32_t c = bucket_of_pindex(J, ndim, e0 + threadIdx.x + kSelThreads * u);
            const uint32_t eb = __float_as_uint(ev[u]);
            hist_add(hist, coarse_digit(mbits - eb));
            if (pos < (uint32_t)kRankStage) {
                st_cluster(es_r + 4 * pos, eb);
                st_cluster(cs_r + 4 * pos, (uint32_t)c);
            } else if (pos < A.S.cap) {
                list[pos] = c;
                list_e[pos] = ev[u];
            }
            pos++;
        }
    }
    const uint32_t nabove = block_sum(above_all);   // (synchronises: this CTA's histogram is complete)
    if (rank != 0) {
        const uint32_t h_r = cluster_addr(hist, 0);
        for (int i = threadIdx.x; i < kDigitBins; i += blockDim.x) {
            const uint32_t v = hist[i];
            if (v) red_add_cluster(h_r + 4 * i, v);
        }
    }
    if (threadIdx.x == 0 && nabove) red_add_cluster(cluster_addr(&sh_above, 0), nabove);
    cluster_arrive();   // this CTA's maxima, counts, digits and bitmap clears, for the first CTA
    if (rank != 0) return;
    cluster_wait();
    HashStats &st = *J.st;
    const uint32_t cnt = sh_cnt, above = sh_above;
    if (threadIdx.x == 0) {
        st.nmax = cnt;
        st.above = above;
    }
    const bool median = A.S.use_median && (int64_t)above > nb - nb / 2 - 1;
    if (median || cnt > (uint32_t)kRankStage) {
        // rare: the whole list in global memory first (the staged part is this CTA's)
        const uint32_t ns = min(cnt, (uint32_t)kRankStage);
        for (uint32_t i = threadIdx.x; i < ns; i += blockDim.x) {
            list[i] = (int32_t)dsm[kRankStage + i];
            list_e[i] = __uint_as_float(dsm[i]);
        }
        __syncthreads();
        cutoff_global(A, l, b, num, (int64_t)cnt, median);
        return;
    }
    if ((int64_t)cnt <= num) {
        // every maximum is kept: the list is the selection
        int32_t *out = A.sel + (int64_t)l * A.S.cap;
        for (uint32_t i = threadIdx.x; i < cnt; i += blockDim.x) {
            const uint32_t c = dsm[kRankStage + i];
            out[i] = (int32_t)c;
            atomicOr(&bits[c >> 5], 1u << (c & 31));
        }
        if (threadIdx.x == 0) st.nsel = cnt;
        return;
    }
    cutoff_staged(A, l, b, num, (int)cnt, mbits, true);
}

// Geometry of the votes at B* = 2^b (per axis): D = n / B preimages per bucket and axis.
struct VoteGeom {
    int b, logn, logD, logDd, lw, L_loc;
    uint32_t need, nmask, Bm, Dh;   // Dh = D / 2
    uint32_t cap;                    // selection list stride (L_loc x cap < 2^31)
};

// Votes of the candidates it = base + u * stride (u < kVoteIlp) below `total`: candidate
// it is preimage q of the s-th selected bucket of hash l0 (off[l0] <= it < off[l0 + 1]);
// it is kept when >= need of the L_loc hashes selected its bucket and none of the hashes
// before l0 did (so that it is emitted once).  STAGED: the bitmaps are in shared memory
// (L_loc x 2^lw words), else read through the read-only cache.
template <int NDIM, bool STAGED>
__device__ __forceinline__ void vote_round(const LocTailArgs &A, const VoteGeom &G,
                                           const uint32_t *bm, const uint32_t *off,
                                           const uint32_t (*sig)[2], const uint32_t (*sinv)[2],
                                           int L_cand, uint32_t base, uint32_t stride,
                                           uint32_t total, uint32_t *keep_s, uint32_t *keep_n)
{
    const int lane = threadIdx.x & 31;
    uint32_t coord[kVoteIlp], cb[kVoteIlp], qv[kVoteIlp];
    int l0v[kVoteIlp];
#pragma unroll
    for (int u = 0; u < kVoteIlp; u++) {
        const uint32_t it = base + (uint32_t)u * stride;
        l0v[u] = -1;
        cb[u] = qv[u] = 0;
        if (it < total) {
            int l0 = 0;
            while (l0 + 1 < L_cand && it >= off[l0 + 1]) l0++;
            const uint32_t rem = it - off[l0];
            qv[u] = rem & ((1u << G.logDd) - 1);
            cb[u] = (uint32_t)__ldg(&A.sel[(uint32_t)l0 * G.cap + (rem >> G.logDd)]);
            l0v[u] = l0;
        }
    }
    // the preimage: bucket c collects permuted positions p in [c D - D/2, c D + D/2 - 1]
#pragma unroll
    for (int u = 0; u < kVoteIlp; u++) {
        const int l0 = l0v[u] < 0 ? 0 : l0v[u];
        const uint32_t c = cb[u], q = qv[u];
        if (NDIM == 1) {
            const uint32_t pp = ((c << G.logD) - G.Dh + q) & G.nmask;
            coord[u] = (sinv[l0][0] * pp) & G.nmask;
        } else {
            const uint32_t c1 = c >> G.b, c2 = c & G.Bm;
            const uint32_t q1 = q >> G.logD, q2 = q & ((1u << G.logD) - 1);
            const uint32_t pp1 = ((c1 << G.logD) - G.Dh + q1) & G.nmask;
            const uint32_t pp2 = ((c2 << G.logD) - G.Dh + q2) & G.nmask;
            coord[u] = (((sinv[l0][0] * pp1) & G.nmask) << G.logn) | ((sinv[l0][1] * pp2) & G.nmask);
        }
    }
    uint32_t votes[kVoteIlp], earlier[kVoteIlp];
#pragma unroll
    for (int u = 0; u < kVoteIlp; u++) votes[u] = earlier[u] = 0;
    // bucket of i under sigma (the half-bin rule of bucket_of, in three operations):
    // floor((2p + 1 + D) / 2D) mod B = ((sigma i + D/2) mod n) >> log2 D, p = sigma i mod n
#pragma unroll 4
    for (int l = 0; l < G.L_loc; l++) {
        const uint32_t s0 = sig[l][0], s1 = NDIM == 2 ? sig[l][1] : 0u;
#pragma unroll
        for (int u = 0; u < kVoteIlp; u++) {
            const uint32_t ci = NDIM == 1 ? coord[u] : coord[u] >> G.logn;
            uint32_t c_l = ((s0 * ci + G.Dh) & G.nmask) >> G.logD;
            if (NDIM == 2) c_l = (c_l << G.b) | (((s1 * (coord[u] & G.nmask) + G.Dh) & G.nmask) >> G.logD);
            const uint32_t w = STAGED ? bm[((uint32_t)l << G.lw) + (c_l >> 5)]
                                      : __ldg(&A.bucketbits[(int64_t)l * A.bucket_words + (c_l >> 5)]);
            const uint32_t sel = (w >> (c_l & 31)) & 1u;
            votes[u] += sel;
            earlier[u] |= sel & (uint32_t)(l < l0v[u]);
        }
    }
    // the kept ones: into the CTA's list (one shared atomic per warp); beyond its
    // kVoteKeep entries, straight into the kept list (one global atomic per warp)
    ExecState *state = A.state;
    const unsigned below = (1u << lane) - 1;
#pragma unroll
    for (int u = 0; u < kVoteIlp; u++) {
        const bool keep = l0v[u] >= 0 && !earlier[u] && votes[u] >= G.need;
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        if (!bal) continue;
        const int lead = __ffs(bal) - 1;
        uint32_t lb = 0;
        if (lane == lead) lb = atomicAdd(keep_n, (uint32_t)__popc(bal));
        const uint32_t li = __shfl_sync(0xffffffffu, lb, lead) + __popc(bal & below);
        const unsigned ovf = __ballot_sync(0xffffffffu, keep && li >= (uint32_t)kVoteKeep);
        uint32_t gb = 0;
        if (ovf) {
            if (lane == __ffs(ovf) - 1)
                gb = (uint32_t)atomicAdd((unsigned long long *)&state->count,
                                         (unsigned long long)__popc(ovf));
            gb = __shfl_sync(0xffffffffu, gb, __ffs(ovf) - 1);
        }
        if (keep) {
            if (li < (uint32_t)kVoteKeep) {
                keep_s[li] = coord[u];
            } else {
                const uint32_t pos = gb + __popc(ovf & below);
                if (pos < A.kept_cap) A.kept[pos] = coord[u];
            }
            atomicOr(&A.coordbits[coord[u] >> 5], 1u << (coord[u] & 31));
            atomicAdd(&A.chunkcnt[coord[u] >> (5 + 10)], 1u);
        }
    }
}

// Votes.  A kept coordinate lies in >= need selected buckets, hence in a selected bucket
// of one of the first L_cand = L_loc - need + 1 hashes; every preimage of those hashes'
// selected buckets counts the hashes whose bucket of it is selected and is emitted once,
// by the first hash that has it.  One CTA per SM: the bitmaps of the L_loc hashes are
// staged in its shared memory when they fit (vote_words > 0), and the candidates are
// spread evenly over all threads (consecutive lanes: consecutive preimages of a bucket).
// The selections and bitmaps were written by the previous kernel: read-only here.
template <int NDIM>
__global__ void __launch_bounds__(kVoteThreads) k_loc_votes(const LocTailArgs A)
{
    pdl_wait();
    pdl_launch_next();
    ExecState *state = A.state;
    if (blockIdx.x == 0 && threadIdx.x == 0) stamp(&state->bar);
    if (state->empty) return;
    extern __shared__ __align__(16) uint32_t bm[];
    __shared__ uint32_t off[kMaxLoops + 1];
    __shared__ uint32_t sh_sig[kMaxLoops][2], sh_sinv[kMaxLoops][2];
    __shared__ uint32_t keep_s[kVoteKeep], keep_n, keep_base;
    VoteGeom G;
    G.b = state->b_star;
    G.logn = A.logn;
    G.logD = A.logn - G.b;
    G.logDd = NDIM == 1 ? G.logD : 2 * G.logD;
    G.lw = max((NDIM == 1 ? G.b : 2 * G.b) - 5, 0);   // bitmap words per hash: 2^lw
    G.L_loc = A.L_loc;
    G.need = A.need;
    G.nmask = (uint32_t)((1ull << A.logn) - 1);
    G.Bm = (1u << G.b) - 1;
    G.Dh = 1u << (G.logD - 1);
    G.cap = (uint32_t)A.S.cap;
    const int L_cand = A.L_loc - (int)A.need + 1;
    if (threadIdx.x < 32) {
        // the candidate counts of the first L_cand hashes (< 2^32 in all: at most 16
        // hashes of B/2 (1D) or B^2/4 (2D) selected buckets of n/B or N^2/B^2 preimages),
        // loaded by one lane each and summed by a warp scan
        static_assert(kMaxLoops <= 32, "one lane per location hash");
        const int l = threadIdx.x;
        const uint32_t c = l < L_cand ? (__ldcg(&A.S.stats[kMaxLogB + l].nsel) << G.logDd) : 0u;
        const uint32_t incl = warp_incl_scan(c);
        if (l <= L_cand) off[l] = incl - c;   // exclusive prefix; off[L_cand] = total
    }
    const bool staged = ((int64_t)A.L_loc << G.lw) <= A.vote_words;
    if (staged) {
        const int64_t nw = (int64_t)A.L_loc << G.lw;
        const uint32_t wm = (1u << G.lw) - 1;
        for (int64_t w = threadIdx.x; w < nw; w += blockDim.x)
            bm[w] = __ldg(&A.bucketbits[(w >> G.lw) * A.bucket_words + (w & wm)]);
    }
    if (threadIdx.x == 0) keep_n = 0;
    if (threadIdx.x < A.L_loc) {
        sh_sig[threadIdx.x][0] = A.sig[threadIdx.x][0];
        sh_sig[threadIdx.x][1] = A.sig[threadIdx.x][1];
        sh_sinv[threadIdx.x][0] = A.sinv[threadIdx.x][0];
        sh_sinv[threadIdx.x][1] = A.sinv[threadIdx.x][1];
    }
    __syncthreads();
    const uint32_t total = off[L_cand];
    const uint32_t stride = gridDim.x * blockDim.x;
    // (the trip count is the same for every lane of a warp: vote_round's warp-wide
    // ballots and shuffles need all 32 lanes; each candidate is checked against total)
    const uint32_t lane = threadIdx.x & 31;
    for (uint32_t wbase = blockIdx.x * blockDim.x + (threadIdx.x - lane); wbase < total;
         wbase += kVoteIlp * stride) {
        const uint32_t base = wbase + lane;
        if (staged)
            vote_round<NDIM, true>(A, G, bm, off, sh_sig, sh_sinv, L_cand, base, stride, total,
                                   keep_s, &keep_n);
        else
            vote_round<NDIM, false>(A, G, bm, off, sh_sig, sh_sinv, L_cand, base, stride, total,
                                    keep_s, &keep_n);
    }
    // this CTA's kept coordinates: their places in the kept list with one atomic
    __syncthreads();
    const uint32_t nk = min(keep_n, (uint32_t)kVoteKeep);
    if (nk == 0) return;
    if (threadIdx.x == 0)
        keep_base = (uint32_t)atomicAdd((unsigned long long *)&state->count, (unsigned long long)nk);
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < nk; i += blockDim.x) {
        const uint64_t pos = (uint64_t)keep_base + i;
        if (pos < (uint64_t)A.kept_cap) A.kept[pos] = keep_s[i];
    }
}

// The outputs: the caller's status words; the kept coordinates in ascending order with
// their Eq. (11) estimates and componentwise medians.  Up to kept_cap kept coordinates:
// each one's rank among them (a warp per coordinate); beyond: the ordered compaction of
// the coordinate bitmap by chunks of kChunkWords words, each chunk's first position the
// sum of the earlier chunks' counts.
__global__ void __launch_bounds__(256) k_loc_finish(const LocTailArgs A)
{
    pdl_wait();
    ExecState *state = A.state;
    if (blockIdx.x == 0 && threadIdx.x == 0) stamp(&state->bar);
    const int lane = threadIdx.x & 31;
    if (state->empty) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            *A.d_count = 0;
            *A.d_k = state->k_star;
            *A.d_status = state->status;
        }
        return;
    }
    const int b = state->b_star;
    const int64_t num = state->k_star;
    const int64_t K = state->count;
    extern __shared__ __align__(16) uint32_t dsm[];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        int st = state->status;
        if (K > A.capacity && st == ATSFFT_OK) st = ATSFFT_E_CAPACITY;
        *A.d_count = K;
        *A.d_k = num;
        *A.d_status = st;
    }
    if (K <= A.kept_cap) {
        // rank = number of kept coordinates below; a warp per coordinate splits the
        // comparisons, then its first L_est lanes compute the estimates
        constexpr int grp = 32;
        const int gl = lane;
        const int per_block = (int)blockDim.x / grp;
        uint32_t *ks = dsm;   // staged kept list chunk
        constexpr int kChunk = 3 * kRankStage;
        for (int64_t base = (int64_t)blockIdx.x * per_block; base < K;
             base += (int64_t)gridDim.x * per_block) {
            const int64_t k = base + threadIdx.x / grp;
            const bool valid = k < K;
            const uint32_t coord = valid ? A.kept[k] : 0u;
            // the estimates need only the coordinate: their loads go out before the rank
            // (a coordinate ranked beyond the capacity discards its estimate)
            float2 v = make_float2(0.f, 0.f);
            if (!A.skip_est && valid && gl < A.L_est) v = estimate_term(coord, A, b, gl);
            uint32_t r = 0;
            for (int64_t c0 = 0; c0 < K; c0 += kChunk) {
                const int64_t c1 = min(c0 + (int64_t)kChunk, K);
                __syncthreads();
                for (int64_t i0 = c0; i0 < c1; i0 += 8 * blockDim.x) {
                    uint32_t kv[8];
#pragma unroll
                    for (int u = 0; u < 8; u++) {
                        const int64_t i = i0 + u * blockDim.x + threadIdx.x;
                        kv[u] = i < c1 ? A.kept[i] : 0u;
                    }
#pragma unroll
                    for (int u = 0; u < 8; u++) {
                        const int64_t i = i0 + u * blockDim.x + threadIdx.x;
                        if (i < c1) ks[i - c0] = kv[u];
                    }
                }
                __syncthreads();
                if (valid) {
                    // four independent partial counts per lane
                    const int m = (int)(c1 - c0);
                    uint32_t r0 = 0, r1 = 0, r2 = 0, r3 = 0;
                    int i = gl;
                    for (; i + 3 * grp < m; i += 4 * grp) {
                        r0 += ks[i] < coord;
                        r1 += ks[i + grp] < coord;
                        r2 += ks[i + 2 * grp] < coord;
                        r3 += ks[i + 3 * grp] < coord;
                    }
                    for (; i < m; i += grp) r0 += ks[i] < coord;
                    r += r0 + r1 + r2 + r3;
                }
            }
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
            const bool inside = valid && r < A.capacity;
            if (!A.skip_est) {
                if (!inside) v = make_float2(0.f, 0.f);
                group_median(v, A.L_est, grp, inside, &A.val[inside ? r : 0],
                             A.msel && inside ? A.msel + 2 * (int64_t)r : nullptr);
            }
            if (valid && gl == 0) {
                A.coordbits[coord >> 5] = 0u;   // only kept coordinates set bits
                if (inside) A.loc[r] = coord;
            }
        }
    } else {
        __shared__ uint32_t tot;
        const int grp = A.est_group;
        const int gl = lane & (grp - 1);
        const int per_warp = 32 / grp;
        const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
        for (int64_t ch = blockIdx.x; ch < A.nchunks; ch += gridDim.x) {
            // the kept coordinates before this chunk: the earlier chunks' counts
            uint32_t part = 0;
            for (int64_t i = threadIdx.x; i < ch; i += blockDim.x) part += A.chunkcnt[i];
            int64_t pos0 = block_sum(part);
            const int64_t first = pos0;
            const int64_t w0 = ch * kChunkWords;
            const int64_t w1 = min(w0 + (int64_t)kChunkWords, A.coord_words);
            for (int64_t wb = w0; wb < w1; wb += blockDim.x) {
                const int64_t w = wb + threadIdx.x;
                uint32_t word = w < w1 ? A.coordbits[w] : 0u;
                int64_t pos = pos0 + block_exclusive_scan((uint32_t)__popc(word), &tot);
                if (word) A.coordbits[w] = 0u;
                while (word) {
                    const int bit = __ffs(word) - 1;
                    word &= word - 1;
                    if (pos < A.capacity) A.loc[pos] = w * 32 + bit;
                    pos++;
                }
                pos0 += tot;
                __syncthreads();
            }
            if (!A.skip_est) {
                // this chunk's coordinates inside the capacity (their loc entries were
                // written by this block: visible after the barrier above)
                const int64_t p1 = min(pos0, A.capacity);
                for (int64_t q0 = first + (int64_t)warp * per_warp; q0 < p1;
                     q0 += (int64_t)nwarps * per_warp) {
                    const int64_t s = q0 + lane / grp;
                    const bool valid = s < p1;
                    float2 v = make_float2(0.f, 0.f);
                    if (valid && gl < A.L_est) v = estimate_term((uint64_t)A.loc[s], A, b, gl);
                    group_median(v, A.L_est, grp, valid, &A.val[valid ? s : 0],
                                 A.msel && valid ? A.msel + 2 * s : nullptr);
                }
            }
            __syncthreads();
        }
    }
}

// ---------------------------------------------------------------------------------
// Launches
// ---------------------------------------------------------------------------------
static StatsParams stats_params(const atsfft_plan_s *P)
{
    StatsParams S;
    S.ndim = P->ndim;
    S.thr_rel = (float)P->p.thr_rel;
    S.thr_med = (float)P->p.thr_med;
    S.up = (float)(1.0 + P->p.tie_eta);
    S.use_median = P->p.thr_med > 0;
    S.ratio = S.use_median ? (float)(P->p.thr_rel / P->p.thr_med * (1.0 - 1.0 / 1048576.0)) : 0.f;
    S.stats = P->d_stats;
    S.lists = P->d_lmax;
    S.list_e = P->d_lmax_e;
    S.cap = P->lmax_cap;
    return S;
}

// Dynamic shared memory of the tail kernels: the largest scratch (the small-hash median:
// kSmallMedian values + 2048 histogram bins; the cutoff and the ordering: 3 kRankStage
// words).
constexpr size_t kTailSmemWords = (kSmallMedian + 2048) > 3 * kRankStage ? (kSmallMedian + 2048)
                                                                          : 3 * kRankStage;
constexpr size_t kTailSmem = sizeof(uint32_t) * kTailSmemWords;

// A tail kernel launched with programmatic stream serialization: its blocks may be
// scheduled before the previous kernel of the stream has finished and wait for it at
// griddepcontrol.wait (every tail kernel starts with that wait); cluster > 0: in
// thread-block clusters of that many CTAs.
template <class Arg>
static cudaError_t launch_pdl(void (*fn)(const Arg), int grid, int block, size_t smem,
                              const Arg &arg, cudaStream_t s, int cluster = 0)
{
    cudaFuncSetAttribute((const void *)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.numAttrs = 1;
    if (cluster > 0) {
        attr[1].id = cudaLaunchAttributeClusterDimension;
        attr[1].val.clusterDim.x = (unsigned)cluster;
        attr[1].val.clusterDim.y = 1;
        attr[1].val.clusterDim.z = 1;
        cfg.numAttrs = 2;
    }
    cfg.attrs = attr;
    return cudaLaunchKernelEx(&cfg, fn, arg);
}

static TuneTailArgs tune_args(const atsfft_plan_s *P)
{
    TuneTailArgs A;
    memset(&A, 0, sizeof(A));
    A.S = stats_params(P);
    A.b0 = P->b0;
    A.b_hi = P->b_hi;
    A.tune_max = P->p.tune_max;
    A.delta2 = P->p.delta2;
    A.tjob = P->d_tjob;
    A.nh_le = P->nh_le;
    A.L_loc = P->L_loc;
    A.lstat = P->d_lstat;
    A.z = P->d_z;
    A.energy = P->d_energy;
    A.e_loc = P->d_energy + P->e_loc_off;
    A.le = P->d_le;
    A.state = P->d_state;
    return A;
}

void launch_fixed_setup(const atsfft_plan_s *P, cudaStream_t s)
{
    const TuneTailArgs A = tune_args(P);
    launch_k(P, k_fixed_setup, dim3(1), dim3(32), 0, s, A, P->b_fixed, P->k_hint);
    count_launch(P);
}

void launch_tune_tail(const atsfft_plan_s *P, int stage, cudaStream_t s)
{
    // the stage's trials, ascending log2 B from b0
    const int lo = P->tune_hi[stage - 1] + 1, hi = P->tune_hi[stage];
    if (lo > hi) return;
    TuneTailArgs A = tune_args(P);
    int64_t tasks = 0;
    for (int b = lo; b <= hi; b++) {
        TrialView &t = A.trial[b - lo];
        const uint32_t mask = (1u << b) - 1;
        const atsfft::HashParam &hp = P->h_tune[b];
        t.e_off = P->tz_off[b];
        t.logB = b;
        t.slot = stats_slot_tune(b);
        t.s1 = hp.sigma[0] & mask;
        t.p1 = hp.sinv[0] & mask;
        t.s2 = hp.sigma[1] & mask;
        t.p2 = hp.sinv[1] & mask;
        const int64_t nb = P->ndim == 1 ? ((int64_t)1 << b) : ((int64_t)1 << (2 * b));
        tasks += (nb + kTask - 1) / kTask;
    }
    A.njobs = hi - lo + 1;
    A.stage = stage;
    A.limit_b = hi;
    const int64_t cap = (int64_t)P->num_sms * 4;
    const int grid = (int)(tasks < cap ? tasks : cap);
    launch_pdl(k_tune_tail, grid, 256, kTailSmem, A, s);
    count_launch(P);
}

void launch_loc_tail(const atsfft_plan_s *P, int64_t *d_loc, float2 *d_val, uint8_t *d_msel,
                     int64_t capacity, int64_t *d_count, int64_t *d_k, int32_t *d_status,
                     cudaStream_t s)
{
    LocTailArgs A;
    memset(&A, 0, sizeof(A));
    A.S = stats_params(P);
    A.L_loc = P->L_loc;
    A.L_est = P->L_est;
    A.est_base = P->est_base;
    A.est_group = 1;
    while (A.est_group < P->L_est) A.est_group *= 2;
    A.eta_up = (float)(1.0 + P->p.tie_eta);
    A.eta_dn = (float)(1.0 - P->p.tie_eta);
    for (int l = 0; l < P->L_loc; l++)
        for (int ax = 0; ax < 2; ax++) {
            A.sig[l][ax] = P->h_le[l].sigma[ax];
            A.sinv[l][ax] = P->h_le[l].sinv[ax];
        }
    A.e_loc = P->d_energy + P->e_loc_off;
    A.sel = P->d_sel;
    A.need = (uint32_t)((P->L_loc + 1) / 2);
    A.bucketbits = P->d_bucketbits;
    A.bucket_words = P->bucket_words;
    A.kept = P->d_kept;
    A.kept_cap = P->kept_cap;
    A.coordbits = P->d_coordbits;
    A.coord_words = P->coord_words;
    A.chunkcnt = P->d_blk;
    A.nchunks = P->nchunks;
    for (int l = 0; l < P->L_est; l++) A.est[l] = P->h_le[P->est_base + l];
    A.z = P->d_z;
    A.rgain = P->d_rgain;
    for (int b = 0; b < kMaxLogB; b++) A.ro.off[b] = P->resp_off[b];
    A.phase = P->d_phase;
    A.phase_s = P->phase_s;
    A.logn = P->logn;
    A.loc = d_loc;
    A.val = d_val;
    A.msel = d_msel;
    A.skip_est = P->p.precision == 1;
    A.capacity = capacity;
    A.d_count = d_count;
    A.d_k = d_k;
    A.d_status = d_status;
    A.state = P->d_state;
    // the votes stage the bitmaps of every B* whose L_loc bitmaps fit kVoteSmem
    const int64_t vote_bytes = (int64_t)P->L_loc * P->bucket_words * 4;
    const size_t vsmem = (size_t)(vote_bytes < kVoteSmem ? vote_bytes : kVoteSmem);
    A.vote_words = (int64_t)(vsmem / 4);
    launch_pdl(k_loc_select, P->L_loc * kSelCluster, kSelThreads, kSelSmem, A, s, kSelCluster);
    if (P->ndim == 1)
        launch_pdl(k_loc_votes<1>, P->num_sms, kVoteThreads, vsmem, A, s);
    else
        launch_pdl(k_loc_votes<2>, P->num_sms, kVoteThreads, vsmem, A, s);
    launch_pdl(k_loc_finish, P->num_sms * 4, 256, kTailSmem, A, s);
    count_launch(P, 3);
}

}  // namespace atsfft
