// bin.cu -- hash function part 1 (Section II-A): random spectrum permutation (Def. 1),
// flat window (Eqs. (8),(9)) and subsampling into B buckets (Lemma 2).
//
// For tap t of the window (|t| <= h) and sample a = (sigma t + tau) mod n, bucket b = t mod B
// receives G_t exp(i pi t/n) x_a.  With t = b + u B (u = floor(t / B)):
//   G_t exp(i pi t/n) = S_b * f_t * R_u,
//   S_b = sin(pi b / B) exp(i pi b / n)            (one factor per bucket),
//   f_t = (A n / pi) exp(-t^2 / (2 s^2)) / t       (real, per sample),
//   R_u = (-1)^u exp(i pi u / D)                   (D = n / B, period 2D in u),
// because sin(pi t / B) = (-1)^u sin(pi b / B).  The centre tap t = 0 (bucket 0, where
// S_0 = 0) is G_0 = A D.  Bucket sums are stored in residue order (common.cuh).
#include <string.h>

#include "devmath.cuh"

namespace atsfft {

constexpr int kGroup = 16;   // hashes accumulated together per thread

// Column form of the location pass (k_bin_cols, below)
constexpr int kColWarps = 3;        // warps per CTA, each with its own tile
constexpr int kColTile = 1024;      // samples per tile (8 KB)
constexpr int kColTileLog = 10;
constexpr int kColMaxLogD = 8;      // D <= 256: at least four columns per tile
constexpr int kColCtas = 9;         // CTAs per SM: 9 x 24 KB of tiles, all 4096 tiles of n = 2^22 in one wave

// Does the column form take the location pass at B* = 2^logB?
__host__ __device__ __forceinline__ bool column_form(int logn, int logB)
{
    return logn >= kColTileLog && logn - logB <= kColMaxLogD;
}

// ---------------------------------------------------------------------------------
// 1D gather form: a group of kGatherLanes lanes per bucket walks the taps t = b + u B of
// the window (about 2h / B + 1 of them, ~35 at the default window), each tap computed
// once and applied to every hash of the group (gathering x at each hash's position);
// the group's partial sums are added by shuffles and its first lane writes the buckets.
// A lane issues the gathers of kTapBatch1D taps (all hashes of its group) before it
// uses any of them, so its scattered loads overlap instead of following one another;
// groups of kGroup1D hashes (one grid row each) give the small B* of this form enough
// warps to cover that latency.
// ---------------------------------------------------------------------------------
constexpr int kGatherLanes = 8;
constexpr int kGroup1D = 4;
constexpr int kTapBatch1D = 6;

__global__ void k_bin_gather_1d(const float2 *__restrict__ x, int logn, const HashParam *hashes,
                                int nh, const WindowParam *win, const Job *job_dev,
                                int logB_static, const float2 *__restrict__ phase, int phase_s,
                                float2 *__restrict__ out)
{
    chain_wait();
    chain_next();
    int logB = logB_static;
    if (job_dev) {
        if (!job_dev->active || job_dev->stream) return;
        logB = job_dev->logB;
        nh = job_dev->nh;
    }
    const int group0 = blockIdx.y * kGroup1D;
    if (group0 >= nh) return;
    const int ng = min(kGroup1D, nh - group0);
    const uint32_t n = 1u << logn, mask = n - 1, B = 1u << logB;
    const WindowParam w = win[logB];
    const int lane = threadIdx.x & 31, q = lane & (kGatherLanes - 1);
    constexpr int kPerWarp = 32 / kGatherLanes;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t tasks = ((int64_t)B + kPerWarp - 1) / kPerWarp;
    float2 half;
    sincospif(ldexpf(1.0f, -logn), &half.y, &half.x);
    uint32_t sig[kGroup1D], tau[kGroup1D];
#pragma unroll
    for (int g = 0; g < kGroup1D; g++) {
        const HashParam hp = hashes[group0 + (g < ng ? g : 0)];
        sig[g] = hp.sigma[0];
        tau[g] = hp.tau[0];
    }
    for (int64_t wt = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); wt < tasks;
         wt += warps) {
        const int64_t bb = wt * kPerWarp + lane / kGatherLanes;
        const bool valid = bb < (int64_t)B;
        const int b = valid ? (int)bb : 0;
        // taps t = b + u B with |t| <= h
        const int u_lo = -((w.h + b) >> logB);          // ceil((-h - b) / B)
        const int u_hi = valid ? (w.h - b) >> logB : u_lo - 1;   // floor((h - b) / B)
        float2 acc[kGroup1D];
#pragma unroll
        for (int g = 0; g < kGroup1D; g++) acc[g] = make_float2(0.f, 0.f);
        for (int u0 = u_lo + q; u0 <= u_hi; u0 += kGatherLanes * kTapBatch1D) {
            float2 v[kTapBatch1D][kGroup1D];
#pragma unroll
            for (int i = 0; i < kTapBatch1D; i++) {
                const int u = u0 + i * kGatherLanes;
                const uint32_t t = (uint32_t)(b + u * (int)B);
#pragma unroll
                for (int g = 0; g < kGroup1D; g++)
                    v[i][g] = (u <= u_hi && g < ng) ? __ldg(&x[(sig[g] * t + tau[g]) & mask])
                                                   : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int i = 0; i < kTapBatch1D; i++) {
                const int u = u0 + i * kGatherLanes;
                const int t = b + u * (int)B;
                if (u > u_hi || t == 0) continue;      // centre tap handled below
                const float tf = (float)t;
                const float f = fast_exp2(fmaf(-w.k2 * tf, tf, w.log2c)) * fast_rcp(tf);
                const float2 R = rot_factor(u, logB, mask, phase, phase_s);
                const float2 c = make_float2(f * R.x, f * R.y);
#pragma unroll
                for (int g = 0; g < kGroup1D; g++) {
                    acc[g].x = fmaf(c.x, v[i][g].x, fmaf(-c.y, v[i][g].y, acc[g].x));
                    acc[g].y = fmaf(c.x, v[i][g].y, fmaf(c.y, v[i][g].x, acc[g].y));
                }
            }
        }
#pragma unroll
        for (int g = 0; g < kGroup1D; g++) {
#pragma unroll
            for (int o = kGatherLanes / 2; o > 0; o >>= 1) {
                acc[g].x += __shfl_xor_sync(0xffffffffu, acc[g].x, o);
                acc[g].y += __shfl_xor_sync(0xffffffffu, acc[g].y, o);
            }
        }
        if (valid && q == 0) {
            const float2 Sb = bucket_factor_tab((uint32_t)b, logB, logn, phase, phase_s, half);
#pragma unroll
            for (int g = 0; g < kGroup1D; g++) {
                if (g < ng) {
                    float2 z = cmul(Sb, acc[g]);
                    if (b == 0) {
                        const float2 v = __ldg(&x[tau[g] & mask]);
                        z.x += w.cA_D * v.x;
                        z.y += w.cA_D * v.y;
                    }
                    const uint32_t r = (sig[g] * (uint32_t)b + tau[g]) & (B - 1);
                    out[(int64_t)(group0 + g) * B + r] = z;
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------------
// 1D residue stream.  Thread = (residue r mod R, row chunk c); it reads the samples
// a = r + j R of its rows coalesced.  For a hash with B | R buckets every such sample
// falls in the same bucket b = sigma^{-1}(r - tau) mod B, so the thread keeps one
// accumulator per hash.  Hash l writes block (c * R/B_l + r / B_l) of B_l partial sums,
// element r mod B_l (residue order); the bucket FFT adds the blocks up.
// Per-hash constants live in the kernel parameter space.
//
// Window test folded into a table.  With t' = t + h mod n = sigma^{-1} a + c0 + h (mod n),
// the tap is in the window iff t' <= 2h.  For all samples of one thread t' = Q B + rho with
// rho fixed, so u = floor(t / B) = Q - kappa with kappa = ceil((h - rho) / B), and the
// window test becomes u <= floor((h - delta) / B), delta = kappa B + rho - h in [0, B),
// which takes one of two values (H - 1 or H, H = floor(h / B)).  Two tables per window,
// E_v[i] = R_u for u = i - (H + 1) <= H - 1 + v and 0 beyond, indexed by Q plus a
// per-thread offset, give R_u and the window test in one shared-memory read.
// ---------------------------------------------------------------------------------
constexpr int kMaxStream = 16;

struct StreamHash {
    uint32_t sinv, c0, tau;   // c0 = -sinv * tau (mod 2^32)
    int32_t logB, h;          // static passes: bucket count and window of this hash
    float k2, log2c, cAD;
    int32_t rot_off;          // its two E_v tables in shared memory (2 (D + 2) entries)
    int64_t out_off;          // its first partial block in `part`
};

struct StreamArgs {
    int nh;                   // hashes in this launch (<= kMaxStream)
    int hash_base;            // dynamic pass: index of the first hash (output block offset)
    int logR;                 // residue modulus (static passes)
    int chunks;               // row chunks (static passes)
    int ring_off;             // first float2 of the sample ring in shared memory
    StreamHash h[kMaxStream];
};

// Shared-memory entries of the two E_v tables of a window with D = n / B.
__host__ __device__ constexpr int rot_entries(uint32_t D) { return 2 * ((int)D + 2); }

// E_0, E_1 of one window (bucket count 2^lb, half-width h) at tab[0 .. 2 (D + 2)).
__device__ __forceinline__ void fill_rot_tables(float2 *tab, int logn, int lb, int h)
{
    const uint32_t D = 1u << (logn - lb);
    const int H = h >> lb;
    for (int e = threadIdx.x; e < rot_entries(D); e += blockDim.x) {
        const int v = e >= (int)D + 2;
        const int u = e - v * ((int)D + 2) - (H + 1);
        const uint32_t um = (uint32_t)u & (2 * D - 1);   // R_u has period 2D in u
        float sn, cs;
        sincospif(ldexpf((float)um, -(logn - lb)), &sn, &cs);
        const float2 r = (um & 1) ? make_float2(-cs, -sn) : make_float2(cs, sn);
        tab[e] = u <= H - 1 + v ? r : make_float2(0.f, 0.f);
    }
}

// The thread's table entry offset for one hash (from the window's first table, which has
// D + 2 entries): residue rho of t' mod B, kappa - H in {0, 1}, table v in {0, 1},
// index i = Q + 1 - (kappa - H).
__device__ __forceinline__ int rot_base(uint32_t rho, int h, int lb, int D2)
{
    const int B = 1 << lb, H = h >> lb, hr = h & (B - 1);
    const int k1 = (int)rho < hr;
    const int delta = (k1 ? B : 0) + (int)rho - hr;
    const int v = ((h - delta) >> lb) - (H - 1);
    return v * D2 + 1 - k1;
}

__device__ __forceinline__ float ld_shared_f32(uint32_t addr)
{
    float v;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(addr));
    return v;
}

// One complex table entry (8-byte aligned) in one shared-memory load.
__device__ __forceinline__ float2 ld_shared_f32x2(uint32_t addr)
{
    float2 v;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr));
    return v;
}

// Window constants of one hash inside the inner loop: uniform across the CTA.
struct TapConst {
    uint32_t c0h;        // c0 + h: t' = sigma^{-1} a + c0 + h (mod n)
    int h, logB;
    float mh;            // -(2^23 + h): t = float(2^23 + t') + mh, exact for n <= 2^23
    float k2, l2c;
};

// One (sample, hash) pair: t' from the exact integer index, E_v entry at the thread's
// table address `tb` (bytes) plus 8 Q, f_t = exp2(l2c - k2 t^2) / t, complex multiply-add.
// t = 0 (centre tap, bucket 0 only) yields inf, which stays in bucket 0's discarded
// accumulator.
template <bool SMALL_N>
__device__ __forceinline__ void tap_mac(float2 &acc, float2 v, uint32_t a, uint32_t sinv,
                                        uint32_t mask, const TapConst &T, uint32_t tb)
{
    const uint32_t tsh = (sinv * a + T.c0h) & mask;
    const uint32_t e = tb + ((tsh >> T.logB) << 3);
    const float2 ev = ld_shared_f32x2(e);
    const float ex = ev.x, ey = ev.y;
    const float tf = SMALL_N ? __uint_as_float(tsh | 0x4B000000u) + T.mh
                             : (float)((int)tsh - T.h);
    const float f = fast_exp2(fmaf(-T.k2 * tf, tf, T.l2c)) * fast_rcp(tf);
    const float cr = f * ex, ci = f * ey;
    acc.x = fmaf(cr, v.x, fmaf(-ci, v.y, acc.x));
    acc.y = fmaf(cr, v.y, fmaf(ci, v.x, acc.y));
}

// Grid: one thread per item (up to the CTAs per SM below), striding beyond.  The
// location pass (B* read on the device) takes CTAs of kStreamThreadsLE threads, which
// spread its usual 2^16 items over the SMs within one CTA of each other (1024 CTAs: 6 or
// 7 per SM, where 256-thread CTAs left SMs with 8 or with 16 warps); the tuning passes,
// whose CTAs fill E_v tables for several windows, take kStreamThreads.
constexpr int kStreamThreads = 256;
constexpr int kStreamCtas = 2;
constexpr int kStreamThreadsLE = 64;
constexpr int kStreamCtasLE = 8;

// Location pass: samples reach shared memory kRing rows ahead of their use.  Each thread
// copies its own sample of a row with cp.async into its own ring slot and reads it back
// after cp.async.wait_group, so no barrier is involved and no register holds a sample in
// flight (long-scoreboard stalls 2.35 -> 0.26 per issued instruction under ncu).
constexpr int kRing = 8;

__device__ __forceinline__ void cp_async8(uint32_t dst, const float2 *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

template <int NH, bool DYN>
__global__ void __launch_bounds__(kStreamThreads, kStreamCtas)
k_bin_stream(const float2 *__restrict__ x, int logn, const StreamArgs A, const Job *job_dev,
             const WindowParam *win, const float2 *__restrict__ phase, int phase_s,
             float2 *__restrict__ part, const int *skip)
{
    chain_wait();
    chain_next();
    extern __shared__ float2 rot[];
    if (skip && *skip) return;
    int logR = A.logR, chunks = A.chunks;
    WindowParam w = {};
    if (DYN) {
        if (!job_dev->active || !job_dev->stream) return;
        logR = job_dev->logB;
        if (column_form(logn, logR)) return;   // k_bin_cols takes this B*
        chunks = job_dev->chunks;
        w = win[logR];
    }
    const uint32_t n = 1u << logn, mask = n - 1, R = 1u << logR;
    if (DYN) {
        fill_rot_tables(rot, logn, logR, w.h);
    } else {
        for (int g = 0; g < NH; g++)
            if (g == 0 || A.h[g].rot_off != A.h[g - 1].rot_off)
                fill_rot_tables(rot + A.h[g].rot_off, logn, A.h[g].logB, A.h[g].h);
    }
    __syncthreads();
    TapConst T[NH];
#pragma unroll
    for (int g = 0; g < NH; g++) {
        const int h = DYN ? w.h : A.h[g].h;
        T[g].c0h = A.h[g].c0 + (uint32_t)h;
        T[g].h = h;
        T[g].logB = DYN ? logR : A.h[g].logB;
        T[g].mh = -(8388608.0f + (float)h);
        T[g].k2 = DYN ? w.k2 : A.h[g].k2;
        T[g].l2c = DYN ? w.log2c : A.h[g].log2c;
    }
    const uint32_t rot_s = (uint32_t)__cvta_generic_to_shared(rot);
    const uint32_t ring_s = rot_s + 8u * ((uint32_t)A.ring_off + threadIdx.x);
    float2 half;
    sincospif(ldexpf(1.0f, -logn), &half.y, &half.x);
    const uint32_t rows = (n >> logR) / (uint32_t)chunks;
    const int64_t items = (int64_t)R * chunks;
    const bool small_n = logn <= 23;
    for (int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; it < items;
         it += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t r = (uint32_t)(it & (R - 1));
        const uint32_t c = (uint32_t)(it >> logR);
        float2 acc[NH];
        uint32_t tb[NH];
#pragma unroll
        for (int g = 0; g < NH; g++) {
            acc[g] = make_float2(0.f, 0.f);
            const int lb = T[g].logB;
            const uint32_t rho = (A.h[g].sinv * r + T[g].c0h) & ((1u << lb) - 1);
            const int e = (DYN ? 0 : A.h[g].rot_off) + rot_base(rho, T[g].h, lb, (int)(n >> lb) + 2);
            tb[g] = rot_s + 8u * (uint32_t)e;
        }
        const uint32_t j0 = c * rows, j1 = j0 + rows;
        if (DYN) {
            // ring prologue: rows j0 .. j0 + kRing - 1, one commit group per row (empty past j1)
#pragma unroll
            for (int p = 0; p < kRing; p++) {
                if (j0 + p < j1) cp_async8(ring_s + 8u * (uint32_t)(p * blockDim.x), &x[r + ((j0 + p) << logR)]);
                cp_async_commit();
            }
            uint32_t slot = 0;
            if (small_n) {
                for (uint32_t j = j0; j < j1; j++) {
                    const uint32_t a = r + (j << logR);
                    cp_async_wait<kRing - 1>();
                    const uint32_t sa = ring_s + 8u * slot * blockDim.x;
                    const float2 v = ld_shared_f32x2(sa);
#pragma unroll
                    for (int g = 0; g < NH; g++) tap_mac<true>(acc[g], v, a, A.h[g].sinv, mask, T[g], tb[g]);
                    // the slot's sample has been used: refill it with row j + kRing
                    if (j + kRing < j1) cp_async8(sa, &x[a + ((uint32_t)kRing << logR)]);
                    cp_async_commit();
                    slot = (slot + 1) & (kRing - 1);
                }
            } else {
                for (uint32_t j = j0; j < j1; j++) {
                    const uint32_t a = r + (j << logR);
                    cp_async_wait<kRing - 1>();
                    const uint32_t sa = ring_s + 8u * slot * blockDim.x;
                    const float2 v = ld_shared_f32x2(sa);
#pragma unroll
                    for (int g = 0; g < NH; g++) tap_mac<false>(acc[g], v, a, A.h[g].sinv, mask, T[g], tb[g]);
                    if (j + kRing < j1) cp_async8(sa, &x[a + ((uint32_t)kRing << logR)]);
                    cp_async_commit();
                    slot = (slot + 1) & (kRing - 1);
                }
            }
            cp_async_wait<0>();
        } else if (small_n) {
            // the tuning passes (a few hashes per sample): plain loads, which the compiler
            // schedules ahead itself (measured faster here than the ring)
            for (uint32_t j = j0; j < j1; j++) {
                const uint32_t a = r + (j << logR);
                const float2 v = __ldg(&x[a]);
#pragma unroll
                for (int g = 0; g < NH; g++) tap_mac<true>(acc[g], v, a, A.h[g].sinv, mask, T[g], tb[g]);
            }
        } else {
            for (uint32_t j = j0; j < j1; j++) {
                const uint32_t a = r + (j << logR);
                const float2 v = __ldg(&x[a]);
#pragma unroll
                for (int g = 0; g < NH; g++) tap_mac<false>(acc[g], v, a, A.h[g].sinv, mask, T[g], tb[g]);
            }
        }
#pragma unroll
        for (int g = 0; g < NH; g++) {
            const int logB = DYN ? logR : A.h[g].logB;
            const uint32_t Bm = (1u << logB) - 1;
            const uint32_t b = (A.h[g].sinv * r + A.h[g].c0) & Bm;
            float2 z;
            if (b == 0) {
                // centre tap G_0 = A D on sample a = tau, added once (its residue, chunk)
                const uint32_t tau = A.h[g].tau;
                const bool mine = r == (tau & (R - 1)) && c == ((tau >> logR) / rows);
                const float cad = DYN ? w.cA_D : A.h[g].cAD;
                const float2 v = __ldg(&x[tau & mask]);
                z = mine ? make_float2(cad * v.x, cad * v.y) : make_float2(0.f, 0.f);
            } else {
                z = cmul(bucket_factor_tab(b, logB, logn, phase, phase_s, half), acc[g]);
            }
            const int64_t out_off = DYN ? (int64_t)(A.hash_base + g) * chunks * R : A.h[g].out_off;
            const uint32_t per_chunk = R >> logB;
            part[out_off + ((int64_t)c * per_chunk + (r >> logB)) * (Bm + 1) + (r & Bm)] = z;
        }
    }
}

// ---------------------------------------------------------------------------------
// 1D column form of the location pass (B* read on the device, D = n / B* <= 2^kColMaxLogD).
// The samples of bucket b of a hash all lie in one residue column r = (sigma b + tau) mod B
// (rows j = a >> log2 B of a = r + j B), and its taps t = b + u B, u_lo <= u <= u_hi, reach
// rows j0 + (u - u_lo) sigma (mod D): a walk over about 35 of the D rows of that column.
// Each warp stages a tile of 1024 samples -- 1024 / D whole columns, all D rows -- in
// shared memory ([row][column], so the lanes of a half-warp, on consecutive columns, hit
// different banks whatever rows they read), then every (column, hash) of the tile walks
// its own taps in u order: f_t from exp2 and a reciprocal as in the other forms, R_u by the
// recurrence R_(u+1) = R_u R_1 from the exact R_(u_lo), the sample from the tile.  Only the
// taps inside the window are evaluated (the residue stream evaluates every row of every
// hash, about 64 where ~35 are inside at B* = n / 64), and each bucket sum is complete:
// the first partial block holds it, further row chunks of the job are written as zeros.
// Lanes: 2^logLC consecutive columns side by side, the hashes dealt out among the lanes of
// one column (lpc of them), more columns per lane where the tile is wider than a warp.
// ---------------------------------------------------------------------------------

__global__ void __launch_bounds__(32 * kColWarps, kColCtas) k_bin_cols(const float2 *__restrict__ x, int logn,
                                                             const HashParam *__restrict__ hashes,
                                                             const Job *job_dev, const WindowParam *win,
                                                             const float2 *__restrict__ phase, int phase_s,
                                                             float2 *__restrict__ part)
{
    chain_wait();
    chain_next();
    extern __shared__ float2 col_tiles[];
    if (!job_dev->active || !job_dev->stream) return;
    const int logB = job_dev->logB, nh = job_dev->nh, chunks = job_dev->chunks;
    const int logD = logn - logB;
    if (!column_form(logn, logB)) return;   // the residue-stream kernel takes these
    const WindowParam w = win[logB];
    const uint32_t n = 1u << logn, mask = n - 1, B = 1u << logB, Bm = B - 1, Dm = (1u << logD) - 1;
    const int logTC = kColTileLog - logD;          // columns per tile
    const int logLC = logTC < 5 ? logTC : 5;       // columns side by side in a warp
    const int lpc = 32 >> logLC;                   // lanes per column
    const int cps = 1 << (logTC - logLC);          // columns per lane
    const int lane = threadIdx.x & 31;
    const int cl = lane & ((1 << logLC) - 1), sub = lane >> logLC;
    float2 *tile = col_tiles + (threadIdx.x >> 5) * kColTile;
    const uint32_t tile_s = (uint32_t)__cvta_generic_to_shared(tile);
    float2 half;
    sincospif(ldexpf(1.0f, -logn), &half.y, &half.x);
    const float2 r1 = rot_factor(1, logB, mask, phase, phase_s);   // R_1 = -exp(i pi / D)
    const int rsh = logTC + 3;   // row -> byte offset in the tile
    const uint32_t rmask = Dm << rsh;
    const float Bf = (float)B;
    const int64_t tiles = (int64_t)1 << (logn - kColTileLog);
    const int64_t nw = (int64_t)gridDim.x * kColWarps;
    for (int64_t tl = (int64_t)blockIdx.x * kColWarps + (threadIdx.x >> 5); tl < tiles; tl += nw) {
        const uint32_t col0 = (uint32_t)tl << logTC;
        __syncwarp();   // the previous tile's reads are done
#pragma unroll 8
        for (int e = lane; e < kColTile; e += 32)
            tile[e] = __ldg(&x[col0 + ((uint32_t)e & ((1u << logTC) - 1)) + ((uint32_t)(e >> logTC) << logB)]);
        __syncwarp();
        for (int sl = 0; sl < cps; sl++) {
            const uint32_t c = (uint32_t)cl + ((uint32_t)sl << logLC);
            const uint32_t r = col0 + c;
            const uint32_t cbase = tile_s + 8u * c;
            for (int g = sub; g < nh; g += lpc) {
                const HashParam hp = hashes[g];
                const uint32_t sig = hp.sigma[0], tau = hp.tau[0];
                const uint32_t b = (hp.sinv[0] * (r - tau)) & Bm;
                float2 z;
                if (b == 0) {
                    // only the centre tap G_0 = A D (on sample tau) reaches bucket 0
                    const float2 v = __ldg(&x[tau & mask]);
                    z = make_float2(w.cA_D * v.x, w.cA_D * v.y);
                } else {
                    const int u_lo = -((w.h + (int)b) >> logB), u_hi = (w.h - (int)b) >> logB;
                    const int t0 = (int)b + u_lo * (int)B;
                    // byte offset of the tap's row in the tile, stepping by sigma rows (mod D)
                    uint32_t jo = (((sig * (uint32_t)t0 + tau) & mask) >> logB) << rsh;
                    const uint32_t djo = (sig & Dm) << rsh;
                    float tf = (float)t0;
                    float2 R = rot_factor(u_lo, logB, mask, phase, phase_s);
                    float2 acc = make_float2(0.f, 0.f);
#pragma unroll 2
                    for (int u = u_lo; u <= u_hi; u++) {
                        const float2 v = ld_shared_f32x2(cbase + jo);
                        const float f = fast_exp2(fmaf(-w.k2 * tf, tf, w.log2c)) * fast_rcp(tf);
                        const float cr = f * R.x, ci = f * R.y;
                        acc.x = fmaf(cr, v.x, fmaf(-ci, v.y, acc.x));
                        acc.y = fmaf(cr, v.y, fmaf(ci, v.x, acc.y));
                        R = cmul(R, r1);
                        tf += Bf;
                        jo = (jo + djo) & rmask;
                    }
                    z = cmul(bucket_factor_tab(b, logB, logn, phase, phase_s, half), acc);
                }
                float2 *o = part + (int64_t)g * chunks * B + r;
                o[0] = z;
                for (int ch = 1; ch < chunks; ch++) o[(int64_t)ch * B] = make_float2(0.f, 0.f);
            }
        }
    }
}

struct GatherHash {
    uint32_t sig, tau;
    int32_t logB, h;
    float k2, log2c, cAD;
    int64_t out_off;
    int64_t bucket_start;    // first bucket of this hash in the launch's bucket list
};

struct GatherArgs {
    int njobs;
    int64_t total_buckets;
    GatherHash j[kMaxLogB];
};

// Tuning hashes with small windows, all in one launch: a group of kTuneLanes lanes per
// bucket (the buckets of all hashes listed back to back), as in k_bin_gather_1d with one
// hash.  Bucket counts are multiples of 32 / kTuneLanes, so a warp's buckets share a hash.
constexpr int kTuneLanes = 4;

__global__ void k_bin_gather_tune(const float2 *__restrict__ x, int logn, const GatherArgs A,
                                  const float2 *__restrict__ phase, int phase_s,
                                  float2 *__restrict__ part)
{
    chain_wait();
    chain_next();
    const uint32_t n = 1u << logn, mask = n - 1;
    const int lane = threadIdx.x & 31, q = lane & (kTuneLanes - 1);
    constexpr int kPerWarp = 32 / kTuneLanes;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t tasks = (A.total_buckets + kPerWarp - 1) / kPerWarp;
    float2 half;
    sincospif(ldexpf(1.0f, -logn), &half.y, &half.x);
    for (int64_t wt = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); wt < tasks;
         wt += warps) {
        const int64_t gb = wt * kPerWarp + lane / kTuneLanes;
        const bool valid = gb < A.total_buckets;
        // the hash whose bucket range holds gb (bucket_start ascending): binary search
        static_assert(kMaxLogB <= 32, "job search covers 32 jobs");
        int jb = 0;
        for (int step = 16; step > 0; step >>= 1)
            if (jb + step < A.njobs && gb >= A.j[jb + step].bucket_start) jb += step;
        const GatherHash &H = A.j[jb];
        const int logB = H.logB;
        const uint32_t B = 1u << logB;
        const int b = valid ? (int)(gb - H.bucket_start) : 0;
        const int u_lo = -((H.h + b) >> logB), u_hi = valid ? (H.h - b) >> logB : u_lo - 1;
        float2 acc = make_float2(0.f, 0.f);
        for (int u = u_lo + q; u <= u_hi; u += kTuneLanes) {
            const int t = b + u * (int)B;
            if (t == 0) continue;
            const float tf = (float)t;
            const float f = fast_exp2(fmaf(-H.k2 * tf, tf, H.log2c)) * fast_rcp(tf);
            const float2 R = rot_factor(u, logB, mask, phase, phase_s);
            const float2 c = make_float2(f * R.x, f * R.y);
            const float2 v = __ldg(&x[(H.sig * (uint32_t)t + H.tau) & mask]);
            acc.x = fmaf(c.x, v.x, fmaf(-c.y, v.y, acc.x));
            acc.y = fmaf(c.x, v.y, fmaf(c.y, v.x, acc.y));
        }
#pragma unroll
        for (int o = kTuneLanes / 2; o > 0; o >>= 1) {
            acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
            acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
        }
        if (valid && q == 0) {
            float2 z = cmul(bucket_factor_tab((uint32_t)b, logB, logn, phase, phase_s, half), acc);
            if (b == 0) {
                const float2 v = __ldg(&x[H.tau & mask]);
                z = make_float2(H.cAD * v.x, H.cAD * v.y);
            }
            part[H.out_off + ((H.sig * (uint32_t)b + H.tau) & (B - 1))] = z;
        }
    }
}

// ---------------------------------------------------------------------------------
// 2D: per-hash, per-axis tap tables indexed by sample position a in [N]:
// tap[a] = G_t exp(i pi t / N) for t = sigma^{-1}(a - tau) mod N (signed), 0 outside
// the window.  FP64 evaluation, stored as complex64.
// ---------------------------------------------------------------------------------
__global__ void k_taps_2d(int logn, const HashParam *hashes, int nh, const WindowParam *win,
                          const Job *job_dev, int logB_static, float2 *taps)
{
    chain_wait();
    chain_next();
    int logB = logB_static;
    if (job_dev) {
        if (!job_dev->active) return;
        logB = job_dev->logB;
        nh = job_dev->nh;
    }
    const int64_t N = (int64_t)1 << logn;
    const WindowParam w = win[logB];
    const int64_t total = (int64_t)nh * 2 * N;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int l = (int)(i / (2 * N));
        const int axis = (int)((i / N) & 1);
        const uint32_t a = (uint32_t)(i & (N - 1));
        const HashParam hp = hashes[l];
        const uint32_t t = (hp.sinv[axis] * (a - hp.tau[axis])) & (uint32_t)(N - 1);
        int64_t ts = t >= (uint32_t)(N / 2) ? (int64_t)t - N : (int64_t)t;
        float2 v = make_float2(0.f, 0.f);
        if (ts >= -w.h && ts <= w.h) {
            double g;
            if (ts == 0) {
                g = w.A * (double)(N >> logB);
            } else {
                const int64_t B = (int64_t)1 << logB;
                int64_t r = ts % (2 * B);
                if (r < 0) r += 2 * B;
                const double sn = (r == 0 || r == B) ? 0.0 : sinpi((double)r / (double)B);
                g = w.A * exp(-((double)ts * (double)ts) / (2.0 * w.s * w.s)) * sn /
                    (M_PI * (double)ts / (double)N);
            }
            double ps, pc;
            sincospi((double)ts / (double)N, &ps, &pc);
            v = make_float2((float)(g * pc), (float)(g * ps));
        }
        taps[i] = v;
    }
}

constexpr uint32_t kRowBatch = 4;   // pixels of a row in flight per thread (2D stream)

// 2D residue stream: thread = (residue pair (r1, r2), chunk of rows j1).  Pixels
// (r1 + j1 B, r2 + j2 B) all feed bucket (b1, b2) of each hash.  Output
// part[(chunk * nh + l) * B^2 + r1 * B + r2].
__global__ void __launch_bounds__(256) k_bin_stream_2d(const float2 *__restrict__ x, int logn,
                                                       int nh, const Job *job_dev,
                                                       int logB_static, int chunks_static,
                                                       const float2 *__restrict__ taps, int64_t tstride,
                                                       float2 *__restrict__ part)
{
    chain_wait();
    chain_next();
    int logB = logB_static, chunks = chunks_static;
    if (job_dev) {
        if (!job_dev->active) return;
        logB = job_dev->logB;
        nh = job_dev->nh;
        chunks = job_dev->chunks;
        taps += (int64_t)logB * tstride;   // the plan's tables of B* (tstride 0: tables of this exec)
    }
    const int group0 = blockIdx.y * kGroup;
    if (group0 >= nh) return;
    const int ng = min(kGroup, nh - group0);
    const uint32_t N = 1u << logn, B = 1u << logB, D = N >> logB;
    const uint32_t rows = D / (uint32_t)chunks;
    const int64_t B2 = (int64_t)B * B;
    const int64_t items = B2 * chunks;
    for (int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; it < items;
         it += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t r2 = (uint32_t)(it & (B - 1));
        const uint32_t r1 = (uint32_t)((it >> logB) & (B - 1));
        const uint32_t ch = (uint32_t)(it >> (2 * logB));
        float2 acc[kGroup];
#pragma unroll
        for (int g = 0; g < kGroup; g++) acc[g] = make_float2(0.f, 0.f);
        for (uint32_t j1 = ch * rows; j1 < (ch + 1) * rows; j1++) {
            const uint32_t a1 = r1 + (j1 << logB);
            const float2 *xrow = x + (int64_t)a1 * N;
            float2 row[kGroup];
#pragma unroll
            for (int g = 0; g < kGroup; g++) row[g] = make_float2(0.f, 0.f);
            uint32_t j2 = 0;
            // kRowBatch pixels of the row (and each hash's taps for them) requested before
            // any is used: one memory round trip per batch instead of per pixel; the sums
            // keep the pixel order
            for (; j2 + kRowBatch <= D; j2 += kRowBatch) {
                float2 v[kRowBatch];
#pragma unroll
                for (int q = 0; q < kRowBatch; q++) v[q] = __ldg(&xrow[r2 + ((j2 + q) << logB)]);
#pragma unroll
                for (int g = 0; g < kGroup; g++) {
                    if (g < ng) {
                        const float2 *tg = taps + ((int64_t)(group0 + g) * 2 + 1) * N + r2;
                        float2 tp[kRowBatch];
#pragma unroll
                        for (int q = 0; q < kRowBatch; q++) tp[q] = __ldg(&tg[(j2 + q) << logB]);
#pragma unroll
                        for (int q = 0; q < kRowBatch; q++) {
                            row[g].x = fmaf(tp[q].x, v[q].x, fmaf(-tp[q].y, v[q].y, row[g].x));
                            row[g].y = fmaf(tp[q].x, v[q].y, fmaf(tp[q].y, v[q].x, row[g].y));
                        }
                    }
                }
            }
            for (; j2 < D; j2++) {
                const uint32_t a2 = r2 + (j2 << logB);
                const float2 v = __ldg(&xrow[a2]);
#pragma unroll
                for (int g = 0; g < kGroup; g++) {
                    if (g < ng) {
                        const float2 tp = __ldg(&taps[((int64_t)(group0 + g) * 2 + 1) * N + a2]);
                        row[g].x = fmaf(tp.x, v.x, fmaf(-tp.y, v.y, row[g].x));
                        row[g].y = fmaf(tp.x, v.y, fmaf(tp.y, v.x, row[g].y));
                    }
                }
            }
#pragma unroll
            for (int g = 0; g < kGroup; g++) {
                if (g < ng) {
                    const float2 tp = __ldg(&taps[((int64_t)(group0 + g) * 2 + 0) * N + a1]);
                    acc[g].x = fmaf(tp.x, row[g].x, fmaf(-tp.y, row[g].y, acc[g].x));
                    acc[g].y = fmaf(tp.x, row[g].y, fmaf(tp.y, row[g].x, acc[g].y));
                }
            }
        }
#pragma unroll
        for (int g = 0; g < kGroup; g++)
            if (g < ng) part[((int64_t)(group0 + g) * chunks + ch) * B2 + (int64_t)r1 * B + r2] = acc[g];
    }
}

// 2D gather for small windows: warp per bucket (b1, b2); lanes walk the window's
// (u1, u2) pairs; taps from the per-axis tables at the permuted positions.
__global__ void k_bin_gather_2d(const float2 *__restrict__ x, int logn, const HashParam *hashes,
                                int nh, const WindowParam *win, const Job *job_dev,
                                int logB_static, const float2 *__restrict__ taps, int64_t tstride,
                                float2 *__restrict__ out)
{
    chain_wait();
    chain_next();
    int logB = logB_static;
    if (job_dev) {
        if (!job_dev->active || job_dev->stream) return;
        logB = job_dev->logB;
        nh = job_dev->nh;
        taps += (int64_t)logB * tstride;
    }
    const uint32_t N = 1u << logn, mask = N - 1, B = 1u << logB;
    const int64_t B2 = (int64_t)B * B;
    const WindowParam w = win[logB];
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int l = blockIdx.y;
    if (l >= nh) return;
    const HashParam hp = hashes[l];
    for (int64_t bw = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); bw < B2;
         bw += warps) {
        const int b1 = (int)(bw >> logB), b2 = (int)(bw & (B - 1));
        const int u1lo = -((w.h + b1) >> logB), u1hi = (w.h - b1) >> logB;
        const int u2lo = -((w.h + b2) >> logB), u2hi = (w.h - b2) >> logB;
        const int n2 = u2hi - u2lo + 1;
        const int64_t cnt = (int64_t)(u1hi - u1lo + 1) * n2;
        float2 acc = make_float2(0.f, 0.f);
        for (int64_t k = lane; k < cnt; k += 32) {
            const int u1 = u1lo + (int)(k / n2), u2 = u2lo + (int)(k % n2);
            const uint32_t t1 = (uint32_t)(b1 + u1 * (int)B), t2 = (uint32_t)(b2 + u2 * (int)B);
            const uint32_t a1 = (hp.sigma[0] * t1 + hp.tau[0]) & mask;
            const uint32_t a2 = (hp.sigma[1] * t2 + hp.tau[1]) & mask;
            const float2 g1 = __ldg(&taps[((int64_t)l * 2 + 0) * N + a1]);
            const float2 g2 = __ldg(&taps[((int64_t)l * 2 + 1) * N + a2]);
            const float2 v = __ldg(&x[(int64_t)a1 * N + a2]);
            const float2 c = cmul(g1, g2);
            acc.x = fmaf(c.x, v.x, fmaf(-c.y, v.y, acc.x));
            acc.y = fmaf(c.x, v.y, fmaf(c.y, v.x, acc.y));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
            acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
        }
        if (lane == 0) {
            const uint32_t r1 = (hp.sigma[0] * (uint32_t)b1 + hp.tau[0]) & (B - 1);
            const uint32_t r2 = (hp.sigma[1] * (uint32_t)b2 + hp.tau[1]) & (B - 1);
            out[(int64_t)l * B2 + (int64_t)r1 * B + r2] = acc;
        }
    }
}

// ---------------------------------------------------------------------------------
// Launches
// ---------------------------------------------------------------------------------

static GatherHash gather_hash(const atsfft_plan_s *P, const HashParam &hp, int b, int64_t out_off)
{
    const WindowParam &w = P->h_win[b];
    GatherHash g;
    g.sig = hp.sigma[0];
    g.tau = hp.tau[0];
    g.logB = b;
    g.h = w.h;
    g.k2 = w.k2;
    g.log2c = w.log2c;
    g.cAD = w.cA_D;
    g.out_off = out_off;
    g.bucket_start = 0;
    return g;
}

// 256-thread CTAs, 8 warps of 32 / kTuneLanes buckets each per round, at most 8 per SM.
static void launch_gather_tune(const atsfft_plan_s *P, const float2 *x, const GatherArgs &G,
                               cudaStream_t s)
{
    const int64_t per_cta = 8 * (32 / kTuneLanes);
    const int64_t blocks = (G.total_buckets + per_cta - 1) / per_cta;
    const int64_t cap = (int64_t)P->num_sms * 8;
    launch_k(P, k_bin_gather_tune, dim3((unsigned)(blocks < cap ? blocks : cap)), dim3(256), 0, s, 
        x, P->logn, G, P->d_phase, P->phase_s, P->d_part);
    count_launch(P);
}

static StreamHash stream_hash(const atsfft_plan_s *P, const HashParam &hp, int b, int64_t out_off)
{
    StreamHash h;
    memset(&h, 0, sizeof(h));
    h.sinv = hp.sinv[0];
    h.c0 = 0u - hp.sinv[0] * hp.tau[0];
    h.tau = hp.tau[0];
    if (b >= 0) {
        const WindowParam &w = P->h_win[b];
        h.logB = b;
        h.h = w.h;
        h.k2 = w.k2;
        h.log2c = w.log2c;
        h.cAD = w.cA_D;
    }
    h.out_off = out_off;
    return h;
}

// `smem` holds the E_v tables; the sample ring follows them.  One thread per item
// (residues x row chunks; for a dynamic pass the most any stream-form B* can have).
template <int NH, bool DYN>
static void launch_stream(const atsfft_plan_s *P, const float2 *x, const StreamArgs &A0,
                          const Job *job_dev, size_t smem, const int *skip, cudaStream_t s)
{
    StreamArgs A = A0;
    const int threads = DYN ? kStreamThreadsLE : kStreamThreads;
    const int per_sm = DYN ? kStreamCtasLE : kStreamCtas;
    A.ring_off = (int)((smem + sizeof(float2) - 1) / sizeof(float2));
    if (DYN) smem = sizeof(float2) * ((size_t)A.ring_off + (size_t)kRing * threads);
    int64_t items = (int64_t)A.chunks << A.logR;
    if (DYN) {
        items = 0;
        for (int b = P->b0; b <= P->b_hi; b++)
            if (P->h_tjob[b].stream && ((int64_t)P->h_tjob[b].chunks << b) > items)
                items = (int64_t)P->h_tjob[b].chunks << b;
    }
    int64_t grid = (items + threads - 1) / threads;
    if (grid > (int64_t)P->num_sms * per_sm) grid = (int64_t)P->num_sms * per_sm;
    if (grid < 1) grid = 1;
    const void *fn = (const void *)k_bin_stream<NH, DYN>;
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    launch_k(P, k_bin_stream<NH, DYN>, dim3((unsigned)grid), dim3((unsigned)threads), smem, s,
        x, P->logn, A, job_dev, P->d_win, P->d_phase, P->phase_s, P->d_part, skip);
    count_launch(P);
}

template <bool DYN>
static void launch_stream_nh(const atsfft_plan_s *P, const float2 *x, const StreamArgs &A,
                             const Job *job_dev, size_t smem, cudaStream_t s,
                             const int *skip = nullptr)
{
#define ATSFFT_NH(k) case k: launch_stream<k, DYN>(P, x, A, job_dev, smem, skip, s); break;
    switch (A.nh) {
    ATSFFT_NH(1) ATSFFT_NH(2) ATSFFT_NH(3) ATSFFT_NH(4) ATSFFT_NH(5) ATSFFT_NH(6) ATSFFT_NH(7)
    ATSFFT_NH(8) ATSFFT_NH(9) ATSFFT_NH(10) ATSFFT_NH(11) ATSFFT_NH(12) ATSFFT_NH(13)
    ATSFFT_NH(14) ATSFFT_NH(15) ATSFFT_NH(16)
    default: break;
    }
#undef ATSFFT_NH
}

// Tuning: every B of the range, one hash each, in up to three stages (tune_hi).  1D
// stage 1: the small-window trials in one gather launch; stages 2 and 3: the
// large-window ones, each stage in one residue-stream pass with R = the largest of its
// B, every kernel of it returning at once when an earlier stage already settled the
// controller.  2D: one stage, one launch per B.  Each stage ends with the bucket FFTs of
// its trials in one batch.  Profiling mark 1 + 3 (stage - 1) separates the two.
void launch_tuning(const atsfft_plan_s *P, const float2 *x, int stage, cudaStream_t s)
{
    int logB[kMaxLogB], chunks[kMaxLogB], nj = 0;
    int64_t in_off[kMaxLogB], out_off[kMaxLogB];
    const int *skip = nullptr;
    const int mark = 1 + 3 * (stage - 1);
    if (P->ndim == 1) {
        const int lo = P->tune_hi[stage - 1] + 1;
        const int hi = P->tune_hi[stage];
        if (lo > hi) {
            prof_mark(P, mark, s);
            return;
        }
        GatherArgs G;
        G.njobs = 0;
        G.total_buckets = 0;
        StreamArgs S;
        memset(&S, 0, sizeof(S));
        int rot_total = 0;
        for (int b = lo; b <= hi; b++) {
            if (P->h_tjob[b].stream) {
                StreamHash &h = S.h[S.nh++];
                h = stream_hash(P, P->h_tune[b], b, P->tpart_off[b]);
                h.rot_off = rot_total;
                rot_total += rot_entries((uint32_t)(P->n >> b));
            } else {
                GatherHash &g = G.j[G.njobs++];
                g = gather_hash(P, P->h_tune[b], b, P->tpart_off[b]);
                g.bucket_start = G.total_buckets;
                G.total_buckets += (int64_t)1 << b;
            }
            logB[nj] = b;
            chunks[nj] = P->tchunks[b];
            in_off[nj] = P->tpart_off[b];
            out_off[nj] = P->tz_off[b];
            nj++;
        }
        if (G.njobs) launch_gather_tune(P, x, G, s);
        if (stage >= 2) skip = &P->d_state->tune_done;
        if (S.nh) {
            S.logR = P->tstream_logR[stage];
            S.chunks = P->tstream_chunks[stage];
            launch_stream_nh<false>(P, x, S, nullptr, sizeof(float2) * rot_total, s, skip);
        }
    } else {
        if (stage != 1) {
            prof_mark(P, mark, s);
            return;
        }
        for (int b = P->b0; b <= P->b_hi; b++) {
            launch_bin_2d(P, x, nullptr, P->h_tjob[b], false, P->d_tune + b, b,
                          P->d_part + P->tpart_off[b], s, P->d_taps_tune + ((size_t)b << (P->logn + 1)));
            logB[nj] = b;
            chunks[nj] = P->tchunks[b];
            in_off[nj] = P->tpart_off[b];
            out_off[nj] = P->tz_off[b];
            nj++;
        }
    }
    prof_mark(P, mark, s);
    launch_bucket_fft_batch(P, nj, logB, chunks, in_off, out_off, P->d_part, P->d_tz, P->d_energy,
                            skip, s);
}

// Location + estimation hashes at the device-chosen B*: every form is launched, the
// one matching the job runs.  1D stream launches take at most kMaxStream hashes each.
void launch_le_bin(const atsfft_plan_s *P, const float2 *x, const Job *job_dev, cudaStream_t s)
{
    const int nh = P->nh_le;
    if (P->ndim == 1) {
        // shared memory for the E_v tables of the smallest B the stream form can take; the
        // column form takes every stream-form B* with D <= 2^kColMaxLogD
        size_t smem = 16;
        bool stream_needed = false;
        for (int b = P->b0; b <= P->b_hi; b++)
            if (P->h_tjob[b].stream) {
                if (smem == 16) smem = sizeof(float2) * rot_entries((uint32_t)(P->n >> b));
                if (!column_form(P->logn, b)) stream_needed = true;
            }
        if (stream_needed) {
            for (int g0 = 0; g0 < nh; g0 += kMaxStream) {
                StreamArgs S;
                memset(&S, 0, sizeof(S));
                S.nh = nh - g0 < kMaxStream ? nh - g0 : kMaxStream;
                S.hash_base = g0;
                for (int g = 0; g < S.nh; g++) S.h[g] = stream_hash(P, P->h_le[g0 + g], -1, 0);
                launch_stream_nh<true>(P, x, S, job_dev, smem, s);
            }
        }
        {
            const size_t csm = sizeof(float2) * (size_t)kColTile * kColWarps;
            const int64_t tiles = P->logn < kColTileLog ? 0 : P->n >> kColTileLog;
            const int64_t grid = (tiles + kColWarps - 1) / kColWarps;
            cudaFuncSetAttribute((const void *)k_bin_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)csm);
            launch_k(P, k_bin_cols, dim3((unsigned)(grid > 0 ? grid : 1)), dim3(32 * kColWarps), csm, s, x,
                     P->logn, (const HashParam *)P->d_le, job_dev, P->d_win, P->d_phase, P->phase_s, P->d_part);
            count_launch(P);
        }
        prof_mark(P, 10, s);
        const int groups = (nh + kGroup1D - 1) / kGroup1D;
        dim3 grid(P->num_sms * kPersistCtas, groups);
        launch_k(P, k_bin_gather_1d, dim3(grid), dim3(256), 0, s, x, P->logn, P->d_le, nh, P->d_win, job_dev, 0,
                                             P->d_phase, P->phase_s, P->d_part);
        count_launch(P);
    } else {
        Job jl;
        memset(&jl, 0, sizeof(jl));
        jl.nh = nh;
        launch_bin_2d(P, x, job_dev, jl, true, P->d_le, 0, P->d_part, s, P->d_taps_le,
                      (int64_t)nh << (P->logn + 1));
    }
}

// One hash (inspection): bins into P->d_part and transforms into `out` (B or B^2 values).
void launch_single_hash(const atsfft_plan_s *P, const float2 *x, int b, const HashParam &hp,
                        const HashParam *hp_dev, float2 *out, cudaStream_t s)
{
    const Job &j = P->h_tjob[b];
    int chunks = j.chunks;
    if (P->ndim == 1) {
        if (j.stream) {
            StreamArgs S;
            memset(&S, 0, sizeof(S));
            S.nh = 1;
            S.logR = b;
            S.chunks = j.chunks;
            S.h[0] = stream_hash(P, hp, b, 0);
            launch_stream_nh<false>(P, x, S, nullptr, sizeof(float2) * rot_entries((uint32_t)(P->n >> b)), s);
        } else {
            GatherArgs G;
            G.njobs = 1;
            G.j[0] = gather_hash(P, hp, b, 0);
            G.total_buckets = (int64_t)1 << b;
            launch_gather_tune(P, x, G, s);
            chunks = 1;
        }
    } else {
        launch_bin_2d(P, x, nullptr, j, false, hp_dev, b, P->d_part, s);
    }
    const int64_t zero = 0;
    launch_bucket_fft_batch(P, 1, &b, &chunks, &zero, &zero, P->d_part, out, nullptr, nullptr, s);
}

// The L_est estimation hashes of a 1D plan at B = 2^b into P->d_part, layout
// [hash][chunk][B] (the form the plan uses at this B); returns the chunk count.
int launch_est_bin(const atsfft_plan_s *P, const float2 *x, int b, cudaStream_t s)
{
    const int L = P->L_est;
    const Job &j = P->h_tjob[b];
    if (j.stream) {
        for (int g0 = 0; g0 < L; g0 += kMaxStream) {
            StreamArgs S;
            memset(&S, 0, sizeof(S));
            S.nh = L - g0 < kMaxStream ? L - g0 : kMaxStream;
            S.logR = b;
            S.chunks = j.chunks;
            for (int g = 0; g < S.nh; g++) {
                S.h[g] = stream_hash(P, P->h_le[P->est_base + g0 + g], b,
                                     ((int64_t)(g0 + g) * j.chunks) << b);
                S.h[g].rot_off = 0;   // one B: every hash's E_v tables are the same
            }
            launch_stream_nh<false>(P, x, S, nullptr, sizeof(float2) * rot_entries((uint32_t)(P->n >> b)), s);
        }
        return j.chunks;
    }
    dim3 grid(P->num_sms * kPersistCtas, (L + kGroup1D - 1) / kGroup1D);
    launch_k(P, k_bin_gather_1d, dim3(grid), dim3(256), 0, s, x, P->logn, P->d_le + P->est_base, L, P->d_win, nullptr, b,
                                         P->d_phase, P->phase_s, P->d_part);
    count_launch(P);
    return 1;
}

// pre_taps: the plan's tap tables of these hashes (static: of B = 2^logB_static; dynamic:
// those of B = 2^b at pre_taps + b * pre_stride); null: built here into the scratch.
void launch_bin_2d(const atsfft_plan_s *P, const float2 *x, const Job *job_dev, const Job &job_host,
                   bool dynamic, const HashParam *hashes, int logB_static, float2 *part,
                   cudaStream_t s, const float2 *pre_taps, int64_t pre_stride)
{
    const int persist = P->num_sms * kPersistCtas;
    const int groups = (job_host.nh + kGroup - 1) / kGroup;
    const Job *jd = dynamic ? job_dev : nullptr;
    const float2 *taps = pre_taps;
    int64_t tstride = dynamic ? pre_stride : 0;
    if (!taps) {
        float2 *t = P->d_fft_tmp;   // per-axis tap tables: nh x 2 x N
        launch_k(P, k_taps_2d, dim3(P->num_sms * 2), dim3(256), 0, s, P->logn, hashes, job_host.nh, P->d_win, jd,
                                                  logB_static, t);
        count_launch(P);
        taps = t;
        tstride = 0;
    }
    if (dynamic || job_host.stream) {
        dim3 grid(persist, groups);
        launch_k(P, k_bin_stream_2d, dim3(grid), dim3(256), 0, s, x, P->logn, job_host.nh, jd, logB_static,
                                             job_host.chunks, taps, tstride, part);
        count_launch(P);
    }
    if (dynamic) prof_mark(P, 10, s);
    if (dynamic || !job_host.stream) {
        dim3 grid(persist, job_host.nh);
        launch_k(P, k_bin_gather_2d, dim3(grid), dim3(256), 0, s, x, P->logn, hashes, job_host.nh, P->d_win, jd,
                                             logB_static, taps, tstride, part);
        count_launch(P);
    }
}

}  // namespace atsfft
