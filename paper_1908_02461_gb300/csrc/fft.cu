// fft.cu -- batched B-point bucket DFTs ("do DFT with length B" in Algorithms 1-2;
// B x B in 2D): Zhat_c = sum_b z_b exp(-2 pi i c b / B), unscaled.
//
// One CTA transforms up to kSmallFFT points in shared memory (radix-2 decimation in
// time, bit reversal folded into the loads, twiddles from a shared-memory copy of the
// table entries of its length, loaded together with the data); 1D transforms of more than
// 2^kSinglePassLog points use the four-step split B = P1 * P2 (j = j1 + P1 j2,
// k = k2 + P2 k1), which spreads one transform over many CTAs:
//   pass 0: Y[j1 + P1 k2] = exp(-2 pi i j1 k2 / B) * sum_j2 z[j1 + P1 j2] w_P2^(j2 k2)
//   pass 1: X[k2 + P2 k1] = sum_j1 Y[j1 + P1 k2] w_P1^(j1 k1).
// 2D is rows (pass 0) then columns (pass 1).  The first pass also sums the binning
// partials: hash h's input is `chunks` consecutive blocks of B (or B^2) values.
#include "common.cuh"

namespace atsfft {

// 1D transforms of up to 2^kSinglePassLog points run in one CTA; larger ones take the
// four-step split over two passes (more CTAs per transform, each with a short chain).
constexpr int kSinglePassLog = 10;
constexpr int kSmallFFTLog = 12;
static_assert((1 << kSmallFFTLog) == kSmallFFT, "kSmallFFTLog");

struct FftShape {
    int logP;            // transform length
    int ntrans;          // transforms per hash
    int64_t in_es, in_bs, out_es, out_bs;
    int64_t hash_stride; // B or B^2
    int tw_logB;         // >= 0: post-multiply by exp(-2 pi i t k / 2^tw_logB)
    int valid;
};

__device__ FftShape fft_shape(int ndim, int logB, int pass)
{
    FftShape f;
    f.valid = 1;
    f.tw_logB = -1;
    if (ndim == 1) {
        const int64_t B = (int64_t)1 << logB;
        f.hash_stride = B;
        if (logB <= kSinglePassLog) {
            if (pass == 1) { f.valid = 0; return f; }
            f.logP = logB; f.ntrans = 1;
            f.in_es = 1; f.in_bs = B; f.out_es = 1; f.out_bs = B;
        } else {
            const int l1 = logB / 2, l2 = logB - l1;
            const int64_t P1 = (int64_t)1 << l1, P2 = (int64_t)1 << l2;
            if (pass == 0) {
                f.logP = l2; f.ntrans = (int)P1;
                f.in_es = P1; f.in_bs = 1; f.out_es = P1; f.out_bs = 1;
                f.tw_logB = logB;
            } else {
                f.logP = l1; f.ntrans = (int)P2;
                f.in_es = 1; f.in_bs = P1; f.out_es = P2; f.out_bs = 1;
            }
        }
    } else {
        const int64_t B = (int64_t)1 << logB;
        f.hash_stride = B * B;
        f.logP = logB; f.ntrans = (int)B;
        if (pass == 0) { f.in_es = 1; f.in_bs = B; f.out_es = 1; f.out_bs = B; }
        else { f.in_es = B; f.in_bs = 1; f.out_es = B; f.out_bs = 1; }
    }
    return f;
}

// Shared-memory index with one pad slot per 16 entries: the register passes below read
// 8-value groups at strides 1, 8, 64, ... (positions in a group are a power of two
// apart) and the padding spreads each half-warp's 64-bit accesses over the banks.
constexpr int kSmemPadded = kSmallFFT + kSmallFFT / 16;
constexpr int kMaxRadixLog = 3;     // 8-value register groups
constexpr int kFftThreads = kSmallFFT >> kMaxRadixLog;

__device__ __forceinline__ int padi(int i) { return i + (i >> 4); }

__device__ __forceinline__ void butterfly(float2 &a, float2 &b, float2 w)
{
    const float2 wb = make_float2(w.x * b.x - w.y * b.y, w.x * b.y + w.y * b.x);
    b = make_float2(a.x - wb.x, a.y - wb.y);
    a = make_float2(a.x + wb.x, a.y + wb.y);
}

// R consecutive radix-2 decimation-in-time stages lm0 .. lm0+R-1 on one group of 2^R
// values held in registers: v[j] is the value at position base + q + j * 2^(lm0-1).
// Stage lm pairs positions p and p + 2^(lm-1) with the twiddle w_(2^lm)^(p mod 2^(lm-1)),
// exactly as the one-stage-at-a-time form.  stw[m] = w_P^m (m < P / 2, P = 2^logP), so
// w_(2^lm)^qq = stw[qq << (logP - lm)].
template <int R>
__device__ __forceinline__ void group_stages(float2 (&v)[1 << R], int q, int lm0,
                                             const float2 *stw, int logP)
{
    const int half = 1 << (lm0 - 1);
#pragma unroll
    for (int s = 0; s < R; s++) {
        const int twsh = logP - (lm0 + s);
#pragma unroll
        for (int j0 = 0; j0 < (1 << R); j0++) {
            if (j0 & (1 << s)) continue;
            const int qq = q + (j0 & ((1 << s) - 1)) * half;
            butterfly(v[j0], v[j0 | (1 << s)], stw[qq << twsh]);
        }
    }
}

// The three radix-2 stages of a group of 8 (positions base + q + j 2^(lm0-1)) with the
// twiddles factored: stage s uses W_(2^(lm0+s))^q times W_(2^(s+1))^(j0 mod 2^s), and
// W_(2^(lm0+s))^q = t2^(2^(2-s)) with t2 = W_(2^(lm0+2))^q, so one table entry (t2) and
// the constants 1, -i, W_8, -i W_8 give all twelve butterfly twiddles.
__device__ __forceinline__ float2 mul_mi(float2 b) { return make_float2(b.y, -b.x); }   // -i b

__device__ __forceinline__ void bfly(float2 &a, float2 &b, float2 wb)
{
    b = make_float2(a.x - wb.x, a.y - wb.y);
    a = make_float2(a.x + wb.x, a.y + wb.y);
}

__device__ __forceinline__ float2 cmulf(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ __forceinline__ void radix8_stages(float2 (&v)[8], float2 t2)
{
    constexpr float r2 = 0.70710678118654752440f;
    const float2 t1 = cmulf(t2, t2), t0 = cmulf(t1, t1);
    const float2 t2w = make_float2((t2.x + t2.y) * r2, (t2.y - t2.x) * r2);   // t2 W_8
#pragma unroll
    for (int j0 = 0; j0 < 8; j0 += 2) bfly(v[j0], v[j0 + 1], cmulf(t0, v[j0 + 1]));
    bfly(v[0], v[2], cmulf(t1, v[2]));
    bfly(v[1], v[3], mul_mi(cmulf(t1, v[3])));
    bfly(v[4], v[6], cmulf(t1, v[6]));
    bfly(v[5], v[7], mul_mi(cmulf(t1, v[7])));
    bfly(v[0], v[4], cmulf(t2, v[4]));
    bfly(v[1], v[5], cmulf(t2w, v[5]));
    bfly(v[2], v[6], mul_mi(cmulf(t2, v[6])));
    bfly(v[3], v[7], mul_mi(cmulf(t2w, v[7])));
}

// The same for q = 0 (the first three stages): all twiddles are 1, -i, W_8 or -i W_8.
__device__ __forceinline__ void radix8_first(float2 (&v)[8])
{
    constexpr float r2 = 0.70710678118654752440f;
#pragma unroll
    for (int j0 = 0; j0 < 8; j0 += 2) bfly(v[j0], v[j0 + 1], v[j0 + 1]);
    bfly(v[0], v[2], v[2]);
    bfly(v[1], v[3], mul_mi(v[3]));
    bfly(v[4], v[6], v[6]);
    bfly(v[5], v[7], mul_mi(v[7]));
    bfly(v[0], v[4], v[4]);
    bfly(v[1], v[5], make_float2((v[5].x + v[5].y) * r2, (v[5].y - v[5].x) * r2));
    bfly(v[2], v[6], mul_mi(v[6]));
    bfly(v[3], v[7], make_float2((v[7].y - v[7].x) * r2, -(v[7].x + v[7].y) * r2));
}

// Bit reversal of the low logP bits (positions inside one transform).
__device__ __forceinline__ int bitrev_in(int j, int logP)
{
    return (int)(__brev((unsigned)j) >> (32 - logP));
}

// First group of stages (lm0 = 1), in place: the loads stored every transform in
// bit-reversed order, so group g is the 2^R consecutive positions g 2^R + j.
template <int R>
__device__ __forceinline__ void first_stages(float2 *sm, int TP, const float2 *stw, int logP)
{
    constexpr int E = 1 << R;
    for (int g = threadIdx.x; g < (TP >> R); g += blockDim.x) {
        float2 v[E];
#pragma unroll
        for (int j = 0; j < E; j++) v[j] = sm[padi(g * E + j)];
        if constexpr (R == 3)
            radix8_first(v);
        else
            group_stages<R>(v, 0, 1, stw, logP);
#pragma unroll
        for (int j = 0; j < E; j++) sm[padi(g * E + j)] = v[j];
    }
    __syncthreads();
}

// Later groups of stages, in place: each group reads and writes only its own positions.
template <int R>
__device__ __forceinline__ void next_stages(float2 *sm, int TP, int lm0, const float2 *stw,
                                            int logP)
{
    constexpr int E = 1 << R;
    const int half = 1 << (lm0 - 1);
    for (int g = threadIdx.x; g < (TP >> R); g += blockDim.x) {
        const int q = g & (half - 1);
        const int base = ((g >> (lm0 - 1)) << (lm0 - 1 + R)) + q;
        float2 v[E];
#pragma unroll
        for (int j = 0; j < E; j++) v[j] = sm[padi(base + j * half)];
        if constexpr (R == 3)
            radix8_stages(v, stw[q << (logP - (lm0 + 2))]);   // w_(2^(lm0+2))^q
        else
            group_stages<R>(v, q, lm0, stw, logP);
#pragma unroll
        for (int j = 0; j < E; j++) sm[padi(base + j * half)] = v[j];
    }
    __syncthreads();
}

constexpr int kMaxTile = 8;    // transforms per tile

// Shared memory of the FFT kernels: the padded tile, then the stage twiddles of the
// current length (w_P^m, m < P / 2 <= kSmallFFT / 2).
constexpr int kStwEntries = kSmallFFT / 2;
constexpr size_t kFftSmemBytes = sizeof(float2) * (size_t)(kSmemPadded + kStwEntries);

// stw[m] = w_P^m = exp(-2 pi i m / P) for m < P / 2, from the table entry tw[m 4096 / P];
// the caller's next barrier (the one after a tile's loads) makes it visible.
__device__ __forceinline__ void load_stage_twiddles(float2 *stw, int logP, const float2 *__restrict__ tw)
{
    for (int m = threadIdx.x; m < ((1 << logP) >> 1); m += blockDim.x)
        stw[m] = __ldg(&tw[m << (kSmallFFTLog - logP)]);
}

// exp(-2 pi i m / B) for B = 2^logB <= 2^24, m < B: sincospif of the exact dyadic
// argument 2 m / B (no table, so no memory round trip in the tile's epilogue).
__device__ __forceinline__ float2 four_step_twiddle(uint32_t m, int logB)
{
    float sn, cs;
    sincospif(ldexpf((float)m, 1 - logB), &sn, &cs);
    return make_float2(cs, -sn);
}

// T = 2^logT adjacent transforms t0..t0+T-1 by the whole CTA (T * P <= kSmallFFT):
// element j of transform t0+u is src[u * in_bs + j * in_es] summed over `chunks` blocks
// chunk_stride apart; the result k (optionally twiddled by exp(-2 pi i t k / 2^tw_logB))
// goes to dst[u * out_bs + k * out_es] (all offsets inside a tile fit in 32 bits).
// Either in_es == 1 (each transform contiguous:
// threads walk j) or in_bs == 1 (the T transforms interleaved: a thread moves the T
// contiguous values of one j with 16-byte accesses); the same for the output.  The
// log2 P radix-2 stages run three at a time on 8-value groups in registers.
__device__ void fft_tile(const float2 *src, int in_es, int in_bs, int chunks,
                         int chunk_stride, float2 *dst, int out_es, int out_bs,
                         int logP, int logT, int tw_logB, int64_t t0, float2 *sm,
                         const float2 *stw, float *edst, uint32_t *emax)
{
    const int P = 1 << logP, T = 1 << logT;
    const int TP = T << logP;
    if (in_es == 1 || T == 1) {
        // four elements per thread at a time, their chunk loads issued together
        for (int idx0 = threadIdx.x; idx0 < TP; idx0 += 4 * blockDim.x) {
            const float2 *p[4];
            float2 v[4];
#pragma unroll
            for (int e = 0; e < 4; e++) {
                const int idx = idx0 + e * blockDim.x;
                const int u = (idx < TP ? idx : 0) >> logP, j = (idx < TP ? idx : 0) & (P - 1);
                p[e] = src + u * in_bs + j;
                v[e] = idx < TP ? p[e][0] : make_float2(0.f, 0.f);
            }
#pragma unroll 2
            for (int c = 1; c < chunks; c++) {
                float2 w[4];
#pragma unroll
                for (int e = 0; e < 4; e++)
                    w[e] = idx0 + e * (int)blockDim.x < TP ? p[e][c * chunk_stride] : make_float2(0.f, 0.f);
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    v[e].x += w[e].x;
                    v[e].y += w[e].y;
                }
            }
#pragma unroll
            for (int e = 0; e < 4; e++) {
                const int idx = idx0 + e * blockDim.x;
                if (idx < TP)
                    sm[padi(((idx >> logP) << logP) + bitrev_in(idx & (P - 1), logP))] = v[e];
            }
        }
    } else {
        for (int j = threadIdx.x; j < P; j += blockDim.x) {
            const float4 *p = reinterpret_cast<const float4 *>(src + j * in_es);
            const int jr = bitrev_in(j, logP);
            // up to eight transforms (four 16-byte loads per chunk) at a time, the loads of
            // a chunk issued together
            for (int u0 = 0; u0 < T; u0 += 8) {
                const int nq = min(4, (T - u0) >> 1);   // 16-byte loads (two transforms each)
                float4 a[4];
#pragma unroll
                for (int q = 0; q < 4; q++)
                    a[q] = q < nq ? p[(u0 >> 1) + q] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 2
                for (int c = 1; c < chunks; c++) {
                    const float4 *pc = p + ((c * chunk_stride) >> 1) + (u0 >> 1);
                    float4 w[4];
#pragma unroll
                    for (int q = 0; q < 4; q++) w[q] = q < nq ? pc[q] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                    for (int q = 0; q < 4; q++) {
                        a[q].x += w[q].x; a[q].y += w[q].y; a[q].z += w[q].z; a[q].w += w[q].w;
                    }
                }
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    if (q < nq) {
                        const int u = u0 + 2 * q;
                        sm[padi((u << logP) + jr)] = make_float2(a[q].x, a[q].y);
                        sm[padi(((u + 1) << logP) + jr)] = make_float2(a[q].z, a[q].w);
                    }
                }
            }
        }
    }
    __syncthreads();
    // stages 1 .. logP: groups of three (the loads already bit-reversed each transform)
    const int r0 = logP < kMaxRadixLog ? logP : kMaxRadixLog;
    switch (r0) {
    case 3: first_stages<3>(sm, TP, stw, logP); break;
    case 2: first_stages<2>(sm, TP, stw, logP); break;
    case 1: first_stages<1>(sm, TP, stw, logP); break;
    default: break;
    }
    for (int lm0 = r0 + 1; lm0 <= logP;) {
        const int r = logP - lm0 + 1 < kMaxRadixLog ? logP - lm0 + 1 : kMaxRadixLog;
        switch (r) {
        case 3: next_stages<3>(sm, TP, lm0, stw, logP); break;
        case 2: next_stages<2>(sm, TP, lm0, stw, logP); break;
        default: next_stages<1>(sm, TP, lm0, stw, logP); break;
        }
        lm0 += r;
    }
    const uint32_t bmask = tw_logB >= 0 ? (uint32_t)((1 << tw_logB) - 1) : 0u;
    float emx = 0.f;
    if (out_es == 1 || T == 1) {
        for (int idx = threadIdx.x; idx < TP; idx += blockDim.x) {
            const int u = idx >> logP, k = idx & (P - 1);
            float2 v = sm[padi(idx)];
            if (tw_logB >= 0) {
                const float2 w = four_step_twiddle((uint32_t)((t0 + u) * k) & bmask, tw_logB);
                v = make_float2(v.x * w.x - v.y * w.y, v.x * w.y + v.y * w.x);
            }
            const int o = u * out_bs + k;
            dst[o] = v;
            if (edst) {
                const float e = fmaf(v.x, v.x, v.y * v.y);
                edst[o] = e;
                emx = fmaxf(emx, e);
            }
        }
    } else {
        // items (k, pair of transforms u, u + 1), consecutive threads on consecutive k: every
        // thread of the CTA takes part; one 16-byte store per item
        const int items = P * (T >> 1);
#pragma unroll 2
        for (int it = threadIdx.x; it < items; it += blockDim.x) {
            const int k = it & (P - 1), u = (it >> logP) << 1;
            float2 a = sm[padi((u << logP) + k)], c = sm[padi(((u + 1) << logP) + k)];
            if (tw_logB >= 0) {
                const float2 wa = four_step_twiddle((uint32_t)((t0 + u) * k) & bmask, tw_logB);
                const float2 wc = four_step_twiddle((uint32_t)((t0 + u + 1) * k) & bmask, tw_logB);
                a = make_float2(a.x * wa.x - a.y * wa.y, a.x * wa.y + a.y * wa.x);
                c = make_float2(c.x * wc.x - c.y * wc.y, c.x * wc.y + c.y * wc.x);
            }
            reinterpret_cast<float4 *>(dst + k * out_es)[u >> 1] = make_float4(a.x, a.y, c.x, c.y);
            if (edst) {
                float *eo = edst + k * out_es;
                const float ea = fmaf(a.x, a.x, a.y * a.y), ec = fmaf(c.x, c.x, c.y * c.y);
                eo[u] = ea;
                eo[u + 1] = ec;
                emx = fmaxf(emx, fmaxf(ea, ec));
            }
        }
    }
    if (emax) {
        // block maximum of the energies, one atomic per tile (E >= 0: bit order = order)
        __shared__ float wmax[32];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) emx = fmaxf(emx, __shfl_xor_sync(0xffffffffu, emx, off));
        if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = emx;
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < (int)(blockDim.x >> 5); w++) emx = fmaxf(emx, wmax[w]);
            if (emx > 0.f) atomicMax(emax, __float_as_uint(emx));
        }
    }
    __syncthreads();
}

// Transforms per CTA: a tile of adjacent ones (strided, or contiguous rows of a 2D pass),
// up to kSmallFFT points; one where a hash has a single transform.
__device__ __forceinline__ int tile_of(const FftShape &f)
{
    int T = kSmallFFT >> f.logP;
    if (T > kMaxTile) T = kMaxTile;
    if (T > f.ntrans) T = f.ntrans;
    return T;
}

// Input loads per tile (values x partial chunks) above which a strided tile is split
// further, so that hashes with many partial chunks spread over more CTAs.
constexpr int64_t kTileLoads = 8192;

// Is `pass` the one that writes the final spectrum?
__device__ __forceinline__ bool final_pass(int ndim, int logB, int pass)
{
    return (ndim == 1 && logB <= kSinglePassLog) ? pass == 0 : pass == 1;
}

// CTAs per SM of the location pass (measured: 3 beats 2 there; the tuning batches, whose
// first pass also adds partial chunks, keep 2 and their registers).
constexpr int kPassCtas = 3;

// Dynamic pass over the nh hashes of the job at B* (shape read on the device).
// part: [hash][chunk][B or B^2]; 1D four-step pass 0 writes `tmp`, pass 1 reads it;
// everything else ends in `fin` (2D pass 1 in place).  The final pass also writes the
// energies |Zhat|^2 of the first n_energy hashes (layout of `fin`, base `energy`) and
// their maxima into stats[kMaxLogB + h].max_bits.
__global__ void __launch_bounds__(kFftThreads, kPassCtas) k_fft_pass(int ndim, int pass, const Job *job,
                                                  const float2 *__restrict__ part, float2 *tmp,
                                                  float2 *fin, const float2 *__restrict__ tw,
                                                  float *energy, HashStats *stats, int n_energy)
{
    chain_wait();
    chain_next();
    extern __shared__ float2 fft_dsm[];
    float2 *sm = fft_dsm, *stw = fft_dsm + kSmemPadded;
    if (!job->active) return;
    const int logB = job->logB, nh = job->nh;
    const int chunks = pass == 0 ? job->chunks : 1;
    const FftShape f = fft_shape(ndim, logB, pass);
    if (!f.valid) return;
    const bool four_step = ndim == 1 && logB > kSinglePassLog;
    const float2 *in = pass == 0 ? part : (ndim == 1 ? tmp : fin);
    float2 *out = (pass == 0 && four_step) ? tmp : fin;
    const int64_t in_hash = (int64_t)chunks * f.hash_stride;
    int T = tile_of(f);
    if (f.in_es != 1 || f.out_es != 1)
        while (T > 4 && ((int64_t)T << f.logP) * chunks > kTileLoads) T >>= 1;
    else
        while (T > 1 && ((int64_t)T << f.logP) * chunks > kTileLoads) T >>= 1;
    const int64_t tiles = f.ntrans / T;
    const int64_t total = (int64_t)nh * tiles;
    const bool fin_pass = energy && final_pass(ndim, logB, pass);
    if ((int64_t)blockIdx.x < total) load_stage_twiddles(stw, f.logP, tw);   // one length per pass
    for (int64_t tr = blockIdx.x; tr < total; tr += gridDim.x) {
        const int64_t h = tr / tiles, t = (tr % tiles) * T;
        const bool e = fin_pass && h < n_energy;
        fft_tile(in + h * in_hash + t * f.in_bs, f.in_es, f.in_bs, chunks, f.hash_stride,
                 out + h * f.hash_stride + t * f.out_bs, f.out_es, f.out_bs, f.logP, __ffs(T) - 1,
                 f.tw_logB,
                 t, sm, stw, e ? energy + h * f.hash_stride + t * f.out_bs : nullptr,
                 e ? &stats[kMaxLogB + h].max_bits : nullptr);
    }
}

// Static batch: every job is one hash of its own B (the tuning trials).
struct FftJob {
    int32_t logB, chunks;
    int32_t T, pad;      // transforms per tile in this pass
    int64_t in_off, tmp_off, out_off;
    int64_t tr_start;    // first tile of this job in the launch
};


struct FftBatch {
    int njobs;
    int64_t total;
    FftJob j[kMaxLogB];
};

// energy != nullptr: the final pass also writes |Zhat|^2 at the output offsets of
// `energy` and the maximum into stats[logB].max_bits (the tuning trial's slot).  A set
// *skip (device flag) makes every CTA return at once.
__global__ void __launch_bounds__(kFftThreads, 2) k_fft_batch(int ndim, int pass, const FftBatch Bt,
                                                   const float2 *__restrict__ part, float2 *tmp,
                                                   float2 *fin, const float2 *__restrict__ tw,
                                                   float *energy, HashStats *stats,
                                                   const int *skip)
{
    chain_wait();
    chain_next();
    extern __shared__ float2 fft_dsm[];
    float2 *sm = fft_dsm, *stw = fft_dsm + kSmemPadded;
    if (skip && *skip) return;
    int stw_logP = -1;   // length whose stage twiddles stw holds (a CTA's tiles span jobs)
    for (int64_t tr = blockIdx.x; tr < Bt.total; tr += gridDim.x) {
        int jb = 0;
        while (jb + 1 < Bt.njobs && tr >= Bt.j[jb + 1].tr_start) jb++;
        const FftJob &J = Bt.j[jb];
        const FftShape f = fft_shape(ndim, J.logB, pass);
        const int T = J.T;
        const int64_t t = (tr - J.tr_start) * T;
        const bool four_step = ndim == 1 && J.logB > kSinglePassLog;
        const float2 *in =
            pass == 0 ? part + J.in_off : (ndim == 1 ? tmp + J.tmp_off : fin + J.out_off);
        float2 *out = (pass == 0 && four_step) ? tmp + J.tmp_off : fin + J.out_off;
        const int chunks = pass == 0 ? J.chunks : 1;
        const bool e = energy && final_pass(ndim, J.logB, pass);
        if (f.logP != stw_logP) {   // the previous tile ended with a barrier
            load_stage_twiddles(stw, f.logP, tw);
            stw_logP = f.logP;
        }
        fft_tile(in + t * f.in_bs, f.in_es, f.in_bs, chunks, f.hash_stride, out + t * f.out_bs,
                 f.out_es, f.out_bs, f.logP, __ffs(T) - 1, f.tw_logB, t, sm, stw,
                 e ? energy + J.out_off + t * f.out_bs : nullptr,
                 e ? &stats[J.logB].max_bits : nullptr);
    }
}

// Dynamic job at B*: both passes always launched; each decides on the device.
void launch_bucket_fft_dynamic(const atsfft_plan_s *P, const Job *job, const float2 *part,
                               float2 *out, float *energy, int n_energy, cudaStream_t s)
{
    const int grid = P->num_sms * kPassCtas;   // resident CTAs; a grid-stride loop covers the tiles
    cudaFuncSetAttribute((const void *)k_fft_pass, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kFftSmemBytes);
    launch_k(P, k_fft_pass, dim3(grid), dim3(kFftThreads), kFftSmemBytes, s, P->ndim, 0, job, part, P->d_fft_tmp, out, P->d_tw,
                                            energy, P->d_stats, n_energy);
    count_launch(P);
    if (P->ndim == 2 || P->b_hi > kSinglePassLog) {
        launch_k(P, k_fft_pass, dim3(grid), dim3(kFftThreads), kFftSmemBytes, s, P->ndim, 1, job, part, P->d_fft_tmp, out, P->d_tw,
                                                energy, P->d_stats, n_energy);
        count_launch(P);
    }
}

// Static batch of single-hash jobs (logB[i], chunks[i], partial offset in_off[i],
// output offset out_off[i]); the four-step intermediate reuses the output offsets.
void launch_bucket_fft_batch(const atsfft_plan_s *P, int njobs, const int *logB, const int *chunks,
                             const int64_t *in_off, const int64_t *out_off, const float2 *part,
                             float2 *out, float *energy, const int *skip, cudaStream_t s)
{
    for (int pass = 0; pass < 2; pass++) {
        FftBatch Bt;
        Bt.njobs = 0;
        Bt.total = 0;
        for (int i = 0; i < njobs; i++) {
            const int lb = logB[i];
            int64_t ntrans;
            int logP;
            bool strided;
            if (P->ndim == 1) {
                if (lb <= kSinglePassLog) {
                    if (pass == 1) continue;
                    ntrans = 1;
                    logP = lb;
                    strided = false;
                } else {
                    ntrans = (int64_t)1 << (pass == 0 ? lb / 2 : lb - lb / 2);
                    logP = pass == 0 ? lb - lb / 2 : lb / 2;
                    strided = true;
                }
            } else {
                ntrans = (int64_t)1 << lb;
                logP = lb;
                strided = pass == 1;
            }
            // tiles of adjacent transforms (whole 32-byte sectors: T >= 4 when strided),
            // smaller where the partial chunks make a tile's input large
            int64_t T = (int64_t)kSmallFFT >> logP;
            if (T > kMaxTile) T = kMaxTile;
            if (T > ntrans) T = ntrans;
            {
                const int64_t ch = pass == 0 ? chunks[i] : 1;
                const int64_t floor_T = strided ? 4 : 1;
                while (T > floor_T && (T << logP) * ch > kTileLoads) T >>= 1;
            }
            ntrans /= T;
            FftJob &J = Bt.j[Bt.njobs++];
            J.logB = lb;
            J.chunks = chunks[i];
            J.T = (int32_t)T;
            J.pad = 0;
            J.in_off = in_off[i];
            J.tmp_off = out_off[i];
            J.out_off = out_off[i];
            J.tr_start = Bt.total;
            Bt.total += ntrans;
        }
        if (Bt.njobs == 0) continue;
        const int64_t cap = (int64_t)P->num_sms * 2;
        const int64_t grid = Bt.total < cap ? Bt.total : cap;
        cudaFuncSetAttribute((const void *)k_fft_batch, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kFftSmemBytes);
        launch_k(P, k_fft_batch, dim3((unsigned)grid), dim3(kFftThreads), kFftSmemBytes, s, P->ndim, pass, Bt, part, P->d_fft_tmp, out,
                                                   P->d_tw, energy, P->d_stats, skip);
        count_launch(P);
    }
}

}  // namespace atsfft
