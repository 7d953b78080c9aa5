// locate.cu -- keep the coordinates that were voted for in at least half of the
// location loops (Section II-B), in ascending order, and clear the vote counters.
//
// Votes are byte counters packed four to a 32-bit word.  Three kernels: per-block
// counts, one exclusive scan over the blocks, then an ordered write (each block writes
// its coordinates at its scanned offset, in index order within the block).
#include "common.cuh"

namespace atsfft {

constexpr int kCompactThreads = 256;
constexpr int kWordsPerThread = 4;   // 16 coordinates per thread, 4096 per block

__device__ __forceinline__ uint32_t count_kept(uint32_t w, uint32_t need)
{
    return ((w & 0xffu) >= need) + (((w >> 8) & 0xffu) >= need) + (((w >> 16) & 0xffu) >= need) +
           ((w >> 24) >= need);
}

__global__ void __launch_bounds__(kCompactThreads) k_compact_count(const uint32_t *votes,
                                                                   int64_t nwords, uint32_t need,
                                                                   uint32_t *blk)
{
    __shared__ uint32_t red[kCompactThreads / 32];
    const int64_t w0 = ((int64_t)blockIdx.x * kCompactThreads + threadIdx.x) * kWordsPerThread;
    uint32_t c = 0;
    for (int k = 0; k < kWordsPerThread; k++)
        if (w0 + k < nwords) c += count_kept(votes[w0 + k], need);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int i = 0; i < kCompactThreads / 32; i++) t += red[i];
        blk[blockIdx.x] = t;
    }
}

// Single block: exclusive scan of the block counts in place; total -> state->count.
__global__ void k_compact_scan(uint32_t *blk, int64_t nblk, ExecState *state)
{
    __shared__ uint32_t part[1024];
    const int64_t per = (nblk + blockDim.x - 1) / blockDim.x;
    const int64_t b0 = threadIdx.x * per;
    uint32_t s = 0;
    for (int64_t i = b0; i < b0 + per && i < nblk; i++) s += blk[i];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t acc = 0;
        for (unsigned t = 0; t < blockDim.x; t++) {
            const uint32_t v = part[t];
            part[t] = acc;
            acc += v;
        }
        state->count = acc;
    }
    __syncthreads();
    uint32_t acc = part[threadIdx.x];
    for (int64_t i = b0; i < b0 + per && i < nblk; i++) {
        const uint32_t v = blk[i];
        blk[i] = acc;
        acc += v;
    }
}

__global__ void __launch_bounds__(kCompactThreads) k_compact_write(uint32_t *votes, int64_t nwords,
                                                                   uint32_t need,
                                                                   const uint32_t *blk,
                                                                   int64_t *loc, int64_t capacity)
{
    __shared__ uint32_t warp_sum[kCompactThreads / 32];
    const int64_t w0 = ((int64_t)blockIdx.x * kCompactThreads + threadIdx.x) * kWordsPerThread;
    uint32_t words[kWordsPerThread];
    uint32_t c = 0;
    for (int k = 0; k < kWordsPerThread; k++) {
        words[k] = (w0 + k < nwords) ? votes[w0 + k] : 0u;
        c += count_kept(words[k], need);
    }
    // block-wide exclusive scan of c
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) warp_sum[wid] = incl;
    __syncthreads();
    uint32_t before = 0;
    for (int i = 0; i < wid; i++) before += warp_sum[i];
    int64_t pos = (int64_t)blk[blockIdx.x] + before + incl - c;
    for (int k = 0; k < kWordsPerThread; k++) {
        for (int by = 0; by < 4; by++) {
            if (((words[k] >> (8 * by)) & 0xffu) >= need) {
                if (pos < capacity) loc[pos] = (w0 + k) * 4 + by;
                pos++;
            }
        }
        if (w0 + k < nwords && words[k]) votes[w0 + k] = 0u;
    }
}

void launch_compact(const atsfft_plan_s *P, int64_t *d_loc, int64_t capacity, cudaStream_t s)
{
    const uint32_t need = (uint32_t)((P->L_loc + 1) / 2);
    const int64_t per_block = (int64_t)kCompactThreads * kWordsPerThread;
    const int64_t nblk = (P->nvote_words + per_block - 1) / per_block;
    count_launch(P, 3);
    k_compact_count<<<(unsigned)nblk, kCompactThreads, 0, s>>>(P->d_votes, P->nvote_words, need,
                                                              P->d_blk);
    k_compact_scan<<<1, 1024, 0, s>>>(P->d_blk, nblk, P->d_state);
    k_compact_write<<<(unsigned)nblk, kCompactThreads, 0, s>>>(P->d_votes, P->nvote_words, need,
                                                              P->d_blk, d_loc, capacity);
}

}  // namespace atsfft
