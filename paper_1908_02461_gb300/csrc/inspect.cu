// inspect.cu -- per-exec reset of the device state, and the bucket-order view of one
// hash's spectrum used by the inspection call atsfft_hash_spectrum.
#include "common.cuh"

namespace atsfft {

// Zeroes the statistics slots, the exec state and the compaction chunk counts (one
// launch instead of one memset node each).
__global__ void k_reset(uint32_t *stats, int64_t stats_words, uint32_t *state, int64_t state_words,
                        uint32_t *chunks, int64_t nchunks)
{
    chain_next();   // (launched plainly: the exec's first kernel follows whatever came before)
    const int64_t total = stats_words + state_words + nchunks;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (i < stats_words)
            stats[i] = 0u;
        else if (i < stats_words + state_words)
            state[i - stats_words] = 0u;
        else
            chunks[i - stats_words - state_words] = 0u;
    }
}

void launch_reset(const atsfft_plan_s *P, cudaStream_t s)
{
    static_assert(sizeof(HashStats) % 4 == 0 && sizeof(ExecState) % 4 == 0, "word-sized state");
    const int64_t sw = (int64_t)(sizeof(HashStats) * (kMaxLogB + kMaxLoops) / 4);
    const int64_t ew = (int64_t)(sizeof(ExecState) / 4);
    const int64_t total = sw + ew + P->nchunks;
    const int blocks = (int)((total + 255) / 256 < 64 ? (total + 255) / 256 : 64);
    k_reset<<<blocks, 256, 0, s>>>((uint32_t *)P->d_stats, sw, (uint32_t *)P->d_state, ew, P->d_blk,
                                   P->nchunks);
    count_launch(P);
}

// Inspection: Zhat[c] = P[sigma' c] exp(2 pi i c sigma' tau / B) in bucket order.
__global__ void k_unpermute(const float2 *spec, const HashParam *hp_dev, int ndim, int logB,
                            float2 *out)
{
    const HashParam hp = *hp_dev;
    const uint64_t B = 1ull << logB, Bm = B - 1;
    const int64_t nb = ndim == 1 ? (int64_t)B : (int64_t)(B * B);
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nb;
         c += (int64_t)gridDim.x * blockDim.x) {
        uint64_t idx, k;
        if (ndim == 1) {
            const uint64_t sp = hp.sinv[0] & Bm;
            idx = (sp * (uint64_t)c) & Bm;
            k = (idx * (hp.tau[0] & Bm)) & Bm;
        } else {
            const uint64_t c1 = (uint64_t)c >> logB, c2 = (uint64_t)c & Bm;
            const uint64_t j1 = ((hp.sinv[0] & Bm) * c1) & Bm, j2 = ((hp.sinv[1] & Bm) * c2) & Bm;
            idx = (j1 << logB) | j2;
            k = ((j1 * (hp.tau[0] & Bm)) + (j2 * (hp.tau[1] & Bm))) & Bm;
        }
        double sn, cs;
        sincospi(2.0 * (double)k / (double)B, &sn, &cs);
        const float2 v = spec[idx];
        out[c] = make_float2((float)(v.x * cs - v.y * sn), (float)(v.x * sn + v.y * cs));
    }
}

void launch_unpermute(const atsfft_plan_s *P, const float2 *spec, const HashParam *hash_dev,
                      int logB, float2 *out, cudaStream_t s)
{
    count_launch(P);
    k_unpermute<<<P->num_sms * 2, 256, 0, s>>>(spec, hash_dev, P->ndim, logB, out);
}

}  // namespace atsfft
