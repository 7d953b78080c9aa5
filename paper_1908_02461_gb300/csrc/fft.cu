// fft.cu -- batched B-point bucket DFTs ("do DFT with length B" in Algorithms 1-2;
// B x B in 2D): Zhat_c = sum_b z_b exp(-2 pi i c b / B), unscaled.
//
// One CTA transforms up to kSmallFFT points in shared memory (radix-2 decimation in
// time, bit-reversed load, table twiddles).  Larger 1D transforms use the four-step
// split B = P1 * P2 (j = j1 + P1 j2, k = k2 + P2 k1):
//   pass 0: Y[j1 + P1 k2] = exp(-2 pi i j1 k2 / B) * sum_j2 z[j1 + P1 j2] w_P2^(j2 k2)
//   pass 1: X[k2 + P2 k1] = sum_j1 Y[j1 + P1 k2] w_P1^(j1 k1).
// 2D is rows (pass 0) then columns (pass 1).  The first pass also sums the binning
// partials: hash h's input is `chunks` consecutive blocks of B (or B^2) values.
#include "common.cuh"

namespace atsfft {

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
        if (logB <= 12) {
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

// T adjacent transforms t0..t0+T-1 by the whole CTA (T * P <= kSmallFFT): element j of
// transform t0+u is src[u * in_bs + j * in_es] summed over `chunks` blocks
// chunk_stride apart; the result k (optionally twiddled by exp(-2 pi i t k / 2^tw_logB))
// goes to dst[u * out_bs + k * out_es].  Threads walk the tile along whichever stride
// is 1, so strided (column) transforms still load and store whole segments.
__device__ void fft_tile(const float2 *src, int64_t in_es, int64_t in_bs, int chunks,
                         int64_t chunk_stride, float2 *dst, int64_t out_es, int64_t out_bs,
                         int logP, int T, int tw_logB, int64_t t0, float2 *sm,
                         const float2 *__restrict__ tw)
{
    const int P = 1 << logP;
    const int TP = T * P;
    const bool in_rows = in_es == 1;     // walk j fastest, else walk the transforms fastest
    for (int idx = threadIdx.x; idx < TP; idx += blockDim.x) {
        const int u = in_rows ? idx >> logP : idx % T;
        const int j = in_rows ? idx & (P - 1) : idx / T;
        const float2 *p = src + (int64_t)u * in_bs + (int64_t)j * in_es;
        float2 v = p[0];
        for (int c = 1; c < chunks; c++) {
            const float2 w = p[(int64_t)c * chunk_stride];
            v.x += w.x;
            v.y += w.y;
        }
        const int r = logP ? (int)(__brev((unsigned)j) >> (32 - logP)) : 0;
        sm[u * P + r] = v;
    }
    __syncthreads();
    for (int lm = 1; lm <= logP; lm++) {
        const int half = 1 << (lm - 1);
        const int twstep = kSmallFFT >> lm;
        for (int k = threadIdx.x; k < TP / 2; k += blockDim.x) {
            const int u = k >> (logP - 1);
            const int kk = k & (P / 2 - 1);
            const int q = kk & (half - 1);
            const int i0 = u * P + ((kk >> (lm - 1)) << lm) + q;
            const int i1 = i0 + half;
            const float2 w = tw[q * twstep];
            const float2 a = sm[i0], b = sm[i1];
            const float2 wb = make_float2(w.x * b.x - w.y * b.y, w.x * b.y + w.y * b.x);
            sm[i0] = make_float2(a.x + wb.x, a.y + wb.y);
            sm[i1] = make_float2(a.x - wb.x, a.y - wb.y);
        }
        __syncthreads();
    }
    const bool out_rows = out_es == 1;
    for (int idx = threadIdx.x; idx < TP; idx += blockDim.x) {
        const int u = out_rows ? idx >> logP : idx % T;
        const int k = out_rows ? idx & (P - 1) : idx / T;
        float2 v = sm[u * P + k];
        if (tw_logB >= 0) {
            const int64_t m = ((t0 + u) * k) & (((int64_t)1 << tw_logB) - 1);
            float sn, cs;
            sincospif(-ldexpf((float)m, 1 - tw_logB), &sn, &cs);
            v = make_float2(v.x * cs - v.y * sn, v.x * sn + v.y * cs);
        }
        dst[(int64_t)u * out_bs + (int64_t)k * out_es] = v;
    }
    __syncthreads();
}

// Transforms per CTA: a tile of adjacent ones when they are strided, one otherwise.
__device__ __forceinline__ int tile_of(const FftShape &f)
{
    if (f.in_es == 1 && f.out_es == 1) return 1;
    int T = kSmallFFT >> f.logP;
    if (T > 16) T = 16;
    if (T > f.ntrans) T = f.ntrans;
    return T;
}

// Dynamic pass over the nh hashes of the job at B* (shape read on the device).
// part: [hash][chunk][B or B^2]; 1D four-step pass 0 writes `tmp`, pass 1 reads it;
// everything else ends in `fin` (2D pass 1 in place).
__global__ void __launch_bounds__(256) k_fft_pass(int ndim, int pass, const Job *job,
                                                  const float2 *__restrict__ part, float2 *tmp,
                                                  float2 *fin, const float2 *__restrict__ tw)
{
    __shared__ float2 sm[kSmallFFT];
    if (!job->active) return;
    const int logB = job->logB, nh = job->nh;
    const int chunks = pass == 0 ? job->chunks : 1;
    const FftShape f = fft_shape(ndim, logB, pass);
    if (!f.valid) return;
    const bool four_step = ndim == 1 && logB > 12;
    const float2 *in = pass == 0 ? part : (ndim == 1 ? tmp : fin);
    float2 *out = (pass == 0 && four_step) ? tmp : fin;
    const int64_t in_hash = (int64_t)chunks * f.hash_stride;
    const int T = tile_of(f);
    const int64_t tiles = f.ntrans / T;
    const int64_t total = (int64_t)nh * tiles;
    for (int64_t tr = blockIdx.x; tr < total; tr += gridDim.x) {
        const int64_t h = tr / tiles, t = (tr % tiles) * T;
        fft_tile(in + h * in_hash + t * f.in_bs, f.in_es, f.in_bs, chunks, f.hash_stride,
                 out + h * f.hash_stride + t * f.out_bs, f.out_es, f.out_bs, f.logP, T, f.tw_logB,
                 t, sm, tw);
    }
}

// Static batch: every job is one hash of its own B (the tuning trials).
struct FftJob {
    int32_t logB, chunks;
    int64_t in_off, tmp_off, out_off;
    int64_t tr_start;    // first transform of this job in the launch (per pass)
};

struct FftBatch {
    int njobs;
    int64_t total;
    FftJob j[kMaxLogB];
};

__global__ void __launch_bounds__(256) k_fft_batch(int ndim, int pass, const FftBatch Bt,
                                                   const float2 *__restrict__ part, float2 *tmp,
                                                   float2 *fin, const float2 *__restrict__ tw)
{
    __shared__ float2 sm[kSmallFFT];
    for (int64_t tr = blockIdx.x; tr < Bt.total; tr += gridDim.x) {
        int jb = 0;
        while (jb + 1 < Bt.njobs && tr >= Bt.j[jb + 1].tr_start) jb++;
        const FftJob &J = Bt.j[jb];
        const FftShape f = fft_shape(ndim, J.logB, pass);
        const int T = tile_of(f);
        const int64_t t = (tr - J.tr_start) * T;
        const bool four_step = ndim == 1 && J.logB > 12;
        const float2 *in =
            pass == 0 ? part + J.in_off : (ndim == 1 ? tmp + J.tmp_off : fin + J.out_off);
        float2 *out = (pass == 0 && four_step) ? tmp + J.tmp_off : fin + J.out_off;
        const int chunks = pass == 0 ? J.chunks : 1;
        fft_tile(in + t * f.in_bs, f.in_es, f.in_bs, chunks, f.hash_stride, out + t * f.out_bs,
                 f.out_es, f.out_bs, f.logP, T, f.tw_logB, t, sm, tw);
    }
}

// Dynamic job at B*: both passes always launched; each decides on the device.
void launch_bucket_fft_dynamic(const atsfft_plan_s *P, const Job *job, const float2 *part,
                               float2 *out, cudaStream_t s)
{
    const int grid = P->num_sms * 8;
    k_fft_pass<<<grid, 256, 0, s>>>(P->ndim, 0, job, part, P->d_fft_tmp, out, P->d_tw);
    count_launch(P);
    if (P->ndim == 2 || P->b_hi > 12) {
        k_fft_pass<<<grid, 256, 0, s>>>(P->ndim, 1, job, part, P->d_fft_tmp, out, P->d_tw);
        count_launch(P);
    }
}

// Static batch of single-hash jobs (logB[i], chunks[i], partial offset in_off[i],
// output offset out_off[i]); the four-step intermediate reuses the output offsets.
void launch_bucket_fft_batch(const atsfft_plan_s *P, int njobs, const int *logB, const int *chunks,
                             const int64_t *in_off, const int64_t *out_off, const float2 *part,
                             float2 *out, cudaStream_t s)
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
                if (lb <= 12) {
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
            // tiles of adjacent transforms, as tile_of() on the device
            int64_t T = 1;
            if (strided) {
                T = (int64_t)kSmallFFT >> logP;
                if (T > 16) T = 16;
                if (T > ntrans) T = ntrans;
            }
            ntrans /= T;
            FftJob &J = Bt.j[Bt.njobs++];
            J.logB = lb;
            J.chunks = chunks[i];
            J.in_off = in_off[i];
            J.tmp_off = out_off[i];
            J.out_off = out_off[i];
            J.tr_start = Bt.total;
            Bt.total += ntrans;
        }
        if (Bt.njobs == 0) continue;
        const int64_t cap = (int64_t)P->num_sms * 8;
        const int64_t grid = Bt.total < cap ? Bt.total : cap;
        k_fft_batch<<<(unsigned)grid, 256, 0, s>>>(P->ndim, pass, Bt, part, P->d_fft_tmp, out,
                                                   P->d_tw);
        count_launch(P);
    }
}

}  // namespace atsfft
