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
#include "common.cuh"

namespace atsfft {

constexpr int kGroup = 16;   // hashes accumulated together per thread

__device__ __forceinline__ float fast_exp2(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float fast_rcp(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// S_b = sin(pi b / B) exp(i pi b / n)
__device__ __forceinline__ float2 bucket_factor(uint32_t b, int logB, int logn)
{
    float s1 = sinpif(ldexpf((float)b, -logB));
    float sc, cc;
    sincospif(ldexpf((float)b, -logn), &sc, &cc);
    return make_float2(s1 * cc, s1 * sc);
}

// ---------------------------------------------------------------------------------
// 1D, warp per bucket: lanes walk the taps t = b + u B of the window, each tap computed
// once and applied to every hash of the group (gathering x at each hash's position).
// ---------------------------------------------------------------------------------
__global__ void k_bin_gather_1d(const float2 *__restrict__ x, int logn, const HashParam *hashes,
                                int nh, const WindowParam *win, const Job *job_dev,
                                int logB_static, float2 *__restrict__ out)
{
    int logB = logB_static;
    if (job_dev) {
        if (!job_dev->active || job_dev->stream) return;
        logB = job_dev->logB;
        nh = job_dev->nh;
    }
    const int group0 = blockIdx.y * kGroup;
    if (group0 >= nh) return;
    const int ng = min(kGroup, nh - group0);
    const uint32_t n = 1u << logn, mask = n - 1, B = 1u << logB;
    const int D = (int)(n >> logB);
    const WindowParam w = win[logB];
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    uint32_t sig[kGroup], tau[kGroup];
#pragma unroll
    for (int g = 0; g < kGroup; g++) {
        const HashParam hp = hashes[group0 + (g < ng ? g : 0)];
        sig[g] = hp.sigma[0];
        tau[g] = hp.tau[0];
    }
    for (int64_t bw = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); bw < B; bw += warps) {
        const int b = (int)bw;
        // taps t = b + u B with |t| <= h
        const int u_lo = -((w.h + b) >> logB);          // ceil((-h - b) / B)
        const int u_hi = (w.h - b) >> logB;             // floor((h - b) / B)
        float2 acc[kGroup];
#pragma unroll
        for (int g = 0; g < kGroup; g++) acc[g] = make_float2(0.f, 0.f);
        for (int u = u_lo + lane; u <= u_hi; u += 32) {
            const int t = b + u * (int)B;
            if (t == 0) continue;                       // centre tap handled below
            const float tf = (float)t;
            const float f = fast_exp2(fmaf(-w.k2 * tf, tf, w.log2c)) * fast_rcp(tf);
            float rs, rc;
            sincospif(ldexpf((float)u, -(logn - logB)), &rs, &rc);
            if (u & 1) { rs = -rs; rc = -rc; }
            const float2 c = make_float2(f * rc, f * rs);
#pragma unroll
            for (int g = 0; g < kGroup; g++) {
                if (g < ng) {
                    const uint32_t a = (sig[g] * (uint32_t)t + tau[g]) & mask;
                    const float2 v = __ldg(&x[a]);
                    acc[g].x = fmaf(c.x, v.x, fmaf(-c.y, v.y, acc[g].x));
                    acc[g].y = fmaf(c.x, v.y, fmaf(c.y, v.x, acc[g].y));
                }
            }
        }
#pragma unroll
        for (int g = 0; g < kGroup; g++) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                acc[g].x += __shfl_xor_sync(0xffffffffu, acc[g].x, o);
                acc[g].y += __shfl_xor_sync(0xffffffffu, acc[g].y, o);
            }
        }
        if (lane == 0) {
            const float2 Sb = bucket_factor((uint32_t)b, logB, logn);
#pragma unroll
            for (int g = 0; g < kGroup; g++) {
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
    (void)D;
}

// ---------------------------------------------------------------------------------
// 1D residue stream: thread = (residue r, row chunk).  Samples a = r + j B are read
// coalesced; for every hash the bucket of all of them is the same, b = sigma^{-1}(r - tau)
// mod B, so each thread keeps one accumulator per hash and no reduction is needed.
// Output: part[(chunk * nh + l) * B + r].
// ---------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_bin_stream_1d(const float2 *__restrict__ x, int logn,
                                                       const HashParam *hashes, int nh,
                                                       const WindowParam *win, const Job *job_dev,
                                                       int logB_static, int chunks_static,
                                                       float2 *__restrict__ part)
{
    extern __shared__ float2 rot[];   // R_u for u in [0, 2D)
    int logB = logB_static, chunks = chunks_static;
    if (job_dev) {
        if (!job_dev->active || !job_dev->stream) return;
        logB = job_dev->logB;
        nh = job_dev->nh;
        chunks = job_dev->chunks;
    }
    const int group0 = blockIdx.y * kGroup;
    if (group0 >= nh) return;
    const int ng = min(kGroup, nh - group0);
    const uint32_t n = 1u << logn, mask = n - 1, B = 1u << logB;
    const uint32_t D = n >> logB;
    const WindowParam w = win[logB];
    const bool full = (2 * (int64_t)w.h + 1) >= (int64_t)n - 1;   // every t but -n/2 inside
    for (uint32_t u = threadIdx.x; u < 2 * D; u += blockDim.x) {
        float s, c;
        sincospif(ldexpf((float)u, -(logn - logB)), &s, &c);
        rot[u] = (u & 1) ? make_float2(-c, -s) : make_float2(c, s);
    }
    __syncthreads();
    const uint32_t rows = D / (uint32_t)chunks;
    const int64_t items = (int64_t)B * chunks;
    uint32_t sinv[kGroup], c0[kGroup];
#pragma unroll
    for (int g = 0; g < kGroup; g++) {
        const HashParam hp = hashes[group0 + (g < ng ? g : 0)];
        sinv[g] = hp.sinv[0];
        c0[g] = 0u - hp.sinv[0] * hp.tau[0];
    }
    const int sh = 32 - logn;
    for (int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; it < items;
         it += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t r = (uint32_t)(it & (B - 1));
        const uint32_t ch = (uint32_t)(it >> logB);
        float2 acc[kGroup];
        float2 cen[kGroup];
#pragma unroll
        for (int g = 0; g < kGroup; g++) {
            acc[g] = make_float2(0.f, 0.f);
            cen[g] = make_float2(0.f, 0.f);
        }
        const uint32_t j0 = ch * rows;
        for (uint32_t j = j0; j < j0 + rows; j++) {
            const uint32_t a = r + (j << logB);
            const float2 v = __ldg(&x[a]);
#pragma unroll
            for (int g = 0; g < kGroup; g++) {
                if (g < ng) {
                    const uint32_t t = (sinv[g] * a + c0[g]) & mask;
                    const int ts = (int)(t << sh) >> sh;
                    if (ts == 0) {
                        cen[g] = v;
                        continue;
                    }
                    if (!full && (ts > w.h || ts < -w.h)) continue;
                    if (full && ts == -(int)(n >> 1)) continue;
                    const float tf = (float)ts;
                    const float f = fast_exp2(fmaf(-w.k2 * tf, tf, w.log2c)) * fast_rcp(tf);
                    const float2 R = rot[(uint32_t)(ts >> logB) & (2 * D - 1)];
                    const float cr = f * R.x, ci = f * R.y;
                    acc[g].x = fmaf(cr, v.x, fmaf(-ci, v.y, acc[g].x));
                    acc[g].y = fmaf(cr, v.y, fmaf(ci, v.x, acc[g].y));
                }
            }
        }
#pragma unroll
        for (int g = 0; g < kGroup; g++) {
            if (g < ng) {
                const uint32_t b = (sinv[g] * r + c0[g]) & (B - 1);
                const float2 Sb = bucket_factor(b, logB, logn);
                float2 z = cmul(Sb, acc[g]);
                z.x += w.cA_D * cen[g].x;
                z.y += w.cA_D * cen[g].y;
                part[((int64_t)ch * nh + group0 + g) * B + r] = z;
            }
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

// 2D residue stream: thread = (residue pair (r1, r2), chunk of rows j1).  Pixels
// (r1 + j1 B, r2 + j2 B) all feed bucket (b1, b2) of each hash.  Output
// part[(chunk * nh + l) * B^2 + r1 * B + r2].
__global__ void __launch_bounds__(256) k_bin_stream_2d(const float2 *__restrict__ x, int logn,
                                                       int nh, const Job *job_dev,
                                                       int logB_static, int chunks_static,
                                                       const float2 *__restrict__ taps,
                                                       float2 *__restrict__ part)
{
    int logB = logB_static, chunks = chunks_static;
    if (job_dev) {
        if (!job_dev->active) return;
        logB = job_dev->logB;
        nh = job_dev->nh;
        chunks = job_dev->chunks;
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
            float2 row[kGroup];
#pragma unroll
            for (int g = 0; g < kGroup; g++) row[g] = make_float2(0.f, 0.f);
            for (uint32_t j2 = 0; j2 < D; j2++) {
                const uint32_t a2 = r2 + (j2 << logB);
                const float2 v = __ldg(&x[(int64_t)a1 * N + a2]);
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
            if (g < ng) part[((int64_t)ch * nh + group0 + g) * B2 + (int64_t)r1 * B + r2] = acc[g];
    }
}

// 2D gather for small windows: warp per bucket (b1, b2); lanes walk the window's
// (u1, u2) pairs; taps from the per-axis tables at the permuted positions.
__global__ void k_bin_gather_2d(const float2 *__restrict__ x, int logn, const HashParam *hashes,
                                int nh, const WindowParam *win, const Job *job_dev,
                                int logB_static, const float2 *__restrict__ taps,
                                float2 *__restrict__ out)
{
    int logB = logB_static;
    if (job_dev) {
        if (!job_dev->active || job_dev->stream) return;
        logB = job_dev->logB;
        nh = job_dev->nh;
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
// Launch: job_host gives the static shape (tuning); dynamic = the job at B* written by
// the controller (every form is launched and all but the matching one exit at once).
// Partial sums go to P->d_part in residue order, [chunk][hash][bucket].
// ---------------------------------------------------------------------------------
void launch_bin(const atsfft_plan_s *P, const float2 *x, const Job *job_dev, const Job &job_host,
                bool dynamic, const HashParam *hashes, int logB_static, cudaStream_t s)
{
    const int persist = P->num_sms * kPersistCtas;
    const int groups = (job_host.nh + kGroup - 1) / kGroup;
    const Job *jd = dynamic ? job_dev : nullptr;
    if (P->ndim == 1) {
        if (dynamic || !job_host.stream) {
            const int64_t want = ((int64_t)1 << logB_static) / 8 + 1;
            dim3 grid(dynamic ? persist : (unsigned)(want < persist ? want : persist), groups);
            k_bin_gather_1d<<<grid, 256, 0, s>>>(x, P->logn, hashes, job_host.nh, P->d_win, jd,
                                                 logB_static, P->d_part);
        }
        if (dynamic || job_host.stream) {
            // rotation table: 2D entries for the smallest D the stream form can see
            int minb = dynamic ? P->b0 : logB_static;
            size_t smem = sizeof(float2) * 2 * (size_t)(P->n >> minb);
            if (smem > 64 * 1024) smem = 64 * 1024;   // stream form requires D <= 4096
            cudaFuncSetAttribute(k_bin_stream_1d, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
            dim3 grid(persist, groups);
            k_bin_stream_1d<<<grid, 256, smem, s>>>(x, P->logn, hashes, job_host.nh, P->d_win, jd,
                                                    logB_static, job_host.chunks, P->d_part);
        }
    } else {
        float2 *taps = P->d_fft_tmp;   // per-axis tap tables: nh x 2 x N (fits: nh * 2N <= nh * B^2)
        k_taps_2d<<<P->num_sms * 2, 256, 0, s>>>(P->logn, hashes, job_host.nh, P->d_win, jd,
                                                  logB_static, taps);
        if (dynamic || !job_host.stream) {
            dim3 grid(persist, job_host.nh);
            k_bin_gather_2d<<<grid, 256, 0, s>>>(x, P->logn, hashes, job_host.nh, P->d_win, jd,
                                                 logB_static, taps, P->d_part);
        }
        if (dynamic || job_host.stream) {
            dim3 grid(persist, groups);
            k_bin_stream_2d<<<grid, 256, 0, s>>>(x, P->logn, job_host.nh, jd, logB_static,
                                                 job_host.chunks, taps, P->d_part);
        }
    }
}

}  // namespace atsfft
