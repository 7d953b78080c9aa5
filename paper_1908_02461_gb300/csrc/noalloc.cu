// noalloc.cu -- atsfft_hash_spectrum_noalloc: the bucket spectrum of one hash without a
// plan and without allocating any memory.
//
// Some callers cannot allocate device memory when they need this result: cudaMalloc can
// synchronise the whole device, which a host callback or a latency-critical serving loop
// must not do, and a process whose device memory is handed out by another allocator (a
// framework's caching allocator with a fixed budget) may not be allowed extra cudaMalloc
// calls at all.  This entry point therefore takes its scratch from one fixed array that
// lives in the library image: every GPU that loads the library holds kNoAllocBytes of it
// until the process exits.  The host code below never dereferences the array's name (on
// the host it only stands for the symbol); it obtains the device address with
// cudaGetSymbolAddress once per device, with that device current.
#include <mutex>
#include <string.h>

#include "common.cuh"

namespace atsfft {

// 12 MiB: bucket partials, four-step intermediate and spectrum (3 x 2^18 complex64),
// FFT twiddles, the window-normalisation partial sums and table (FP64), and the
// two-level table of exp(2 pi i m / n).
constexpr size_t kNoAllocBytes = (size_t)12 << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kNoAllocMaxLogN = 22;
constexpr int kMaxDevices = 64;

struct NoAllocDevice {
    bool ready;
    unsigned char *base;   // device address of g_noalloc_scratch on this device
};

static NoAllocDevice g_dev[kMaxDevices];
static std::mutex g_dev_mutex;

// Byte offsets inside the scratch array (all 256-aligned).
constexpr size_t kElems18 = (size_t)1 << 18;
constexpr size_t kOffPart = 0;
constexpr size_t kOffTmp = kOffPart + kElems18 * sizeof(float2);
constexpr size_t kOffZ = kOffTmp + kElems18 * sizeof(float2);
constexpr size_t kOffTw = kOffZ + kElems18 * sizeof(float2);
constexpr size_t kOffWin = kOffTw + (size_t)kTwEntries * sizeof(float2);
constexpr size_t kOffS0 = kOffWin + 4096;                         // WindowParam table
constexpr size_t kOffResp = kOffS0 + 256;
constexpr size_t kOffPhase = kOffResp + kElems18 * sizeof(double);   // exp(2 pi i m / n) table
constexpr size_t kPhaseEntries = (size_t)2 << ((kNoAllocMaxLogN + 1) / 2);
constexpr size_t kOffPartial = kOffPhase + kPhaseEntries * sizeof(float2);
constexpr size_t kPartialDoubles = (kNoAllocBytes - kOffPartial) / sizeof(double);
static_assert(kOffPartial < kNoAllocBytes, "no-alloc scratch layout overflows");
static_assert(sizeof(WindowParam) * kMaxLogB <= 4096, "window table slot too small");

// Stores this call's window parameters in the scratch's window table (passed by value,
// so nothing on the host stack has to outlive the call).
__global__ void k_noalloc_store_window(WindowParam *slot, WindowParam w) { *slot = w; }

// Bucket order: Zhat[c] = P[sigma' c] exp(2 pi i c sigma' tau / B), hash passed by value.
__global__ void k_noalloc_unpermute(const float2 *spec, HashParam hp, int logB, float2 *out)
{
    const uint64_t B = 1ull << logB, Bm = B - 1;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < (int64_t)B;
         c += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t idx = ((hp.sinv[0] & Bm) * (uint64_t)c) & Bm;
        const uint64_t k = (idx * (hp.tau[0] & Bm)) & Bm;
        double sn, cs;
        sincospi(2.0 * (double)k / (double)B, &sn, &cs);
        const float2 v = spec[idx];
        out[c] = make_float2((float)(v.x * cs - v.y * sn), (float)(v.x * sn + v.y * cs));
    }
}

// plan.cu's plan-time kernels: window normalisation, FFT twiddles
__global__ void k_twiddles(float2 *tw);
__global__ void k_window_partial(int64_t n, int logB, double s, int h, double *partial, int nchunks);
__global__ void k_window_finish(int64_t D, const double *partial, int nchunks, double *resp,
                                double *S0_out);
__global__ void k_phase_table(int logn, int s_bits, float2 *tab);

// Once per device, with it current: the scratch's device address and the twiddles.
// The result is kept for the life of the process, so a cudaDeviceReset (which
// reinitialises the array) is not supported between calls.
static atsfft_status noalloc_setup(int dev, cudaStream_t s, unsigned char **base)
{
    std::lock_guard<std::mutex> lock(g_dev_mutex);
    NoAllocDevice &d = g_dev[dev];
    if (!d.ready) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_status(e);
        d.base = (unsigned char *)ptr;
        k_twiddles<<<kTwEntries / 256, 256, 0, s>>>((float2 *)(d.base + kOffTw));
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_status(e);
        d.ready = true;
    }
    *base = d.base;
    return ATSFFT_OK;
}

}  // namespace atsfft

using namespace atsfft;

extern "C" atsfft_status atsfft_hash_spectrum_noalloc(const void *d_x, int64_t n, int64_t B,
                                                      uint64_t seed, int phase, int index,
                                                      void *d_zhat, void *stream)
{
    if (!d_x || !d_zhat || n <= 0 || (n & (n - 1)) || B <= 0 || (B & (B - 1)) || phase < 0 ||
        phase > 2 || index < 0)
        return ATSFFT_E_INVALID_ARG;
    int logn = 0, b = 0;
    while (((int64_t)1 << logn) < n) logn++;
    while (((int64_t)1 << b) < B) b++;
    if (logn < 8 || logn > kNoAllocMaxLogN || b < 4 || b > logn - 4) return ATSFFT_E_INVALID_ARG;
    if (caller_error_pending()) return ATSFFT_E_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e);
    if (dev < 0 || dev >= kMaxDevices) return ATSFFT_E_INVALID_ARG;
    unsigned char *base = nullptr;
    atsfft_status st = noalloc_setup(dev, s, &base);
    if (st != ATSFFT_OK) return st;

    // a plan view on the host stack whose scratch pointers lie in the fixed array
    atsfft_plan_s P;
    memset(&P, 0, sizeof(P));
    P.ndim = 1;
    P.logn = logn;
    P.n = n;
    P.ncoord = n;
    atsfft_default_params(&P.p);
    P.seed = seed;
    P.b_lo = P.b0 = 4;
    P.b_hi = logn - 4;
    P.device = dev;
    cudaDeviceGetAttribute(&P.num_sms, cudaDevAttrMultiProcessorCount, dev);
    P.d_part = (float2 *)(base + kOffPart);
    P.d_fft_tmp = (float2 *)(base + kOffTmp);
    P.d_z = (float2 *)(base + kOffZ);
    P.d_tw = (float2 *)(base + kOffTw);
    P.d_win = (WindowParam *)(base + kOffWin);
    P.d_phase = (float2 *)(base + kOffPhase);
    P.phase_s = (logn + 1) / 2;
    P.part_elems = kElems18;

    // window of this B (Section II-A-2): shape on the host, normalisation sum on the device
    WindowParam w = window_shape(n, b, P.p.filter_alpha, P.p.filter_tol);
    const int64_t D = n >> b;
    const int nch = (int)((w.h + 8191) / 8192);
    if ((size_t)(D + 1) * (size_t)nch > kPartialDoubles || (size_t)D > kElems18)
        return ATSFFT_E_INVALID_ARG;
    double *partial = (double *)(base + kOffPartial);
    double *resp = (double *)(base + kOffResp);
    double *S0_dev = (double *)(base + kOffS0);
    dim3 grid((unsigned)((D + 1 + 127) / 128), (unsigned)nch);
    k_phase_table<<<P.num_sms, 256, 0, s>>>(logn, P.phase_s, P.d_phase);
    k_window_partial<<<grid, 128, 0, s>>>(n, b, w.s, w.h, partial, nch);
    k_window_finish<<<1, 256, 0, s>>>(D, partial, nch, resp, S0_dev);
    double S0 = 0.0;
    e = cudaMemcpyAsync(&S0, S0_dev, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_status(e);
    w.A = (double)n / S0;
    w.log2c = (float)log2(w.A * (double)n / M_PI);
    w.cA_D = (float)(w.A * (double)D);
    P.h_win[b] = w;
    P.h_tjob[b] = make_job(&P, b, 1);
    if ((size_t)P.h_tjob[b].chunks * (size_t)B > kElems18) return ATSFFT_E_INVALID_ARG;
    // the device copy of the window, as a plan's table holds it (P.d_win[b])
    k_noalloc_store_window<<<1, 1, 0, s>>>(P.d_win + b, w);

    HashParam hp;
    hash_params_for(seed, phase, index, n, 1, &hp);
    launch_single_hash(&P, (const float2 *)d_x, b, hp, nullptr, P.d_z, s);
    k_noalloc_unpermute<<<P.num_sms * 2, 256, 0, s>>>(P.d_z, hp, b, (float2 *)d_zhat);
    return cuda_status(cudaGetLastError());
}
