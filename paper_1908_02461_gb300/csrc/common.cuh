// common.cuh -- internal definitions shared by the ATSFFT CUDA translation units.
//
// Data layout convention ("residue order").  For a hash (sigma, tau) at B buckets the
// binning kernels store the bucket sums not at bucket index b but at the residue
// r = (sigma b + tau) mod B of the samples that feed it (a = r mod B for every sample
// a of bucket b).  The bucket FFT transforms that array as it is, giving P.  By the
// permutation property (Lemma 1 applied to the B-point DFT) the bucket spectrum is
//     Zhat[c] = P[sigma' c mod B] * exp(2 pi i c sigma' tau / B),  sigma' = sigma^{-1} mod B,
// per axis in 2D.  Energies |Zhat[c]|^2 = |P[sigma' c]|^2 need no phase; the estimator
// applies the phase together with omega^{tau i} in one FP64 angle.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "atsfft.h"

namespace atsfft {

constexpr int kMaxLoops = 31;        // location / estimation hashes each
constexpr int kMaxLogB = 26;         // log2 B range table size
constexpr int kSmallFFT = 4096;      // largest FFT done in one CTA
constexpr int kTwEntries = 2 * kSmallFFT;   // coarse exp(-2 pi i j / 4096), fine exp(-2 pi i j / 2^24)
constexpr int kMaxTrialsTrace = 64;
constexpr int kHistBins = 4096;      // radix-select histogram bins (12-bit digits)
constexpr int kKeptCap = 8192;       // kept coordinates ordered by rank (beyond: bitmap compaction)
constexpr int kChunkWords = 1024;    // coordinate-bitmap words per compaction chunk
constexpr int kAdjRotMax = 8192;     // adjoint: R_u table entries kept in shared memory
constexpr int kPersistCtas = 4;      // persistent CTAs per SM
constexpr int kPhases = 13;          // profiled phases of one exec (see atsfft.h)

// Permutation of one hash (Def. 1), per axis.
struct HashParam {
    uint32_t sigma[2];   // odd, < n
    uint32_t tau[2];     // < n
    uint32_t sinv[2];    // sigma^{-1} mod n
};

// Window of one bucket count B (Section II-A-2): taps t in [-h, h],
// G_t = A exp(-t^2/(2 s^2)) sin(pi t/B)/(pi t/n) applied with exp(i pi t/n).
struct WindowParam {
    int32_t h;
    float k2;            // log2(e) / (2 s^2)
    float log2c;         // log2(A n / pi): scale of the per-sample factor
    float cA_D;          // A * D (the centre tap G_0)
    double s;
    double A;
};

// A set of equally shaped hashes processed together (the tuning hash of one B, or the
// location + estimation hashes at B*).  Written by the host for tuning, by the
// controller kernel for B*.
struct Job {
    int32_t logB;        // per axis
    int32_t nh;          // hashes in this job
    int32_t chunks;      // residue-stream row chunks (partials summed by the FFT)
    int32_t stream;      // 1: residue-stream binning, 0: gather form (lanes per bucket)
    int32_t active;      // 0: nothing to do (skipped by every kernel)
    int32_t pad[3];
};

// Offsets of each B's table in the plan's concatenated Ghat' tables (by log2 B).
struct RespOffsets {
    int64_t off[kMaxLogB];
};

// One hash's spectrum for the energy / threshold / local-maximum kernels.
struct StatJob {
    const float2 *spec;    // P (residue-order FFT output), B or B^2 values
    float *energy;         // |P|^2, same layout
    const HashParam *hash;
    int32_t logB;          // per axis
    int32_t slot;          // HashStats slot
    int32_t list;          // >= 0: append local maxima (bucket indices c) to that list
    int32_t active;
};

// Per-hash statistics of the bucket energies (Section III-A local maxima).
struct HashStats {
    uint32_t max_bits;     // bits of max E (E >= 0: bit order = value order)
    uint32_t above;        // #{E > X}, X just below thr_rel/thr_med * max
    uint32_t need_median;  // 1 if the median can exceed X (then it is computed exactly)
    uint32_t prefix;       // radix-select: digits fixed so far
    uint32_t rank;         // radix-select: rank within the prefix class
    uint32_t med_bits;
    float T;               // threshold
    uint32_t nmax;         // local maxima
    uint32_t nsel;         // selected by the top-num cutoff
    uint32_t v_bits;       // top-num pivot: bits of the num-th largest maximum energy
    uint32_t pad[6];
};

// Diagnostic time stamps of the tail kernels (tail.cu).
struct TailStamps {
    unsigned nstamp;
    unsigned pad[3];
    unsigned long long stamp[32];   // %globaltimer at tail kernel starts and phase ends
};

// Device-resident state of one exec.
struct ExecState {
    TailStamps bar;
    // completion counters of the tail kernels (a block that finishes a task counts it;
    // the block that counts the last task of a hash, or of the whole launch, goes on with
    // the step that needs all of them): per statistics slot, and per launch
    uint32_t done[kMaxLogB + kMaxLoops];
    uint32_t done_all[8];
    int32_t b_star;        // log2 B* (per axis)
    int32_t status;
    int64_t k_star;
    int64_t count;         // kept coordinates
    int32_t ntrials;
    int32_t empty;         // 1: nothing to locate
    int32_t tune_done;     // 1: the controller stopped within the small-B trials (1D)
    int32_t pad0;
    int64_t trial_B[kMaxTrialsTrace];
    int64_t trial_k[kMaxTrialsTrace];
    Job job;               // location + estimation job at B*
};

}  // namespace atsfft

struct atsfft_plan_s {
    int ndim;
    int logn;              // log2 n (1D) or log2 N (2D, per axis)
    int64_t n;             // n or N
    int64_t ncoord;        // n or N^2
    atsfft_params p;
    uint64_t seed;
    int b_lo, b_hi, b0;
    int64_t k_hint;
    int b_fixed;           // fixed-k mode: log2 B (per axis)
    int est_base;          // index of the first estimation hash in h_le / d_le
    int nh_le;             // location + estimation hashes binned at B* (distinct ones)
    // FP64 path (precision 1): FP32 copy of the input, FP64 estimation spectra (two
    // Stockham buffers, [L_est][B*] or [L_est][B* x B*]) and their twiddles
    float2 *d_x32;
    double2 *d_f64a, *d_f64b, *d_tw64;
    double2 *d_wtab64;     // 2D: the modulated window taps of B* in FP64 (2h + 1 <= N - 1)
    int L_loc, L_est;
    int device;
    int num_sms;

    atsfft::HashParam h_tune[atsfft::kMaxLogB];   // tuning hash of each log2 B
    atsfft::HashParam h_le[2 * atsfft::kMaxLoops]; // location then estimation hashes
    atsfft::WindowParam h_win[atsfft::kMaxLogB];
    int64_t resp_off[atsfft::kMaxLogB];
    atsfft::Job h_tjob[atsfft::kMaxLogB];
    int64_t tpart_off[atsfft::kMaxLogB];          // tuning partial sums of each B in d_part
    int tchunks[atsfft::kMaxLogB];                // partial blocks the FFT adds up per B
    // tuning stages s = 1..3 take the trials (tune_hi[s-1], tune_hi[s]] (tune_hi[0] = b0 - 1;
    // an empty stage repeats the previous bound); the 1D residue-stream trials of stage s
    // share one pass of modulus 2^tstream_logR[s] (-1: none) and tstream_chunks[s] chunks
    int tune_hi[4];
    int tstream_logR[4], tstream_chunks[4];

    atsfft::HashParam *d_tune, *d_le;
    atsfft::WindowParam *d_win;
    double *d_resp;        // Ghat' tables for every B of the range, concatenated
    float *d_rgain;        // 1 / Ghat', same layout, rounded to FP32
    float2 *d_phase;       // exp(2 pi i m / n): [2^phase_s] low part, [n >> phase_s] high part
    int phase_s;
    float2 *d_tw;          // [0, 4096): exp(-2 pi i j / 4096); [4096, 8192): exp(-2 pi i j / 2^24)
    // 2D: per-axis tap tables built at plan time (they depend on the hashes and windows
    // only): the tuning hash of B = 2^b at d_taps_tune + b * 2N, the nh_le location and
    // estimation hashes at B = 2^b at d_taps_le + b * nh_le * 2N (layout as k_taps_2d)
    float2 *d_taps_tune, *d_taps_le;

    float2 *d_part;        // binning partial sums (residue order)
    size_t part_elems;
    float2 *d_tz;          // tuning spectra P, all B concatenated (offsets tz_off)
    int64_t tz_off[atsfft::kMaxLogB];
    float2 *d_z;           // location + estimation spectra at B*
    float2 *d_fft_tmp;     // four-step intermediate
    float *d_energy;       // energies (tuning region then location region)
    int64_t e_loc_off;
    atsfft::HashStats *d_stats;   // [kMaxLogB tuning slots][L_loc location slots]
    int32_t *d_lmax;              // local-maximum lists [L_loc][lmax_cap]
    float *d_lmax_e;              // their energies, same layout
    int32_t *d_sel;               // selected buckets    [L_loc][lmax_cap]
    int64_t lmax_cap;
    uint32_t *d_bucketbits;       // [L_loc][bucket_words] selected location buckets
    int64_t bucket_words;
    uint32_t *d_kept;             // kept coordinates of the last transform, unordered
    int64_t kept_cap;
    uint32_t *d_coordbits;        // one bit per coordinate, zero between transforms
    int64_t coord_words;
    uint32_t *d_blk;              // kept coordinates per chunk of kChunkWords coordinate words
    int64_t nchunks;
    atsfft::ExecState *d_state;
    atsfft::Job *d_tjob;
    atsfft::StatJob *d_tstat;     // tuning stat jobs (built at plan time)
    atsfft::StatJob *d_lstat;     // location stat jobs (written by the controller)
    int ntstat;

    // 1 while an exec is being enqueued: its kernels after the reset are launched with
    // programmatic stream serialization (each waits for its predecessor at its top)
    mutable int pdl;
    // profiling: events at phase boundaries (when enabled) and a launch counter
    int prof;
    cudaEvent_t ev[atsfft::kPhases + 1];
    mutable int64_t launches;     // kernel launches enqueued by the last exec
};

namespace atsfft {

atsfft_status cuda_status(cudaError_t e);

// True when a CUDA error is already pending on the calling thread as an entry point
// starts (the caller's own earlier work).  Entry points then return ATSFFT_E_CUDA before
// doing anything and leave the error pending, so the library never consumes an error it
// did not cause; the errors of its own calls are read (and cleared) after its launches.
inline bool caller_error_pending() { return cudaPeekAtLastError() != cudaSuccess; }

inline void prof_mark(const atsfft_plan_s *P, int i, cudaStream_t s)
{
    if (P->prof) cudaEventRecord(P->ev[i], s);
}
inline void count_launch(const atsfft_plan_s *P, int k = 1) { P->launches += k; }

// Programmatic dependent launch inside an exec.  Every kernel of the exec chain starts
// with chain_wait(): it touches no memory before the kernel ahead of it in the stream has
// completed (exactly the order of a plain launch), but its blocks can be scheduled while
// that kernel finishes; chain_next() lets the next kernel's blocks be scheduled.  Both
// return at once in a kernel launched without the dependency.
__device__ __forceinline__ void chain_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void chain_next()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(const atsfft_plan_s *P, void (*kernel)(KArgs...), dim3 grid, dim3 block,
                            size_t smem, cudaStream_t s, Args &&...args)
{
    cudaLaunchConfig_t cfg;
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = P->pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<Args &&>(args)...);
}

inline int stats_slot_tune(int logB) { return logB; }
inline int stats_slot_loc(int l) { return kMaxLogB + l; }

// plan.cu
uint64_t splitmix64_next(uint64_t *state);
void hash_params_for(uint64_t seed, int phase, int index, int64_t n, int ndim, HashParam *out);
uint32_t inv_mod_pow2(uint32_t sigma, int64_t n);
WindowParam window_shape(int64_t n, int logB, double alpha, double tol);
Job make_job(const atsfft_plan_s *P, int logB, int nh);

// bin.cu
// Binning of tuning stage 1 (every trial in 2D; the small-window trials in 1D), 2 (1D: the
// residue-stream trials but the largest) or 3 (1D: the largest trial); stages 2 and 3 are
// skipped on the device when an earlier stage settled the controller.
void launch_tuning(const atsfft_plan_s *P, const float2 *x, int stage, cudaStream_t s);
void launch_le_bin(const atsfft_plan_s *P, const float2 *x, const Job *job_dev, cudaStream_t s);
void launch_single_hash(const atsfft_plan_s *P, const float2 *x, int b, const HashParam &hp,
                        const HashParam *hp_dev, float2 *out, cudaStream_t s);
int launch_est_bin(const atsfft_plan_s *P, const float2 *x, int b, cudaStream_t s);
__global__ void k_taps_2d(int logn, const HashParam *hashes, int nh, const WindowParam *win,
                          const Job *job_dev, int logB_static, float2 *taps);
void launch_bin_2d(const atsfft_plan_s *P, const float2 *x, const Job *job_dev, const Job &job_host,
                   bool dynamic, const HashParam *hashes, int logB_static, float2 *part,
                   cudaStream_t s, const float2 *pre_taps = nullptr, int64_t pre_stride = 0);

// fft.cu
// Bucket FFTs.  energy != nullptr: the final pass also writes |Zhat|^2 (same layout as
// the spectra) and the per-hash maximum into the HashStats slot of the hash (dynamic
// job: the first n_energy hashes, slots kMaxLogB + h; batch: slot logB).
void launch_bucket_fft_dynamic(const atsfft_plan_s *P, const Job *job, const float2 *part,
                               float2 *out, float *energy, int n_energy, cudaStream_t s);
void launch_bucket_fft_batch(const atsfft_plan_s *P, int njobs, const int *logB, const int *chunks,
                             const int64_t *in_off, const int64_t *out_off, const float2 *part,
                             float2 *out, float *energy, const int *skip, cudaStream_t s);

// tail.cu
void launch_tune_tail(const atsfft_plan_s *P, int stage, cudaStream_t s);
void launch_fixed_setup(const atsfft_plan_s *P, cudaStream_t s);   // fixed-k mode

// fp64.cu (precision 1)
void launch_to_f32(const atsfft_plan_s *P, const void *d_x, cudaStream_t s);
void launch_estimate_fp64(const atsfft_plan_s *P, const void *d_x, const int64_t *d_loc,
                          void *d_val, int64_t capacity, cudaStream_t s);
void launch_loc_tail(const atsfft_plan_s *P, int64_t *d_loc, float2 *d_val, uint8_t *d_msel,
                     int64_t capacity, int64_t *d_count, int64_t *d_k, int32_t *d_status,
                     cudaStream_t s);

// inspect.cu
void launch_reset(const atsfft_plan_s *P, cudaStream_t s);
void launch_unpermute(const atsfft_plan_s *P, const float2 *spec, const HashParam *hash_dev,
                      int logB, float2 *out, cudaStream_t s);

}  // namespace atsfft
