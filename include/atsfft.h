/*
 * atsfft.h -- C ABI of the GB300 (sm_103a) ATSFFT library.
 *
 * ATSFFT (Shi, Yang, Zhang, You, arXiv 1908.02461) is a sparse FFT that also detects
 * the sparsity k.  Each transform runs, entirely on the GPU:
 *   tuning   (Algorithm 2, Eqs. (12)-(14)): hashes at growing bucket counts B, each
 *            counting the local maxima of the bucket energies, until the count is
 *            stable; the final B is B*, its count k*;
 *   location (Algorithm 1, Section II-B): L_loc hashes at B*, the k* largest local
 *            maxima of each vote for the coordinates that hash to them; coordinates
 *            with votes >= ceil(L_loc/2) are kept;
 *   estimation (Eq. (11), Section II-B): L_est hashes at B*, per kept coordinate the
 *            componentwise median of Zhat_h(i) * omega^(tau i) / Ghat'(o(i)).
 * A hash is the random spectrum permutation of Def. 1, the flat window of Section
 * II-A-2 (box car of one bucket width convolved with a Gaussian, Eqs. (8),(9)),
 * subsampling into B buckets (Lemma 2) and a B-point DFT.
 *
 * Conventions (Section II): the DFT is unscaled, xhat[f] = sum_t x[t] exp(-2 pi i f t/n);
 * sizes are powers of two; 2D images are N x N, row-major, and 2D locations are linear
 * indices i*N + j (i = row frequency, j = column frequency).
 *
 * Memory: every `d_` pointer is device memory owned by the caller; the plan owns its
 * tables and scratch.  Calls that take a stream only enqueue work on it and never
 * synchronise, except where stated.  A plan may be used by one stream at a time
 * (one scratch set).  Errors are returned as status codes; nothing aborts or throws.
 * A CUDA error already pending on the calling thread when a call starts (left by the
 * caller's own earlier work) makes the call return ATSFFT_E_CUDA before it does anything,
 * and stays pending: the library never clears an error it did not cause.
 */
#ifndef ATSFFT_H
#define ATSFFT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct atsfft_plan_s *atsfft_plan_t;

typedef enum {
    ATSFFT_OK = 0,
    ATSFFT_E_INVALID_ARG = 1,   /* bad size, pointer or parameter                         */
    ATSFFT_E_NOMEM = 2,         /* device or host allocation failed                       */
    ATSFFT_E_CUDA = 3,          /* a CUDA call or launch failed                           */
    ATSFFT_E_NOT_CONVERGED = 4, /* tuning used all its trials; result at the last B       */
    ATSFFT_E_NOT_SPARSE = 5,    /* tuning wanted B beyond its maximum; result at the max  */
    ATSFFT_E_CAPACITY = 6       /* more outputs than `capacity`; *d_count = number needed */
} atsfft_status;

/* Parameters of Algorithm 2 and of the readings of points the paper leaves open. */
typedef struct {
    double delta1, delta2;      /* Eq. (14) ratio bands, paper: 0.02, 0.05                */
    double eps1, eps2;          /* Eq. (13)/(14) factors, paper: 0.5, 1.0 (only values
                                   accepted: they keep B a power of two)                 */
    int tune_max;               /* cap on tuning trials (default 32)                     */
    int loops_loc, loops_est;   /* location / estimation hashes (default 7, 7)           */
    double filter_alpha;        /* window transition width, fraction of half a bucket    */
    double filter_tol;          /* window Gaussian tail tolerance (default 1e-6)         */
    double thr_rel, thr_med;    /* local-maximum threshold max(thr_rel*maxE,
                                   thr_med*medianE) (default 1e-3, 20)                   */
    double tie_eta;             /* relative band inside which energies tie (1e-2)        */
    int b_min_log2, b_max_log2; /* tuning range of log2 B (per axis in 2D); 0 = default:
                                   1D [4, log2 n - 4], 2D [3, log2 N - 2]                */
    int coop_blocks_per_sm;     /* accepted in [0, 8] and without effect: the tail kernels
                                   no longer run as a cooperative grid (kept so that the
                                   struct keeps its layout)                              */
    int tune_stages;            /* 1D tuning batches: 3 (default) evaluates the trials with
                                   gather-form windows first, then the residue-stream
                                   trials but the largest, then the largest, each batch
                                   only if the controller has not stopped; 2 keeps the
                                   residue-stream trials in one batch; 1 evaluates every
                                   trial in one batch.  Same results either way         */
    int fixed_k;                /* 1: no tuning (the SFFT setting): B is the smallest power of
                                   two with B^2 >= n k (2D: B^4 >= N^2 k) for k = k_hint,
                                   which must then be > 0; k* = k_hint.  0 (default): tune */
    int est_reuse_loc;          /* 1: the estimation loops reuse the location hashes
                                   (requires loops_est <= loops_loc): half the binning and
                                   FFT work at B*.  0 (default): fresh estimation hashes  */
    int precision;              /* 0 (default): complex64 input and values, FP32 path.
                                   1: complex128 input and values (1D and 2D); locations
                                   as in the FP32 path (on the input rounded to complex64),
                                   the estimation stage in FP64 (Eq. (11) values to
                                   ~1e-12 of an FP64 evaluation).  Slow: FP64 runs at
                                   1/64 of the FP32 rate on GB300                         */
    int coop_sms;               /* accepted (>= 0) and without effect, like
                                   coop_blocks_per_sm                                    */
} atsfft_params;

/* Fills *p with the defaults listed above. */
void atsfft_default_params(atsfft_params *p);

/* Creates a plan for 1D signals of length shape[0] (ndim = 1; a power of two in
 * [2^8, 2^28]) or N x N images (ndim = 2, shape = {N, N}, N a power of two in
 * [2^5, 2^14]).  k_hint > 0 starts the tuning at the smallest power-of-two B >= 2 k_hint
 * (2D: B^2 >= 2 k_hint); 0 means k is unknown.  p = NULL takes the defaults.  seed
 * keys the SplitMix64 streams of the hash permutations (Def. 1).  Builds the window
 * tables (Section II-A-2) for every B of the tuning range on the current device and
 * synchronises it.  On error *out is NULL. */
atsfft_status atsfft_plan(atsfft_plan_t *out, int ndim, const int64_t *shape, int64_t k_hint,
                          const atsfft_params *p, uint64_t seed);

/* A new plan equal to `src` (same shape, parameters, hint and seed, so its transforms
 * give bit-identical results) with its own scratch, on the current device (which must be
 * src's).  The window, phase and twiddle tables are copied from src rather than
 * computed, so this is much cheaper than atsfft_plan; one plan per concurrent transform
 * (a batch branch, a stream) is what the scratch ownership requires.  src stays
 * independent: either may be destroyed first. */
atsfft_status atsfft_plan_clone(atsfft_plan_t src, atsfft_plan_t *out);

/* One 1D transform of d_x (n complex64, interleaved re/im floats, device).
 *   d_loc   int64[capacity]: kept coordinates (frequencies), ascending;
 *   d_val   complex64[capacity]: their estimated DFT values (Eq. (11), median);
 *   d_count int64: number of kept coordinates (may exceed capacity);
 *   d_k     int64: detected sparsity k*;
 *   d_status int32: atsfft_status of the transform (OK, NOT_CONVERGED, NOT_SPARSE,
 *           CAPACITY).  All outputs are device memory, written by the GPU on `stream`
 *           (a cudaStream_t; NULL = legacy default stream).  The return value only
 *           reports argument and launch errors. */
atsfft_status atsfft_exec(atsfft_plan_t plan, const void *d_x, int64_t *d_loc, void *d_val,
                          int64_t capacity, int64_t *d_count, int64_t *d_k, int32_t *d_status,
                          void *stream);

/* One 2D transform of the N x N row-major complex64 image d_img; locations are
 * linear indices i*N + j.  Other arguments as atsfft_exec. */
atsfft_status atsfft_exec_2d(atsfft_plan_t plan, const void *d_img, int64_t *d_loc, void *d_val,
                             int64_t capacity, int64_t *d_count, int64_t *d_k,
                             int32_t *d_status, void *stream);

/* Releases the plan's device and host memory (synchronises the device first). */
atsfft_status atsfft_destroy(atsfft_plan_t plan);

/* Static, NUL-terminated description of a status code. */
const char *atsfft_status_string(atsfft_status s);

/* ---- inspection (tests and diagnostics) ---------------------------------------- */

/* One hash of the plan's signal shape at bucket count B (per axis in 2D), for
 * (phase, index) = (0 tuning, log2 B), (1 location, l) or (2 estimation, l): writes the
 * bucket spectrum Zhat (complex64; B values, or B*B row-major in 2D) to d_zhat on
 * `stream`.  B must lie in the plan's tuning range.  FP32 plans (precision 0) only:
 * ATSFFT_E_INVALID_ARG otherwise. */
atsfft_status atsfft_hash_spectrum(atsfft_plan_t plan, const void *d_x, int64_t B, int phase,
                                   int index, void *d_zhat, void *stream);

/* Copies the plan's window response Ghat'(o) at the half-integer bucket offsets
 * o = j - D/2 + 1/2, j in [0, D), D = n/B (per axis in 2D), to the host array h_resp
 * (double[D]).  Synchronous. */
atsfft_status atsfft_window_response(atsfft_plan_t plan, int64_t B, double *h_resp);

/* After an exec has completed on its stream: the tuning trajectory of that exec
 * (B and local-maximum count of each trial, in order) into host arrays of length
 * max_trials, and the number of trials.  Synchronises `stream`. */
atsfft_status atsfft_last_trace(atsfft_plan_t plan, int64_t *h_B, int64_t *h_k, int max_trials,
                                int *h_ntrials, void *stream);

/* After an exec: B* (per axis in 2D) and k* of the last transform of this plan
 * (synchronises `stream`). */
atsfft_status atsfft_last_result(atsfft_plan_t plan, int64_t *h_B, int64_t *h_k, void *stream);

/* Turns per-phase CUDA events on (1) or off (0) for later execs of this plan.  The
 * thirteen phases of one exec, in order: 0 binning of the first tuning stage (1D: the
 * trials with gather-form windows; 2D: every trial), 1 their bucket FFTs, 2 their
 * statistics and the controller, 3-5 the same for the second tuning stage (1D: the
 * residue-stream trials but the largest), 6-8 for the third (1D: the largest trial);
 * a later stage runs only when the controller did not stop within the earlier ones,
 * 9 binning of the location/estimation hashes in the residue-stream form (1D; 2D: tap
 * tables + stream form), 10 the same in the gather form, 11 their bucket FFTs, 12
 * location statistics, top-num cutoff, votes, ordering, estimation and median.  A form,
 * shape or stage that does not apply exits at once (or is not launched), so its phase
 * measures only an empty launch or nothing. */
atsfft_status atsfft_set_profiling(atsfft_plan_t plan, int on);

/* After an exec: per-phase device times in ms (h_ms[max_phases], read only if profiling
 * was on for that exec; synchronises `stream`), the number of phases, and the number of
 * kernel launches that exec enqueued (h_launches may be NULL). */
atsfft_status atsfft_phase_times(atsfft_plan_t plan, float *h_ms, int max_phases, int *h_nphases,
                                 int64_t *h_launches, void *stream);

/* Diagnostics after an exec: device time stamps (ns, %globaltimer) taken at the start
 * of every tail kernel, once the kernel before it has completed (the tuning statistics
 * of each stage, the location maxima with their cutoffs, the votes and the outputs),
 * and when a tuning stage's controller has walked, in the order they happened (at most
 * 32).  Synchronises `stream`. */
atsfft_status atsfft_tail_stamps(atsfft_plan_t plan, uint64_t *h_ns, int max_stamps,
                                 int *h_nstamps, void *stream);

/* The measured rate of the GPU's special-function unit on the two operations every
 * window tap of the residue-stream binning costs (an exp2 and a reciprocal: the
 * Gaussian envelope and the box car's 1/t of Section II-A-2): a kernel of independent
 * ex2.approx / rcp.approx chains on every SM (iters iterations of 8 chains per thread,
 * 2048 threads per SM, in [1, 2^24]), timed with CUDA events on `stream`.  Writes the
 * operations per second to *h_ops_per_s (half of it is the sample-hash pairs per
 * second).  Synchronises `stream`.  A diagnostic: the paper has no counterpart. */
atsfft_status atsfft_mufu_probe(int64_t iters, double *h_ops_per_s, void *stream);

/* ---- gradients at a fixed recovered support (1D) ---------------------------------- */

/* atsfft_exec (or atsfft_exec_2d) that also writes, for each output position p <
 * capacity, the estimation-hash indices the componentwise median selected (Section II-B,
 * Eq. (11)): d_medsel[2p] for the real part, d_medsel[2p + 1] for the imaginary part
 * (uint8, 0 .. loops_est - 1).  Together with the locations and B* (the last entry of
 * atsfft_last_trace) they fix the real-linear map atsfft_estimate_apply evaluates and
 * atsfft_estimate_adjoint transposes. */
atsfft_status atsfft_exec_sel(atsfft_plan_t plan, const void *d_x, int64_t *d_loc, void *d_val,
                              uint8_t *d_medsel, int64_t capacity, int64_t *d_count, int64_t *d_k,
                              int32_t *d_status, void *stream);

/* Eq. (11) at a fixed support as a function of the input, for a 1D plan: d_out[p] =
 * (Re v_{l_r}(p), Im v_{l_i}(p)) where v_l(p) is the estimate of coordinate d_loc[p]
 * from estimation hash l of the plan at B buckets applied to d_u (n complex64), and
 * (l_r, l_i) = d_medsel[2p], d_medsel[2p + 1].  For d_u = the transformed signal this
 * reproduces the transform's values.  Uses the plan's scratch (not reentrant with its
 * execs); B must lie in the plan's tuning range.  FP32 plans (precision 0) only:
 * ATSFFT_E_INVALID_ARG otherwise. */
atsfft_status atsfft_estimate_apply(atsfft_plan_t plan, int64_t B, const void *d_u,
                                    const int64_t *d_loc, const uint8_t *d_medsel, int64_t count,
                                    void *d_out, void *stream);

/* The adjoint of atsfft_estimate_apply with respect to the real inner products of the
 * input and output: given d_gval[p] = dL/dRe y_p + i dL/dIm y_p for count outputs, writes
 * d_gx[a] = dL/dRe u_a + i dL/dIm u_a for every sample a < n (complex64, overwritten).
 * This is the permuted, conjugate-phase scatter of the gradient back through Eq. (11),
 * the bucket DFT, the binning and the window.  Same arguments and scratch rules. */
atsfft_status atsfft_estimate_adjoint(atsfft_plan_t plan, int64_t B, const int64_t *d_loc,
                                      const uint8_t *d_medsel, int64_t count, const void *d_gval,
                                      void *d_gx, void *stream);

/* ---- batched execution in one CUDA graph ----------------------------------------- */

typedef struct atsfft_batch_s *atsfft_batch_t;

/* Records the transforms of n distinct plans -- plan i on input d_x[i] with outputs
 * d_loc[i], d_val[i], capacity[i], d_count[i], d_k[i], d_status[i], exactly as
 * atsfft_exec (1D plans) or atsfft_exec_2d (2D plans) take them -- into one CUDA graph
 * whose n branches run concurrently, and instantiates it on the current device.  Nothing
 * runs yet.  The pointers are fixed in the graph: the buffers must stay allocated and
 * are re-read on every launch.  Profiling must be off on every plan.  A plan may appear
 * at most once (each branch uses its plan's scratch).  On error *out is NULL. */
atsfft_status atsfft_batch_create(int n, const atsfft_plan_t *plans, const void *const *d_x,
                                  int64_t *const *d_loc, void *const *d_val,
                                  const int64_t *capacity, int64_t *const *d_count,
                                  int64_t *const *d_k, int32_t *const *d_status,
                                  atsfft_batch_t *out);

/* atsfft_batch_create whose graph also moves the data between pinned host memory and
 * the device: input i is copied from h_x[i] (ncoord complex values of the plan's
 * precision) to d_x[i] on one copy chain in index order, and transform i starts as soon
 * as its own input has landed, so every transform but the last overlaps the later
 * copies; after transform i its outputs go back to h_loc[i] and h_val[i] (capacity[i]
 * entries each) and its count, k* and status to *h_count[i], *h_k[i], *h_status[i].
 * Any of the h_ arrays, or any of their entries, may be NULL (no copy).  The host
 * buffers must be pinned (cudaHostAlloc / cudaHostRegister) and stay valid while the
 * batch exists; the caller orders the inputs (e.g. the longest transform first). */
atsfft_status atsfft_batch_create_io(int n, const atsfft_plan_t *plans, const void *const *h_x,
                                     const void *const *d_x, int64_t *const *d_loc,
                                     void *const *d_val, const int64_t *capacity,
                                     int64_t *const *d_count, int64_t *const *d_k,
                                     int32_t *const *d_status, int64_t *const *h_loc,
                                     void *const *h_val, int64_t *const *h_count,
                                     int64_t *const *h_k, int32_t *const *h_status,
                                     atsfft_batch_t *out);

/* Runs the n transforms of the batch on `stream` (one graph launch; asynchronous).  The
 * outputs of each branch are those of the corresponding plain exec. */
atsfft_status atsfft_batch_launch(atsfft_batch_t batch, void *stream);

/* Kernel launches one batch launch makes (the sum over its branches). */
atsfft_status atsfft_batch_kernels(atsfft_batch_t batch, int64_t *h_kernels);

/* Frees the graph.  The plans stay valid. */
atsfft_status atsfft_batch_destroy(atsfft_batch_t batch);

/* ---- allocation-free variant ---------------------------------------------------- */

/* The bucket spectrum of one hash of a 1D signal -- the same values atsfft_hash_spectrum
 * gives for a plan of length n with the default parameters and this seed -- computed
 * without a plan and without allocating any memory.  The paper has no counterpart: this
 * call exists for callers that cannot allocate device memory when they need the result
 * (cudaMalloc can synchronise the whole device, which a host callback or a latency-
 * critical serving loop must not do; a process whose device memory belongs to another
 * allocator with a fixed budget may not be allowed extra cudaMalloc calls).
 *
 * Scratch: a fixed 12 MiB array inside the library, held by every GPU that loads the
 * library until the process exits.  Sizes are limited so that everything fits: n a power
 * of two in [2^8, 2^22], B a power of two in [16, n/16]; anything else returns
 * ATSFFT_E_INVALID_ARG.  d_x: n complex64 on the current device; d_zhat: B complex64
 * (bucket order) written on `stream`.  The first call on a device also sets that device
 * up (looks up the array's device address and fills a twiddle table); make that first
 * call before any stream capture.  Each call synchronises `stream` once (to read back
 * the window normalisation).  All calls share the one array and every call writes all
 * of it that it reads, so nothing needs clearing between calls; calls that overlap on
 * the GPU (other streams, other threads) race on it.  The device address found by the
 * first call is kept for the life of the process: a cudaDeviceReset between calls is
 * not supported. */
atsfft_status atsfft_hash_spectrum_noalloc(const void *d_x, int64_t n, int64_t B, uint64_t seed,
                                           int phase, int index, void *d_zhat, void *stream);

#ifdef __cplusplus
}
#endif
#endif
