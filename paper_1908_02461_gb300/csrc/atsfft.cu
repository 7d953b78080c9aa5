// atsfft.cu -- C ABI entry points: one transform = tuning, location, estimation, all
// enqueued on the caller's stream with no host synchronisation.
//
//  tuning   : the hash of every B in the plan's range is evaluated (bin, bucket FFT,
//             energies, threshold, local-maximum count); the controller then walks
//             Eqs. (12)/(14) over those counts on the device and fixes B*, k*.  Because the
//             stop reading visits every B at most once, evaluating them up front gives
//             exactly the sequential trajectory while replacing a chain of dependent
//             trials by a batch.  1D runs two batches: the small-window trials, then --
//             only if the walk has not stopped among them (a device flag every kernel of
//             the second batch reads) -- the residue-stream trials.
//  location : the L_loc + L_est hashes at B* are binned in one pass over the signal,
//             transformed, and the location hashes' maxima are cut to k* and vote.
//  estimate : kept coordinates in ascending order, Eq. (11), median.
// Kernels that depend on B* read it from device memory; every shape they could need is
// launched and the ones that do not match exit at once.
#include <new>
#include <string.h>
#include <vector>

#include "common.cuh"

using namespace atsfft;

static atsfft_status exec_common(atsfft_plan_t P, int ndim, const void *d_x, int64_t *d_loc,
                                 void *d_val, int64_t capacity, int64_t *d_count, int64_t *d_k,
                                 int32_t *d_status, void *stream, uint8_t *d_msel = nullptr)
{
    if (!P || P->ndim != ndim || !d_x || capacity < 0 || (capacity > 0 && (!d_loc || !d_val)) ||
        !d_count || !d_k || !d_status)
        return ATSFFT_E_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const float2 *x = (const float2 *)d_x;
    if (caller_error_pending()) return ATSFFT_E_CUDA;
    P->launches = 0;
    const bool fp64 = P->p.precision == 1;
    if (fp64) {
        if (d_msel) return ATSFFT_E_INVALID_ARG;   // selections belong to the FP32 estimates
        launch_to_f32(P, d_x, s);
        x = P->d_x32;
    }
    launch_reset(P, s);
    P->pdl = 1;   // the kernels after the reset: programmatic dependent launches
    prof_mark(P, 0, s);
    if (P->p.fixed_k) {
        launch_fixed_setup(P, s);   // B* and k* from the plan: the tuning phases are empty
        for (int i = 1; i <= 9; i++) prof_mark(P, i, s);
    } else {
        for (int stage = 1; stage <= 3; stage++) {
            launch_tuning(P, x, stage, s);   // marks 1 + 3 (stage - 1) after its binning
            prof_mark(P, 3 * stage - 1, s);
            launch_tune_tail(P, stage, s);
            prof_mark(P, 3 * stage, s);
        }
    }
    const Job *jd = &P->d_state->job;
    launch_le_bin(P, x, jd, s);   // marks phase 10 after the stream-form kernel
    prof_mark(P, 11, s);
    launch_bucket_fft_dynamic(P, jd, P->d_part, P->d_z, P->d_energy + P->e_loc_off, P->L_loc, s);
    prof_mark(P, 12, s);
    launch_loc_tail(P, d_loc, (float2 *)d_val, d_msel, capacity, d_count, d_k, d_status, s);
    P->pdl = 0;
    if (fp64) launch_estimate_fp64(P, d_x, d_loc, d_val, capacity, s);
    prof_mark(P, 13, s);
    return cuda_status(cudaGetLastError());
}

extern "C" atsfft_status atsfft_exec(atsfft_plan_t plan, const void *d_x, int64_t *d_loc,
                                     void *d_val, int64_t capacity, int64_t *d_count,
                                     int64_t *d_k, int32_t *d_status, void *stream)
{
    return exec_common(plan, 1, d_x, d_loc, d_val, capacity, d_count, d_k, d_status, stream);
}

extern "C" atsfft_status atsfft_exec_2d(atsfft_plan_t plan, const void *d_img, int64_t *d_loc,
                                        void *d_val, int64_t capacity, int64_t *d_count,
                                        int64_t *d_k, int32_t *d_status, void *stream)
{
    return exec_common(plan, 2, d_img, d_loc, d_val, capacity, d_count, d_k, d_status, stream);
}

extern "C" atsfft_status atsfft_exec_sel(atsfft_plan_t plan, const void *d_x, int64_t *d_loc,
                                         void *d_val, uint8_t *d_medsel, int64_t capacity,
                                         int64_t *d_count, int64_t *d_k, int32_t *d_status,
                                         void *stream)
{
    if (!plan || (capacity > 0 && !d_medsel)) return ATSFFT_E_INVALID_ARG;
    return exec_common(plan, plan->ndim, d_x, d_loc, d_val, capacity, d_count, d_k, d_status,
                       stream, d_medsel);
}

extern "C" atsfft_status atsfft_hash_spectrum(atsfft_plan_t P, const void *d_x, int64_t B,
                                              int phase, int index, void *d_zhat, void *stream)
{
    if (!P || !d_x || !d_zhat || B <= 0 || (B & (B - 1)) || phase < 0 || phase > 2 || index < 0 ||
        P->p.precision != 0)
        return ATSFFT_E_INVALID_ARG;
    int b = 0;
    while (((int64_t)1 << b) < B) b++;
    if (b < P->b0 || b > P->b_hi) return ATSFFT_E_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    HashParam hp;
    hash_params_for(P->seed, phase, index, P->n, P->ndim, &hp);
    // the inspection hash lives in the spare slot after the location/estimation hashes
    HashParam *d_hp = P->d_le + 2 * kMaxLoops;
    if (caller_error_pending()) return ATSFFT_E_CUDA;
    cudaError_t e = cudaMemcpyAsync(d_hp, &hp, sizeof(hp), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_status(e);
    launch_single_hash(P, (const float2 *)d_x, b, hp, d_hp, P->d_z, s);
    launch_unpermute(P, P->d_z, d_hp, b, (float2 *)d_zhat, s);
    e = cudaStreamSynchronize(s);   // hp lives on this call's stack
    if (e != cudaSuccess) return cuda_status(e);
    return cuda_status(cudaGetLastError());
}

extern "C" atsfft_status atsfft_last_trace(atsfft_plan_t P, int64_t *h_B, int64_t *h_k,
                                           int max_trials, int *h_ntrials, void *stream)
{
    if (!P || !h_ntrials || max_trials < 0 || (max_trials > 0 && (!h_B || !h_k)))
        return ATSFFT_E_INVALID_ARG;
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_status(e);
    ExecState st;
    e = cudaMemcpy(&st, P->d_state, sizeof(st), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_status(e);
    *h_ntrials = st.ntrials;
    for (int i = 0; i < max_trials && i < st.ntrials && i < kMaxTrialsTrace; i++) {
        h_B[i] = st.trial_B[i];
        h_k[i] = st.trial_k[i];
    }
    return ATSFFT_OK;
}

extern "C" atsfft_status atsfft_last_result(atsfft_plan_t P, int64_t *h_B, int64_t *h_k,
                                            void *stream)
{
    if (!P || !h_B || !h_k) return ATSFFT_E_INVALID_ARG;
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_status(e);
    int32_t b = 0;
    int64_t k = 0;
    e = cudaMemcpy(&b, &P->d_state->b_star, sizeof(b), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&k, &P->d_state->k_star, sizeof(k), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_status(e);
    *h_B = (int64_t)1 << b;
    *h_k = k;
    return ATSFFT_OK;
}

extern "C" atsfft_status atsfft_set_profiling(atsfft_plan_t P, int on)
{
    if (!P) return ATSFFT_E_INVALID_ARG;
    if (on && !P->prof) {
        for (int i = 0; i <= kPhases; i++) {
            cudaError_t e = cudaEventCreate(&P->ev[i]);
            if (e != cudaSuccess) return cuda_status(e);
        }
    }
    if (!on && P->prof)
        for (int i = 0; i <= kPhases; i++) cudaEventDestroy(P->ev[i]);
    P->prof = on ? 1 : 0;
    return ATSFFT_OK;
}

extern "C" atsfft_status atsfft_phase_times(atsfft_plan_t P, float *h_ms, int max_phases,
                                            int *h_nphases, int64_t *h_launches, void *stream)
{
    if (!P || !h_nphases || max_phases < 0 || (max_phases > 0 && !h_ms)) return ATSFFT_E_INVALID_ARG;
    if (h_launches) *h_launches = P->launches;
    if (!P->prof) {
        *h_nphases = 0;
        return ATSFFT_OK;
    }
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_status(e);
    *h_nphases = kPhases;
    for (int i = 0; i < kPhases && i < max_phases; i++) {
        e = cudaEventElapsedTime(&h_ms[i], P->ev[i], P->ev[i + 1]);
        if (e != cudaSuccess) return cuda_status(e);
    }
    return ATSFFT_OK;
}

extern "C" atsfft_status atsfft_tail_stamps(atsfft_plan_t P, uint64_t *h_ns, int max_stamps,
                                            int *h_nstamps, void *stream)
{
    if (!P || !h_nstamps || max_stamps < 0 || (max_stamps > 0 && !h_ns)) return ATSFFT_E_INVALID_ARG;
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_status(e);
    TailStamps gb;
    e = cudaMemcpy(&gb, &P->d_state->bar, sizeof(gb), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_status(e);
    const int n = gb.nstamp < 32 ? (int)gb.nstamp : 32;
    *h_nstamps = n;
    for (int i = 0; i < n && i < max_stamps; i++) h_ns[i] = gb.stamp[i];
    return ATSFFT_OK;
}

// ---- batched execution: one graph with a branch per plan --------------------------

struct atsfft_batch_s {
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    int64_t kernels;
};

// Records the batch graph.  With host buffers (any pointer of an h_ array may be null:
// no copy), the graph also copies input i from pinned host memory on one copy chain in
// index order (transform i starts as soon as its own input has landed) and copies its
// outputs back after its exec.
static atsfft_status batch_create_impl(int n, const atsfft_plan_t *plans, const void *const *h_x,
                                       const void *const *d_x, int64_t *const *d_loc,
                                       void *const *d_val, const int64_t *capacity,
                                       int64_t *const *d_count, int64_t *const *d_k,
                                       int32_t *const *d_status, int64_t *const *h_loc,
                                       void *const *h_val, int64_t *const *h_count,
                                       int64_t *const *h_k, int32_t *const *h_status,
                                       atsfft_batch_t *out)
{
    if (!out) return ATSFFT_E_INVALID_ARG;
    *out = nullptr;
    if (n <= 0 || !plans || !d_x || !d_loc || !d_val || !capacity || !d_count || !d_k || !d_status)
        return ATSFFT_E_INVALID_ARG;
    for (int i = 0; i < n; i++) {
        if (!plans[i] || plans[i]->prof) return ATSFFT_E_INVALID_ARG;
        for (int j = 0; j < i; j++)
            if (plans[j] == plans[i]) return ATSFFT_E_INVALID_ARG;
    }
    atsfft_batch_s *B = new (std::nothrow) atsfft_batch_s;
    if (!B) return ATSFFT_E_NOMEM;
    memset(B, 0, sizeof(*B));
    // capture: fork from `main` to one stream per plan (and a copy stream for the host
    // inputs), each runs its exec, join back
    cudaStream_t main = nullptr, copy = nullptr;
    std::vector<cudaStream_t> side(n, nullptr);
    std::vector<cudaEvent_t> done(n, nullptr), landed(n, nullptr);
    cudaEvent_t fork = nullptr, copied = nullptr;
    atsfft_status st = ATSFFT_OK;
    cudaError_t e = cudaStreamCreateWithFlags(&main, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&copy, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&copied, cudaEventDisableTiming);
    for (int i = 0; i < n && e == cudaSuccess; i++) {
        e = cudaStreamCreateWithFlags(&side[i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&done[i], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&landed[i], cudaEventDisableTiming);
    }
    bool capturing = false;
    if (e == cudaSuccess) e = cudaStreamBeginCapture(main, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
        capturing = true;
        e = cudaEventRecord(fork, main);
    }
    if (e == cudaSuccess) e = cudaStreamWaitEvent(copy, fork, 0);
    for (int i = 0; i < n && e == cudaSuccess && st == ATSFFT_OK; i++) {
        atsfft_plan_s *P = plans[i];
        const size_t es = P->p.precision == 1 ? 16 : 8;   // complex value size
        if (h_x && h_x[i]) {
            e = cudaMemcpyAsync((void *)d_x[i], h_x[i], es * (size_t)P->ncoord,
                                cudaMemcpyHostToDevice, copy);
            if (e == cudaSuccess) e = cudaEventRecord(landed[i], copy);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(side[i], landed[i], 0);
        } else {
            e = cudaStreamWaitEvent(side[i], fork, 0);
        }
        if (e != cudaSuccess) break;
        st = exec_common(P, P->ndim, d_x[i], d_loc[i], d_val[i], capacity[i], d_count[i], d_k[i],
                         d_status[i], side[i]);
        B->kernels += P->launches;
        if (st != ATSFFT_OK) break;
        const size_t cap = (size_t)capacity[i];
        if (h_loc && h_loc[i] && cap)
            e = cudaMemcpyAsync(h_loc[i], d_loc[i], 8 * cap, cudaMemcpyDeviceToHost, side[i]);
        if (e == cudaSuccess && h_val && h_val[i] && cap)
            e = cudaMemcpyAsync(h_val[i], d_val[i], es * cap, cudaMemcpyDeviceToHost, side[i]);
        if (e == cudaSuccess && h_count && h_count[i])
            e = cudaMemcpyAsync(h_count[i], d_count[i], 8, cudaMemcpyDeviceToHost, side[i]);
        if (e == cudaSuccess && h_k && h_k[i])
            e = cudaMemcpyAsync(h_k[i], d_k[i], 8, cudaMemcpyDeviceToHost, side[i]);
        if (e == cudaSuccess && h_status && h_status[i])
            e = cudaMemcpyAsync(h_status[i], d_status[i], 4, cudaMemcpyDeviceToHost, side[i]);
        if (e == cudaSuccess) e = cudaEventRecord(done[i], side[i]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(main, done[i], 0);
    }
    if (e == cudaSuccess && st == ATSFFT_OK) e = cudaEventRecord(copied, copy);
    if (e == cudaSuccess && st == ATSFFT_OK) e = cudaStreamWaitEvent(main, copied, 0);
    if (capturing) {
        cudaGraph_t g = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(main, &g);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess && st == ATSFFT_OK) {
            B->graph = g;
            e = cudaGraphInstantiate(&B->exec, g, 0);
        } else if (g) {
            cudaGraphDestroy(g);
        }
    }
    for (int i = 0; i < n; i++) {
        if (done[i]) cudaEventDestroy(done[i]);
        if (landed[i]) cudaEventDestroy(landed[i]);
        if (side[i]) cudaStreamDestroy(side[i]);
    }
    if (fork) cudaEventDestroy(fork);
    if (copied) cudaEventDestroy(copied);
    if (copy) cudaStreamDestroy(copy);
    if (main) cudaStreamDestroy(main);
    if (st == ATSFFT_OK && e != cudaSuccess) st = cuda_status(e);
    if (st != ATSFFT_OK) {
        if (B->exec) cudaGraphExecDestroy(B->exec);
        if (B->graph) cudaGraphDestroy(B->graph);
        delete B;
        cudaGetLastError();
        return st;
    }
    *out = B;
    return ATSFFT_OK;
}

extern "C" atsfft_status atsfft_batch_create(int n, const atsfft_plan_t *plans,
                                             const void *const *d_x, int64_t *const *d_loc,
                                             void *const *d_val, const int64_t *capacity,
                                             int64_t *const *d_count, int64_t *const *d_k,
                                             int32_t *const *d_status, atsfft_batch_t *out)
{
    return batch_create_impl(n, plans, nullptr, d_x, d_loc, d_val, capacity, d_count, d_k, d_status,
                             nullptr, nullptr, nullptr, nullptr, nullptr, out);
}

extern "C" atsfft_status atsfft_batch_create_io(
    int n, const atsfft_plan_t *plans, const void *const *h_x, const void *const *d_x,
    int64_t *const *d_loc, void *const *d_val, const int64_t *capacity, int64_t *const *d_count,
    int64_t *const *d_k, int32_t *const *d_status, int64_t *const *h_loc, void *const *h_val,
    int64_t *const *h_count, int64_t *const *h_k, int32_t *const *h_status, atsfft_batch_t *out)
{
    return batch_create_impl(n, plans, h_x, d_x, d_loc, d_val, capacity, d_count, d_k, d_status,
                             h_loc, h_val, h_count, h_k, h_status, out);
}

extern "C" atsfft_status atsfft_batch_launch(atsfft_batch_t B, void *stream)
{
    if (!B || !B->exec) return ATSFFT_E_INVALID_ARG;
    return cuda_status(cudaGraphLaunch(B->exec, (cudaStream_t)stream));
}

extern "C" atsfft_status atsfft_batch_kernels(atsfft_batch_t B, int64_t *h_kernels)
{
    if (!B || !h_kernels) return ATSFFT_E_INVALID_ARG;
    *h_kernels = B->kernels;
    return ATSFFT_OK;
}

extern "C" atsfft_status atsfft_batch_destroy(atsfft_batch_t B)
{
    if (!B) return ATSFFT_E_INVALID_ARG;
    if (B->exec) cudaGraphExecDestroy(B->exec);
    if (B->graph) cudaGraphDestroy(B->graph);
    delete B;
    return ATSFFT_OK;
}
