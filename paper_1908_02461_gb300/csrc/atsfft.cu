// atsfft.cu -- C ABI entry points: one transform = tuning, location, estimation, all
// enqueued on the caller's stream with no host synchronisation.
//
//  tuning   : the hash of every B in the plan's range is evaluated (bin, bucket FFT,
//             energies, threshold, local-maximum count); the controller then walks
//             Eqs. (12)/(14) over those counts on the device and fixes B*, k*.  Because the
//             stop reading visits every B at most once, evaluating all of them up front
//             gives exactly the sequential trajectory while replacing a chain of dependent
//             trials by one batch.
//  location : the L_loc + L_est hashes at B* are binned in one pass over the signal,
//             transformed, and the location hashes' maxima are cut to k* and vote.
//  estimate : kept coordinates in ascending order, Eq. (11), median.
// Kernels that depend on B* read it from device memory; every shape they could need is
// launched and the ones that do not match exit at once.
#include <string.h>

#include "common.cuh"

using namespace atsfft;

static atsfft_status exec_common(atsfft_plan_t P, int ndim, const void *d_x, int64_t *d_loc,
                                 void *d_val, int64_t capacity, int64_t *d_count, int64_t *d_k,
                                 int32_t *d_status, void *stream)
{
    if (!P || P->ndim != ndim || !d_x || capacity < 0 || (capacity > 0 && (!d_loc || !d_val)) ||
        !d_count || !d_k || !d_status)
        return ATSFFT_E_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const float2 *x = (const float2 *)d_x;
    cudaGetLastError();   // clear a stale error so the status below is this call's
    P->launches = 0;
    launch_reset(P, s);
    prof_mark(P, 0, s);
    launch_tuning(P, x, s);       // marks phases 1 and 2 between its kernels
    prof_mark(P, 3, s);
    launch_tune_tail(P, s);
    prof_mark(P, 4, s);
    const Job *jd = &P->d_state->job;
    launch_le_bin(P, x, jd, s);   // marks phase 5 after the stream-form kernel
    prof_mark(P, 6, s);
    launch_bucket_fft_dynamic(P, jd, P->d_part, P->d_z, P->d_energy + P->e_loc_off, P->L_loc, s);
    prof_mark(P, 7, s);
    launch_loc_tail(P, d_loc, (float2 *)d_val, capacity, d_count, d_k, d_status, s);
    prof_mark(P, 8, s);
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

extern "C" atsfft_status atsfft_hash_spectrum(atsfft_plan_t P, const void *d_x, int64_t B,
                                              int phase, int index, void *d_zhat, void *stream)
{
    if (!P || !d_x || !d_zhat || B <= 0 || (B & (B - 1)) || phase < 0 || phase > 2 || index < 0)
        return ATSFFT_E_INVALID_ARG;
    int b = 0;
    while (((int64_t)1 << b) < B) b++;
    if (b < P->b0 || b > P->b_hi) return ATSFFT_E_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    HashParam hp;
    hash_params_for(P->seed, phase, index, P->n, P->ndim, &hp);
    // the inspection hash lives in the spare slot after the location/estimation hashes
    HashParam *d_hp = P->d_le + 2 * kMaxLoops;
    cudaGetLastError();
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
    GridBarrier gb;
    e = cudaMemcpy(&gb, &P->d_state->bar, sizeof(gb), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_status(e);
    const int n = gb.nstamp < 32 ? (int)gb.nstamp : 32;
    *h_nstamps = n;
    for (int i = 0; i < n && i < max_stamps; i++) h_ns[i] = gb.stamp[i];
    return ATSFFT_OK;
}
