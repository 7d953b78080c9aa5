"""ctypes binding of the ATSFFT C ABI (include/atsfft.h).

Argument marshalling only: every step of a transform runs in the CUDA library.  The
functions keep the C names; device buffers are passed as torch CUDA tensors (their
data pointers) or raw integers.  Loading fails loudly when the library is missing.
"""

from __future__ import annotations

import ctypes as C
import os

from .build import LIB_PATH

OK = 0
E_INVALID_ARG = 1
E_NOMEM = 2
E_CUDA = 3
E_NOT_CONVERGED = 4
E_NOT_SPARSE = 5
E_CAPACITY = 6


class atsfft_params(C.Structure):
    _fields_ = [
        ("delta1", C.c_double), ("delta2", C.c_double),
        ("eps1", C.c_double), ("eps2", C.c_double),
        ("tune_max", C.c_int), ("loops_loc", C.c_int), ("loops_est", C.c_int),
        ("filter_alpha", C.c_double), ("filter_tol", C.c_double),
        ("thr_rel", C.c_double), ("thr_med", C.c_double), ("tie_eta", C.c_double),
        ("b_min_log2", C.c_int), ("b_max_log2", C.c_int),
        ("coop_blocks_per_sm", C.c_int),
        ("tune_stages", C.c_int),
        ("fixed_k", C.c_int), ("est_reuse_loc", C.c_int),
        ("precision", C.c_int), ("coop_sms", C.c_int),
    ]


EXPORTED = ["atsfft_default_params", "atsfft_plan", "atsfft_exec", "atsfft_exec_2d",
            "atsfft_destroy", "atsfft_status_string", "atsfft_hash_spectrum",
            "atsfft_window_response", "atsfft_last_trace", "atsfft_set_profiling",
            "atsfft_phase_times", "atsfft_tail_stamps", "atsfft_hash_spectrum_noalloc",
            "atsfft_batch_create", "atsfft_batch_create_io", "atsfft_batch_launch",
            "atsfft_batch_kernels",
            "atsfft_batch_destroy", "atsfft_plan_clone", "atsfft_exec_sel",
            "atsfft_estimate_apply", "atsfft_estimate_adjoint", "atsfft_last_result",
            "atsfft_mufu_probe"]

PHASES = ["tune1_bin", "tune1_fft", "tune1_tail", "tune2_bin", "tune2_fft", "tune2_tail",
          "tune3_bin", "tune3_fft", "tune3_tail", "le_bin_stream", "le_bin_gather", "le_fft",
          "loc_tail"]

_lib = None


def load(path: str | None = None):
    """Load libatsfft.so (raises if it has not been built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise ImportError(f"ATSFFT CUDA library not built ({p}); run "
                          "paper_1908_02461_gb300.build.build() first")
    L = C.CDLL(p)
    vp, i64, i32, u64, P = C.c_void_p, C.c_int64, C.c_int, C.c_uint64, C.POINTER
    L.atsfft_default_params.argtypes = [P(atsfft_params)]
    L.atsfft_default_params.restype = None
    L.atsfft_plan.argtypes = [P(vp), i32, P(i64), i64, P(atsfft_params), u64]
    L.atsfft_plan.restype = i32
    L.atsfft_exec.argtypes = [vp, vp, vp, vp, i64, vp, vp, vp, vp]
    L.atsfft_exec.restype = i32
    L.atsfft_exec_2d.argtypes = L.atsfft_exec.argtypes
    L.atsfft_exec_2d.restype = i32
    L.atsfft_destroy.argtypes = [vp]
    L.atsfft_destroy.restype = i32
    L.atsfft_status_string.argtypes = [i32]
    L.atsfft_status_string.restype = C.c_char_p
    L.atsfft_hash_spectrum.argtypes = [vp, vp, i64, i32, i32, vp, vp]
    L.atsfft_hash_spectrum.restype = i32
    L.atsfft_window_response.argtypes = [vp, i64, vp]
    L.atsfft_window_response.restype = i32
    L.atsfft_last_trace.argtypes = [vp, vp, vp, i32, P(i32), vp]
    L.atsfft_last_trace.restype = i32
    L.atsfft_set_profiling.argtypes = [vp, i32]
    L.atsfft_set_profiling.restype = i32
    L.atsfft_phase_times.argtypes = [vp, vp, i32, P(i32), P(i64), vp]
    L.atsfft_phase_times.restype = i32
    L.atsfft_tail_stamps.argtypes = [vp, vp, i32, P(i32), vp]
    L.atsfft_tail_stamps.restype = i32
    L.atsfft_hash_spectrum_noalloc.argtypes = [vp, i64, i64, u64, i32, i32, vp, vp]
    L.atsfft_hash_spectrum_noalloc.restype = i32
    L.atsfft_last_result.argtypes = [vp, P(i64), P(i64), vp]
    L.atsfft_last_result.restype = i32
    L.atsfft_exec_sel.argtypes = [vp, vp, vp, vp, vp, i64, vp, vp, vp, vp]
    L.atsfft_exec_sel.restype = i32
    L.atsfft_estimate_apply.argtypes = [vp, i64, vp, vp, vp, i64, vp, vp]
    L.atsfft_estimate_apply.restype = i32
    L.atsfft_estimate_adjoint.argtypes = [vp, i64, vp, vp, i64, vp, vp, vp]
    L.atsfft_estimate_adjoint.restype = i32
    L.atsfft_plan_clone.argtypes = [vp, P(vp)]
    L.atsfft_plan_clone.restype = i32
    L.atsfft_batch_create.argtypes = [i32, vp, vp, vp, vp, vp, vp, vp, vp, P(vp)]
    L.atsfft_batch_create.restype = i32
    L.atsfft_batch_create_io.argtypes = [i32, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp,
                                         vp, P(vp)]
    L.atsfft_batch_create_io.restype = i32
    L.atsfft_batch_launch.argtypes = [vp, vp]
    L.atsfft_batch_launch.restype = i32
    L.atsfft_batch_kernels.argtypes = [vp, P(i64)]
    L.atsfft_batch_kernels.restype = i32
    L.atsfft_batch_destroy.argtypes = [vp]
    L.atsfft_batch_destroy.restype = i32
    L.atsfft_mufu_probe.argtypes = [i64, P(C.c_double), vp]
    L.atsfft_mufu_probe.restype = i32
    if path is None:
        _lib = L
    return L


def _ptr(t):
    """Device (or host) address of a tensor / array / integer."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if hasattr(t, "data_ptr"):
        return t.data_ptr()
    if hasattr(t, "ctypes"):
        return t.ctypes.data
    raise TypeError(f"cannot take the address of {type(t)}")


def atsfft_default_params() -> atsfft_params:
    p = atsfft_params()
    load().atsfft_default_params(C.byref(p))
    return p


def atsfft_status_string(status: int) -> str:
    return load().atsfft_status_string(status).decode()


def atsfft_plan(ndim: int, shape, k_hint: int = 0, params: atsfft_params | None = None,
                seed: int = 0):
    """Returns (status, plan handle)."""
    h = C.c_void_p()
    sh = (C.c_int64 * 2)(*(list(shape) + [0] * (2 - len(shape))))
    st = load().atsfft_plan(C.byref(h), ndim, sh, k_hint, C.byref(params) if params else None,
                            seed & 0xFFFFFFFFFFFFFFFF)
    return st, h.value


def atsfft_exec(plan, d_x, d_loc, d_val, capacity, d_count, d_k, d_status, stream=None) -> int:
    return load().atsfft_exec(plan, _ptr(d_x), _ptr(d_loc), _ptr(d_val), capacity, _ptr(d_count),
                              _ptr(d_k), _ptr(d_status), _ptr(stream))


def atsfft_exec_2d(plan, d_img, d_loc, d_val, capacity, d_count, d_k, d_status, stream=None) -> int:
    return load().atsfft_exec_2d(plan, _ptr(d_img), _ptr(d_loc), _ptr(d_val), capacity,
                                 _ptr(d_count), _ptr(d_k), _ptr(d_status), _ptr(stream))


def atsfft_destroy(plan) -> int:
    return load().atsfft_destroy(plan)


def atsfft_hash_spectrum(plan, d_x, B, phase, index, d_zhat, stream=None) -> int:
    return load().atsfft_hash_spectrum(plan, _ptr(d_x), B, phase, index, _ptr(d_zhat), _ptr(stream))


def atsfft_window_response(plan, B, h_resp) -> int:
    return load().atsfft_window_response(plan, B, _ptr(h_resp))


def atsfft_last_trace(plan, h_B, h_k, max_trials, stream=None):
    """Returns (status, number of trials)."""
    nt = C.c_int()
    st = load().atsfft_last_trace(plan, _ptr(h_B), _ptr(h_k), max_trials, C.byref(nt), _ptr(stream))
    return st, nt.value


def atsfft_set_profiling(plan, on: bool) -> int:
    return load().atsfft_set_profiling(plan, 1 if on else 0)


def atsfft_phase_times(plan, h_ms, max_phases, stream=None):
    """Returns (status, number of phases, launches of the last exec)."""
    nph = C.c_int()
    nl = C.c_int64()
    st = load().atsfft_phase_times(plan, _ptr(h_ms), max_phases, C.byref(nph), C.byref(nl),
                                   _ptr(stream))
    return st, nph.value, nl.value


def atsfft_tail_stamps(plan, h_ns, max_stamps, stream=None):
    """Returns (status, number of stamps)."""
    n = C.c_int()
    st = load().atsfft_tail_stamps(plan, _ptr(h_ns), max_stamps, C.byref(n), _ptr(stream))
    return st, n.value


def atsfft_hash_spectrum_noalloc(d_x, n, B, seed, phase, index, d_zhat, stream=None) -> int:
    """One hash's bucket spectrum without a plan or any allocation (see include/atsfft.h)."""
    return load().atsfft_hash_spectrum_noalloc(_ptr(d_x), n, B, seed & 0xFFFFFFFFFFFFFFFF, phase,
                                               index, _ptr(d_zhat), _ptr(stream))


def atsfft_batch_create(plans, d_x, d_loc, d_val, capacity, d_count, d_k, d_status):
    """Returns (status, batch handle).  Every argument is a sequence of equal length."""
    n = len(plans)
    arr = lambda xs: (C.c_void_p * n)(*[_ptr(x) for x in xs])
    h = C.c_void_p()
    st = load().atsfft_batch_create(n, (C.c_void_p * n)(*plans), arr(d_x), arr(d_loc), arr(d_val),
                                    (C.c_int64 * n)(*capacity), arr(d_count), arr(d_k),
                                    arr(d_status), C.byref(h))
    return st, h.value


def atsfft_batch_create_io(plans, h_x, d_x, d_loc, d_val, capacity, d_count, d_k, d_status,
                           h_loc, h_val, h_count, h_k, h_status):
    """Returns (status, batch handle); host sequences may hold None (no copy)."""
    n = len(plans)
    arr = lambda xs: (C.c_void_p * n)(*[_ptr(x) if x is not None else None for x in xs])
    h = C.c_void_p()
    st = load().atsfft_batch_create_io(n, (C.c_void_p * n)(*plans), arr(h_x), arr(d_x), arr(d_loc),
                                       arr(d_val), (C.c_int64 * n)(*capacity), arr(d_count),
                                       arr(d_k), arr(d_status), arr(h_loc), arr(h_val),
                                       arr(h_count), arr(h_k), arr(h_status), C.byref(h))
    return st, h.value


def atsfft_batch_launch(batch, stream=None) -> int:
    return load().atsfft_batch_launch(batch, _ptr(stream))


def atsfft_batch_kernels(batch):
    """Returns (status, kernel launches per batch launch)."""
    k = C.c_int64()
    st = load().atsfft_batch_kernels(batch, C.byref(k))
    return st, k.value


def atsfft_batch_destroy(batch) -> int:
    return load().atsfft_batch_destroy(batch)


def atsfft_plan_clone(src):
    """Returns (status, plan handle)."""
    h = C.c_void_p()
    st = load().atsfft_plan_clone(src, C.byref(h))
    return st, h.value


def atsfft_exec_sel(plan, d_x, d_loc, d_val, d_medsel, capacity, d_count, d_k, d_status,
                    stream=None) -> int:
    return load().atsfft_exec_sel(plan, _ptr(d_x), _ptr(d_loc), _ptr(d_val), _ptr(d_medsel),
                                  capacity, _ptr(d_count), _ptr(d_k), _ptr(d_status), _ptr(stream))


def atsfft_estimate_apply(plan, B, d_u, d_loc, d_medsel, count, d_out, stream=None) -> int:
    return load().atsfft_estimate_apply(plan, B, _ptr(d_u), _ptr(d_loc), _ptr(d_medsel), count,
                                        _ptr(d_out), _ptr(stream))


def atsfft_estimate_adjoint(plan, B, d_loc, d_medsel, count, d_gval, d_gx, stream=None) -> int:
    return load().atsfft_estimate_adjoint(plan, B, _ptr(d_loc), _ptr(d_medsel), count,
                                          _ptr(d_gval), _ptr(d_gx), _ptr(stream))


def atsfft_last_result(plan, stream=None):
    """Returns (status, B*, k*) of the plan's last transform."""
    B, k = C.c_int64(), C.c_int64()
    st = load().atsfft_last_result(plan, C.byref(B), C.byref(k), _ptr(stream))
    return st, B.value, k.value


def atsfft_mufu_probe(iters, stream=None):
    """Returns (status, measured exp2 + reciprocal operations per second)."""
    r = C.c_double()
    st = load().atsfft_mufu_probe(int(iters), C.byref(r), _ptr(stream))
    return st, r.value
