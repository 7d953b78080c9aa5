"""ctypes wrapper around the C oracle (atsfft_oracle.c) -- TEST INFRASTRUCTURE ONLY.

`build()` compiles the C file with the system gcc into oracle/_build/; every
other function loads that library on first use (building it if missing).
"""

from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "atsfft_oracle.c")
_HDR = os.path.join(_HERE, "atsfft_oracle.h")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

MAX_TRIALS = 64


class OracleParams(C.Structure):
    _fields_ = [
        ("delta1", C.c_double), ("delta2", C.c_double),
        ("eps1", C.c_double), ("eps2", C.c_double),
        ("tune_max", C.c_int), ("loops_loc", C.c_int), ("loops_est", C.c_int),
        ("filter_alpha", C.c_double), ("filter_tol", C.c_double),
        ("thr_rel", C.c_double), ("thr_med", C.c_double), ("tie_eta", C.c_double),
        ("b_min_log2", C.c_int), ("b_max_log2", C.c_int),
        ("fixed_k", C.c_int), ("est_reuse_loc", C.c_int),
    ]


class _CResult(C.Structure):
    _fields_ = [
        ("status", C.c_int),
        ("B_star", C.c_int64), ("k_star", C.c_int64), ("count", C.c_int64),
        ("n_trials", C.c_int),
        ("trial_B", C.c_int64 * MAX_TRIALS), ("trial_k", C.c_int64 * MAX_TRIALS),
        ("trial_r", C.c_double * MAX_TRIALS),
        ("min_margin", C.c_double),
    ]


class OracleDecision(C.Structure):
    _fields_ = [
        ("phase", C.c_int32), ("hash", C.c_int32), ("kind", C.c_int32), ("pad", C.c_int32),
        ("c", C.c_int64), ("m", C.c_int64), ("margin", C.c_double),
    ]


DEC_THRESHOLD, DEC_DOMINANCE, DEC_TOPNUM, DEC_PIVOT = 1, 2, 3, 4
DEC_KIND = {1: "threshold", 2: "dominance", 3: "topnum", 4: "pivot"}


@dataclass
class Decision:
    phase: int      # 0 tuning trial, 1 location hash
    hash: int       # tuning: log2 B of the trial; location: hash index l
    kind: str       # threshold, dominance, topnum, pivot
    c: int
    m: int          # -1 when one bucket decides
    margin: float


@dataclass
class OracleResult:
    status: int
    B_star: int
    k_star: int
    count: int
    trials: list            # [(B, k, r), ...]
    min_margin: float
    loc: np.ndarray         # int64, ascending
    val: np.ndarray         # complex128


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, IEEE semantics, no -march flags)."""
    with _lock:
        newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
            os.makedirs(_OUT_DIR, exist_ok=True)
            tmp = _LIB + f".{os.getpid()}.tmp"
            subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"],
                           check=True)
            os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        # ATSFFT_ORACLE_LIB: load a prebuilt copy instead (the mutation test's builds of
        # the oracle with one planted mistake each)
        override = os.environ.get("ATSFFT_ORACLE_LIB")
        L = C.CDLL(override if override else build())
        i64, i32, dbl, u64 = C.c_int64, C.c_int, C.c_double, C.c_uint64
        P = C.POINTER
        L.orc_default_params.argtypes = [P(OracleParams)]
        L.orc_splitmix64_next.argtypes = [P(u64)]
        L.orc_splitmix64_next.restype = u64
        L.orc_hash_params.argtypes = [u64, i32, i32, i64, i32, P(i64)]
        L.orc_inv_mod.argtypes = [i64, i64]
        L.orc_inv_mod.restype = i64
        L.orc_filter_taps.argtypes = [i64, i64, dbl, dbl, P(i64), P(dbl), C.c_void_p]
        L.orc_filter_response.argtypes = [i64, i64, dbl, dbl, C.c_void_p]
        L.orc_fft.argtypes = [C.c_void_p, i64]
        L.orc_hash_spectrum_1d.argtypes = [C.c_void_p, i64, i64, u64, i32, i32, dbl, dbl, C.c_void_p]
        L.orc_hash_spectrum_2d.argtypes = [C.c_void_p, i64, i64, u64, i32, i32, dbl, dbl, C.c_void_p]
        L.orc_local_maxima.argtypes = [C.c_void_p, i64, i32, dbl, dbl, dbl, C.c_void_p,
                                       P(dbl), P(dbl)]
        L.orc_local_maxima.restype = i64
        L.orc_controller_branch.argtypes = [i64, i64, dbl, dbl]
        L.orc_top_num.argtypes = [C.c_void_p, C.c_void_p, i64, i64, dbl, C.c_void_p]
        L.orc_top_num.restype = i64
        L.orc_median_componentwise.argtypes = [C.c_void_p, i32, C.c_void_p]
        L.orc_atsfft_1d.argtypes = [C.c_void_p, i64, i64, P(OracleParams), u64, C.c_void_p,
                                    C.c_void_p, i64, P(_CResult)]
        L.orc_atsfft_2d.argtypes = L.orc_atsfft_1d.argtypes
        L.orc_estimates_1d.argtypes = [C.c_void_p, i64, i64, P(OracleParams), u64, C.c_void_p, i64,
                                       C.c_void_p]
        L.orc_local_maxima_log.argtypes = [C.c_void_p, i64, i32, dbl, dbl, dbl, i32, dbl,
                                           C.c_void_p, P(dbl), P(dbl), C.c_void_p, i64, P(i64)]
        L.orc_local_maxima_log.restype = i64
        L.orc_location_select_log.argtypes = [C.c_void_p, i64, i32, P(OracleParams), i64, dbl,
                                              C.c_void_p, P(dbl), C.c_void_p, i64, P(i64)]
        L.orc_location_select_log.restype = i64
        L.orc_bucket_of.argtypes = [i64, i64, i64, i64]
        L.orc_bucket_of.restype = i64
        L.orc_atsfft_log.argtypes = [C.c_void_p, i32, i64, i64, P(OracleParams), u64, C.c_void_p,
                                     C.c_void_p, i64, P(_CResult), dbl, C.c_void_p, i64, P(i64)]
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


def default_params(**overrides) -> OracleParams:
    p = OracleParams()
    lib().orc_default_params(C.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def splitmix64_stream(state: int, count: int) -> list:
    s = C.c_uint64(state)
    return [lib().orc_splitmix64_next(C.byref(s)) for _ in range(count)]


def hash_params(seed, phase, index, n, ndim=1):
    out = (C.c_int64 * 4)()
    lib().orc_hash_params(seed, phase, index, n, ndim, out)
    return list(out)[: 2 * ndim]


def inv_mod(sigma, n):
    return lib().orc_inv_mod(sigma, n)


def filter_taps(n, B, alpha=0.5, tol=1e-6):
    h, s = C.c_int64(), C.c_double()
    st = lib().orc_filter_taps(n, B, alpha, tol, C.byref(h), C.byref(s), None)
    if st:
        raise ValueError(f"orc_filter_taps status {st}")
    taps = np.zeros(2 * h.value + 1)
    lib().orc_filter_taps(n, B, alpha, tol, C.byref(h), C.byref(s), _ptr(taps))
    return h.value, s.value, taps


def filter_response(n, B, alpha=0.5, tol=1e-6):
    resp = np.zeros(n // B)
    st = lib().orc_filter_response(n, B, alpha, tol, _ptr(resp))
    if st:
        raise ValueError(f"orc_filter_response status {st}")
    return resp


def fft(a):
    buf = np.ascontiguousarray(a, dtype=np.complex128).copy()
    st = lib().orc_fft(_ptr(buf), len(buf))
    if st:
        raise ValueError(f"orc_fft status {st}")
    return buf


def _as_c128(x):
    return np.ascontiguousarray(np.asarray(x).astype(np.complex128))


def hash_spectrum_1d(x, B, seed, phase, index, alpha=0.5, tol=1e-6):
    xx = _as_c128(x)
    out = np.zeros(B, dtype=np.complex128)
    st = lib().orc_hash_spectrum_1d(_ptr(xx), len(xx), B, seed, phase, index, alpha, tol, _ptr(out))
    if st:
        raise ValueError(f"orc_hash_spectrum_1d status {st}")
    return out


def hash_spectrum_2d(x, B, seed, phase, index, alpha=0.5, tol=1e-6):
    xx = _as_c128(x)
    N = xx.shape[0]
    out = np.zeros((B, B), dtype=np.complex128)
    st = lib().orc_hash_spectrum_2d(_ptr(xx), N, B, seed, phase, index, alpha, tol, _ptr(out))
    if st:
        raise ValueError(f"orc_hash_spectrum_2d status {st}")
    return out


def local_maxima(E, ndim=1, thr_rel=1e-3, thr_med=20.0, eta=1e-2):
    E = np.ascontiguousarray(E, dtype=np.float64)
    side = E.shape[0]
    lst = np.zeros(E.size, dtype=np.int64)
    T, m = C.c_double(), C.c_double()
    cnt = lib().orc_local_maxima(_ptr(E), side, ndim, thr_rel, thr_med, eta, _ptr(lst),
                                 C.byref(T), C.byref(m))
    return lst[:cnt].copy(), T.value, m.value


def top_num(E, lm, num, eta=1e-2):
    """The location step's "num largest" cutoff (Algorithm 1) of the ascending local-maximum
    list lm with energies E (indexed by bucket): the kept buckets, ascending."""
    E = np.ascontiguousarray(E, dtype=np.float64)
    lm = np.ascontiguousarray(lm, dtype=np.int64)
    sel = np.zeros(max(len(lm), 1), dtype=np.int64)
    ns = lib().orc_top_num(_ptr(E), _ptr(lm), len(lm), num, eta, _ptr(sel))
    if ns < 0:
        raise ValueError(f"orc_top_num: invalid num {num}")
    return sel[:ns].copy()


def _decisions(buf, n):
    return [Decision(d.phase, d.hash, DEC_KIND[d.kind], d.c, d.m, d.margin) for d in buf[:n]]


def _logged(call, cap=4096):
    """Runs call(buffer, capacity, byref(count)) with a record buffer large enough for
    every record (once more with the exact size if the first buffer was too small)."""
    while True:
        buf = (OracleDecision * max(cap, 1))()
        n = C.c_int64()
        out = call(buf, cap, C.byref(n))
        if n.value <= cap:
            return out, _decisions(buf, n.value)
        cap = n.value


def local_maxima_log(E, ndim=1, mode=1, band=np.inf, thr_rel=1e-3, thr_med=20.0, eta=1e-2):
    """orc_local_maxima_log: (list, T, margin, decisions) with every deciding comparison
    whose margin is below `band` (mode 0: the count is the outcome; 1: the maxima set)."""
    E = np.ascontiguousarray(E, dtype=np.float64)
    side = E.shape[0]
    lst = np.zeros(E.size, dtype=np.int64)
    T, m = C.c_double(), C.c_double()
    cnt, dec = _logged(lambda buf, cap, n: lib().orc_local_maxima_log(
        _ptr(E), side, ndim, thr_rel, thr_med, eta, mode, band, _ptr(lst), C.byref(T),
        C.byref(m), buf, cap, n))
    return lst[:cnt].copy(), T.value, m.value, dec


def location_select_log(E, num, ndim=1, band=np.inf, params=None):
    """orc_location_select_log: (selected buckets, margin, decisions) of one location hash."""
    E = np.ascontiguousarray(E, dtype=np.float64)
    side = E.shape[0]
    sel = np.zeros(E.size, dtype=np.int64)
    m = C.c_double()
    p = params or default_params()
    ns, dec = _logged(lambda buf, cap, n: lib().orc_location_select_log(
        _ptr(E), side, ndim, C.byref(p), num, band, _ptr(sel), C.byref(m), buf, cap, n))
    if ns < 0:
        raise ValueError("orc_location_select_log: invalid arguments")
    return sel[:ns].copy(), m.value, dec


def bucket_of(i, sigma, n, B):
    """Bucket of coordinate i under a hash with this sigma on one axis (Eq. (10))."""
    h = lib().orc_bucket_of(int(i), int(sigma), int(n), int(B))
    if h < 0:
        raise ValueError("orc_bucket_of: invalid arguments")
    return h


def median_componentwise(v):
    v = np.ascontiguousarray(v, dtype=np.complex128)
    out = np.zeros(2)
    st = lib().orc_median_componentwise(_ptr(v), len(v), _ptr(out))
    if st:
        raise ValueError(f"orc_median_componentwise status {st}")
    return complex(out[0], out[1])


def controller_branch(k_prev, k_cur, delta1=0.02, delta2=0.05):
    return lib().orc_controller_branch(k_prev, k_cur, delta1, delta2)


def _run(fn, x, side, k_hint, params, seed, capacity):
    xx = _as_c128(x)
    if params is None:
        params = default_params()
    if capacity is None:
        capacity = 1 << 20
    loc = np.zeros(max(capacity, 1), dtype=np.int64)
    val = np.zeros(max(capacity, 1), dtype=np.complex128)
    r = _CResult()
    fn(_ptr(xx), side, k_hint, C.byref(params), seed, _ptr(loc), _ptr(val), capacity, C.byref(r))
    cnt = min(r.count, capacity)
    trials = [(r.trial_B[i], r.trial_k[i], r.trial_r[i]) for i in range(r.n_trials)]
    return OracleResult(r.status, r.B_star, r.k_star, r.count, trials, r.min_margin,
                        loc[:cnt].copy(), val[:cnt].copy())


def atsfft_1d(x, k_hint=0, params=None, seed=0, capacity=None) -> OracleResult:
    x = np.asarray(x)
    return _run(lib().orc_atsfft_1d, x, x.shape[0], k_hint, params, seed, capacity)


def atsfft_2d(x, k_hint=0, params=None, seed=0, capacity=None) -> OracleResult:
    x = np.asarray(x)
    return _run(lib().orc_atsfft_2d, x, x.shape[0], k_hint, params, seed, capacity)


def atsfft_log(x, k_hint=0, params=None, seed=0, capacity=None, band=2e-4):
    """atsfft_1d / atsfft_2d (by x's shape) that also returns the decisions whose margin
    lies below `band`: (OracleResult, [Decision, ...])."""
    x = np.asarray(x)
    ndim = x.ndim
    xx = _as_c128(x)
    if params is None:
        params = default_params()
    if capacity is None:
        capacity = 1 << 20
    loc = np.zeros(max(capacity, 1), dtype=np.int64)
    val = np.zeros(max(capacity, 1), dtype=np.complex128)
    r = _CResult()

    def call(buf, cap, n):
        lib().orc_atsfft_log(_ptr(xx), ndim, x.shape[0], k_hint, C.byref(params), seed,
                             _ptr(loc), _ptr(val), capacity, C.byref(r), band, buf, cap, n)

    _, dec = _logged(call)
    cnt = min(r.count, capacity)
    trials = [(r.trial_B[i], r.trial_k[i], r.trial_r[i]) for i in range(r.n_trials)]
    res = OracleResult(r.status, r.B_star, r.k_star, r.count, trials, r.min_margin,
                       loc[:cnt].copy(), val[:cnt].copy())
    return res, dec


def estimates_1d(x, B, loc, params=None, seed=0):
    """All loops_est estimates (Eq. (11), FP64, no median) of the coordinates `loc` of a
    1D signal at B buckets: complex array [len(loc), loops_est]."""
    x = _as_c128(x)
    p = params or default_params()
    loc = np.ascontiguousarray(np.asarray(loc, dtype=np.int64))
    out = np.zeros((len(loc), p.loops_est), dtype=np.complex128)
    st = lib().orc_estimates_1d(_ptr(x), x.size, B, C.byref(p), seed & 0xFFFFFFFFFFFFFFFF,
                                _ptr(loc), len(loc), _ptr(out))
    if st != 0:
        raise ValueError(f"orc_estimates_1d: status {st}")
    return out
