"""GB300 (sm_103a) ATSFFT: sparse FFT with sparsity detection (arXiv 1908.02461).

The compute path is the CUDA library behind include/atsfft.h; this package is its
ctypes binding (`_lib`, same function names as the C ABI) plus `Plan`, a small
convenience wrapper that allocates the output buffers with torch.  PyTorch only
provides device memory and streams here.  There is no CPU fallback: using a plan
without the built library or without a GPU raises.
"""

from __future__ import annotations

from . import _lib
from ._lib import (  # noqa: F401
    E_CAPACITY,
    E_CUDA,
    E_INVALID_ARG,
    E_NOMEM,
    E_NOT_CONVERGED,
    E_NOT_SPARSE,
    OK,
    atsfft_batch_create,
    atsfft_batch_create_io,
    atsfft_batch_destroy,
    atsfft_batch_kernels,
    atsfft_batch_launch,
    atsfft_default_params,
    atsfft_destroy,
    atsfft_estimate_adjoint,
    atsfft_estimate_apply,
    atsfft_exec_sel,
    atsfft_exec,
    atsfft_exec_2d,
    atsfft_hash_spectrum,
    atsfft_last_result,
    atsfft_last_trace,
    atsfft_mufu_probe,
    atsfft_params,
    atsfft_phase_times,
    atsfft_plan,
    atsfft_plan_clone,
    atsfft_set_profiling,
    atsfft_status_string,
    atsfft_tail_stamps,
    atsfft_window_response,
)
from .build import build  # noqa: F401


class ATSFFTError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {atsfft_status_string(status)} (status {status})")
        self.status = status


class ArgumentError(ATSFFTError, ValueError):
    """A buffer the binding refuses before calling the library: the C ABI takes raw
    pointers, so a tensor of the wrong element type, size or device would be read or
    written out of bounds there."""

    def __init__(self, what: str, detail: str):
        RuntimeError.__init__(self, f"{what}: {detail}")
        self.status = E_INVALID_ARG


def check_buffer(what: str, name: str, t, dtype, device=None, numel=None, min_numel=None,
                 pinned=False):
    """Raises ArgumentError unless `t` is a contiguous tensor of `dtype` with exactly
    `numel` (or at least `min_numel`) elements, on `device` (or, with pinned=True, in
    pinned host memory)."""
    import torch

    if not isinstance(t, torch.Tensor):
        raise ArgumentError(what, f"{name} must be a torch tensor, not {type(t).__name__}")
    if t.dtype != dtype:
        raise ArgumentError(what, f"{name} must be {dtype}, not {t.dtype}")
    if not t.is_contiguous():
        raise ArgumentError(what, f"{name} must be contiguous")
    if numel is not None and t.numel() != numel:
        raise ArgumentError(what, f"{name} must hold {numel} elements, not {t.numel()}")
    if min_numel is not None and t.numel() < min_numel:
        raise ArgumentError(what, f"{name} must hold at least {min_numel} elements, not {t.numel()}")
    if pinned:
        if t.device.type != "cpu" or not t.is_pinned():
            raise ArgumentError(what, f"{name} must be a pinned CPU tensor")
    elif device is not None and t.device != device:
        raise ArgumentError(what, f"{name} must be on {device}, not {t.device}")


def _power_of_two(v) -> bool:
    import operator

    try:
        v = operator.index(v)   # Python and NumPy integers
    except TypeError:
        return False
    return v > 0 and (v & (v - 1)) == 0


def atsfft_hash_spectrum_noalloc(d_x, n, B, seed, phase, index, d_zhat, stream=None) -> int:
    """The allocation-free bucket spectrum of one hash (include/atsfft.h), with the two
    buffers checked first: d_x must be a contiguous complex64 tensor of n values and
    d_zhat one of at least B values, both on the current CUDA device (the C call reads
    and writes them through raw pointers).  Returns the status code."""
    import torch

    what = "atsfft_hash_spectrum_noalloc"
    if not (_power_of_two(n) and _power_of_two(B)):
        return E_INVALID_ARG
    dev = (torch.device("cuda", torch.cuda.current_device()) if torch.cuda.is_available()
           else torch.device("cuda"))
    check_buffer(what, "d_x", d_x, torch.complex64, dev, numel=int(n))
    check_buffer(what, "d_zhat", d_zhat, torch.complex64, dev, min_numel=int(B))
    return _lib.atsfft_hash_spectrum_noalloc(d_x, int(n), int(B), seed, phase, index, d_zhat,
                                             stream)


def params(**overrides) -> atsfft_params:
    p = atsfft_default_params()
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


class Plan:
    """A plan for 1D signals of length n (shape=(n,)) or N x N images (shape=(N, N))."""

    def __init__(self, shape, k_hint: int = 0, params: atsfft_params | None = None, seed: int = 0):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("ATSFFT needs a CUDA GPU; there is no CPU path")
        self.shape = tuple(int(s) for s in shape)
        self.ndim = len(self.shape)
        st, h = atsfft_plan(self.ndim, self.shape, k_hint, params, seed)
        if st != OK:
            raise ATSFFTError(st, "atsfft_plan")
        self.handle = h
        self.device = torch.device("cuda", torch.cuda.current_device())
        self._scalars = torch.zeros(3, dtype=torch.int64, device=self.device)
        # input and value dtype: complex128 for the FP64 path
        self.dtype = torch.complex128 if (params is not None and params.precision == 1) else torch.complex64

    @property
    def numel(self) -> int:
        """Samples of one input: n, or N * N."""
        m = 1
        for s in self.shape:
            m *= s
        return m

    def check_exec_buffers(self, what, x, loc, val, count, k, status):
        """The buffers of one transform (capacity = loc.numel())."""
        import torch

        check_buffer(what, "x", x, self.dtype, self.device, numel=self.numel)
        check_buffer(what, "loc", loc, torch.int64, self.device)
        check_buffer(what, "val", val, self.dtype, self.device, min_numel=loc.numel())
        check_buffer(what, "count", count, torch.int64, self.device, min_numel=1)
        check_buffer(what, "k", k, torch.int64, self.device, min_numel=1)
        check_buffer(what, "status", status, torch.int32, self.device, min_numel=1)

    def clone(self) -> "Plan":
        """A plan with the same tables and its own scratch (atsfft_plan_clone)."""
        import torch

        st, h = atsfft_plan_clone(self.handle)
        if st != OK:
            raise ATSFFTError(st, "atsfft_plan_clone")
        other = Plan.__new__(Plan)
        other.shape, other.ndim, other.handle, other.device = self.shape, self.ndim, h, self.device
        other.dtype = self.dtype
        other._scalars = torch.zeros(3, dtype=torch.int64, device=self.device)
        return other

    def close(self):
        if getattr(self, "handle", None):
            atsfft_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def exec_async(self, x, loc, val, count, k, status, stream=None):
        """Enqueue one transform into caller-provided device buffers."""
        import torch

        self.check_exec_buffers("exec", x, loc, val, count, k, status)
        s = stream if stream is not None else torch.cuda.current_stream().cuda_stream
        fn = atsfft_exec if self.ndim == 1 else atsfft_exec_2d
        st = fn(self.handle, x, loc, val, loc.numel(), count, k, status, s)
        if st != OK:
            raise ATSFFTError(st, "atsfft_exec")

    def __call__(self, x, capacity: int | None = None):
        """Transform x (complex64 CUDA tensor); returns (loc, val, k_star, status, count) after sync."""
        import torch

        check_buffer("exec", "x", x, self.dtype, self.device, numel=self.numel)
        if tuple(x.shape) != self.shape:
            raise ArgumentError("exec", f"x has shape {tuple(x.shape)}, the plan {self.shape}")
        cap = capacity if capacity is not None else 1 << 16
        loc = torch.empty(cap, dtype=torch.int64, device=x.device)
        val = torch.empty(cap, dtype=self.dtype, device=x.device)
        count = torch.zeros(1, dtype=torch.int64, device=x.device)
        k = torch.zeros(1, dtype=torch.int64, device=x.device)
        status = torch.zeros(1, dtype=torch.int32, device=x.device)
        self.exec_async(x, loc, val, count, k, status)
        n = int(count.item())
        m = min(n, cap)
        return loc[:m], val[:m], int(k.item()), int(status.item()), n

    def exec_sel(self, x, capacity: int | None = None):
        """Transform x (1D or 2D) and also return the median's hash selections.

        Returns (loc, val, medsel, B_star, k_star, status, count); medsel is uint8
        [count, 2]: the estimation hash of the real and of the imaginary median."""
        import torch

        check_buffer("exec_sel", "x", x, torch.complex64, self.device, numel=self.numel)
        cap = capacity if capacity is not None else 1 << 16
        loc = torch.empty(cap, dtype=torch.int64, device=x.device)
        val = torch.empty(cap, dtype=torch.complex64, device=x.device)
        msel = torch.zeros(cap, 2, dtype=torch.uint8, device=x.device)
        count = torch.zeros(1, dtype=torch.int64, device=x.device)
        k = torch.zeros(1, dtype=torch.int64, device=x.device)
        status = torch.zeros(1, dtype=torch.int32, device=x.device)
        st = atsfft_exec_sel(self.handle, x, loc, val, msel, cap, count, k, status,
                             torch.cuda.current_stream().cuda_stream)
        if st != OK:
            raise ATSFFTError(st, "atsfft_exec_sel")
        n = int(count.item())
        m = min(n, cap)
        st, B, _ = atsfft_last_result(self.handle, torch.cuda.current_stream().cuda_stream)
        if st != OK:
            raise ATSFFTError(st, "atsfft_last_result")
        return loc[:m], val[:m], msel[:m], B, int(k.item()), int(status.item()), n

    def estimate_apply(self, B: int, u, loc, msel):
        """Eq. (11) at the fixed support `loc` with median selections `msel`, applied to u."""
        import torch

        check_buffer("estimate_apply", "u", u, torch.complex64, self.device, numel=self.numel)
        check_buffer("estimate_apply", "loc", loc, torch.int64, self.device)
        check_buffer("estimate_apply", "msel", msel, torch.uint8, self.device,
                     min_numel=2 * loc.numel())
        out = torch.empty(loc.numel(), dtype=torch.complex64, device=u.device)
        st = atsfft_estimate_apply(self.handle, B, u, loc, msel, loc.numel(), out,
                                   torch.cuda.current_stream().cuda_stream)
        if st != OK:
            raise ATSFFTError(st, "atsfft_estimate_apply")
        return out

    def estimate_adjoint(self, B: int, loc, msel, g):
        """Adjoint of estimate_apply for the output gradient g (complex64 [count])."""
        import torch

        g = g.contiguous()
        check_buffer("estimate_adjoint", "loc", loc, torch.int64, self.device)
        check_buffer("estimate_adjoint", "msel", msel, torch.uint8, self.device,
                     min_numel=2 * loc.numel())
        check_buffer("estimate_adjoint", "g", g, torch.complex64, self.device,
                     min_numel=loc.numel())
        gx = torch.empty(self.numel, dtype=torch.complex64, device=g.device)
        st = atsfft_estimate_adjoint(self.handle, B, loc, msel, loc.numel(), g, gx,
                                     torch.cuda.current_stream().cuda_stream)
        if st != OK:
            raise ATSFFTError(st, "atsfft_estimate_adjoint")
        return gx

    def hash_spectrum(self, x, B: int, phase: int, index: int):
        import torch

        check_buffer("hash_spectrum", "x", x, torch.complex64, self.device, numel=self.numel)
        if not _power_of_two(B) or B > self.shape[0]:
            raise ArgumentError("hash_spectrum", f"B = {B} is not a power of two up to {self.shape[0]}")
        out = torch.empty((B,) if self.ndim == 1 else (B, B), dtype=torch.complex64, device=x.device)
        st = atsfft_hash_spectrum(self.handle, x, B, phase, index, out,
                                  torch.cuda.current_stream().cuda_stream)
        if st != OK:
            raise ATSFFTError(st, "atsfft_hash_spectrum")
        return out

    def window_response(self, B: int):
        import numpy as np

        D = self.shape[0] // B
        out = np.zeros(D, dtype=np.float64)
        st = atsfft_window_response(self.handle, B, out)
        if st != OK:
            raise ATSFFTError(st, "atsfft_window_response")
        return out

    def set_profiling(self, on: bool = True):
        st = atsfft_set_profiling(self.handle, on)
        if st != OK:
            raise ATSFFTError(st, "atsfft_set_profiling")

    def phase_times(self, stream=None):
        """Per-phase ms of the last exec (dict) and its kernel launch count."""
        import numpy as np
        import torch

        from ._lib import PHASES

        ms = np.zeros(len(PHASES), dtype=np.float32)
        s = stream if stream is not None else torch.cuda.current_stream().cuda_stream
        st, nph, nl = atsfft_phase_times(self.handle, ms, len(PHASES), s)
        if st != OK:
            raise ATSFFTError(st, "atsfft_phase_times")
        return dict(zip(PHASES[:nph], ms[:nph].tolist())), nl

    def tail_stamps(self):
        """Device ns stamps of the last exec's tail kernels (starts and barriers)."""
        import numpy as np
        import torch

        buf = np.zeros(32, dtype=np.uint64)
        st, n = atsfft_tail_stamps(self.handle, buf, 32, torch.cuda.current_stream().cuda_stream)
        if st != OK:
            raise ATSFFTError(st, "atsfft_tail_stamps")
        return buf[:n].tolist()

    def last_trace(self):
        import numpy as np
        import torch

        Bs = np.zeros(64, dtype=np.int64)
        ks = np.zeros(64, dtype=np.int64)
        st, nt = atsfft_last_trace(self.handle, Bs, ks, 64, torch.cuda.current_stream().cuda_stream)
        if st != OK:
            raise ATSFFTError(st, "atsfft_last_trace")
        return list(zip(Bs[:nt].tolist(), ks[:nt].tolist()))


class Batch:
    """Several plans' transforms recorded into one CUDA graph (atsfft_batch_create).

    `items` is a sequence of (plan, x, loc, val, count, k, status) with device tensors
    that must stay alive and in place; `launch()` replays all transforms at once.  With
    `host` (one dict per item with pinned CPU tensors under any of the keys x, loc, val,
    count, k, status), the graph also copies each input from host memory first, in item
    order, and the outputs back (atsfft_batch_create_io)."""

    def __init__(self, items, host=None):
        import torch

        self._keep = list(items)   # the graph holds raw pointers into these tensors
        for it in items:
            it[0].check_exec_buffers("batch", *it[1:7])
        if host is not None:
            if len(host) != len(items):
                raise ArgumentError("batch", f"{len(host)} host dicts for {len(items)} items")
            for it, hd in zip(items, host):
                plan, cap = it[0], it[2].numel()
                want = dict(x=(plan.dtype, plan.numel, None), loc=(torch.int64, None, cap),
                            val=(plan.dtype, None, cap), count=(torch.int64, None, 1),
                            k=(torch.int64, None, 1), status=(torch.int32, None, 1))
                for key, t in hd.items():
                    if key not in want:
                        raise ArgumentError("batch", f"unknown host buffer {key!r}")
                    dt, num, least = want[key]
                    check_buffer("batch", f"host {key}", t, dt, numel=num, min_numel=least,
                                 pinned=True)
        plans = [it[0].handle for it in items]
        if host is None:
            st, h = atsfft_batch_create(plans, [it[1] for it in items], [it[2] for it in items],
                                        [it[3] for it in items], [it[2].numel() for it in items],
                                        [it[4] for it in items], [it[5] for it in items],
                                        [it[6] for it in items])
        else:
            self._keep_host = list(host)
            get = lambda key: [hd.get(key) for hd in host]
            st, h = atsfft_batch_create_io(plans, get("x"), [it[1] for it in items],
                                           [it[2] for it in items], [it[3] for it in items],
                                           [it[2].numel() for it in items],
                                           [it[4] for it in items], [it[5] for it in items],
                                           [it[6] for it in items], get("loc"), get("val"),
                                           get("count"), get("k"), get("status"))
        if st != OK:
            raise ATSFFTError(st, "atsfft_batch_create")
        self.handle = h
        self._torch = torch

    def launch(self, stream=None):
        s = stream if stream is not None else self._torch.cuda.current_stream().cuda_stream
        st = atsfft_batch_launch(self.handle, s)
        if st != OK:
            raise ATSFFTError(st, "atsfft_batch_launch")

    def kernels(self) -> int:
        st, k = atsfft_batch_kernels(self.handle)
        if st != OK:
            raise ATSFFTError(st, "atsfft_batch_kernels")
        return k

    def close(self):
        if getattr(self, "handle", None):
            atsfft_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sparse_fft(x, plan: "Plan", capacity: int | None = None):
    """Differentiable 1D ATSFFT: returns (loc, val) with val differentiable in x.

    The support (loc) and the median's hash selections are fixed by the forward pass;
    the gradient flows through Eq. (11), the bucket DFTs, the binning and the window at
    that support (atsfft_estimate_adjoint)."""
    return _SparseFFT.apply(x, plan, capacity)


def _sparse_fft_class():
    import torch

    class SparseFFT(torch.autograd.Function):
        @staticmethod
        def forward(ctx, x, plan, capacity):
            loc, val, msel, B, _, _, _ = plan.exec_sel(x.detach().contiguous(), capacity)
            ctx.plan, ctx.B = plan, B
            ctx.save_for_backward(loc, msel)
            ctx.mark_non_differentiable(loc)
            return loc, val.clone()

        @staticmethod
        def backward(ctx, g_loc, g_val):
            loc, msel = ctx.saved_tensors
            if g_val is None:
                return None, None, None
            gx = ctx.plan.estimate_adjoint(ctx.B, loc, msel, g_val.to(torch.complex64))
            return gx, None, None

    return SparseFFT


class _Lazy:
    """Creates the autograd Function on first use (torch is imported lazily)."""

    def __init__(self, make):
        self._make, self._cls = make, None

    def apply(self, *args):
        if self._cls is None:
            self._cls = self._make()
        return self._cls.apply(*args)


_SparseFFT = _Lazy(_sparse_fft_class)
