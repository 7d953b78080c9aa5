"""Argument checks of the Python binding, on the CPU: the C ABI takes raw pointers, so the
binding refuses buffers of the wrong element type, size, layout or device before any
library call (ArgumentError, which is both an ATSFFTError with the invalid-argument
status and a ValueError)."""

import pytest

torch = pytest.importorskip("torch")

import paper_1908_02461_gb300 as A  # noqa: E402

CPU = torch.device("cpu")


def _raises(fn, match):
    with pytest.raises(A.ArgumentError, match=match) as ei:
        fn()
    assert isinstance(ei.value, ValueError) and isinstance(ei.value, A.ATSFFTError)
    assert ei.value.status == A.E_INVALID_ARG


def test_accepts_a_matching_buffer():
    A.check_buffer("exec", "loc", torch.zeros(8, dtype=torch.int64), torch.int64, CPU,
                   numel=8)
    A.check_buffer("exec", "val", torch.zeros(9, dtype=torch.complex64), torch.complex64, CPU,
                   min_numel=8)


def test_refuses_wrong_type_layout_size_and_device():
    c = lambda t, **kw: (lambda: A.check_buffer("exec", "loc", t, torch.int64, **kw))
    _raises(c([0, 1], device=CPU), "must be a torch tensor")
    _raises(c(torch.zeros(8, dtype=torch.int32), device=CPU), "must be torch.int64")
    _raises(c(torch.zeros(8, 2, dtype=torch.int64)[:, 0], device=CPU), "contiguous")
    _raises(c(torch.zeros(7, dtype=torch.int64), device=CPU, numel=8), "hold 8 elements")
    _raises(c(torch.zeros(7, dtype=torch.int64), device=CPU, min_numel=8), "at least 8")
    _raises(c(torch.zeros(8, dtype=torch.int64), device=torch.device("cuda", 0)), "must be on")
    _raises(c(torch.zeros(8, dtype=torch.int64), pinned=True), "pinned")


class _FakePlan:
    """Stands in for a Plan in the host-buffer checks of Batch, which run before any
    library call (every case below fails them)."""

    handle = None
    dtype = torch.complex64
    numel = 1 << 10

    def check_exec_buffers(self, what, *bufs):
        pass


def _item(cap=16):
    return (_FakePlan(), torch.zeros(1 << 10, dtype=torch.complex64),
            torch.zeros(cap, dtype=torch.int64), torch.zeros(cap, dtype=torch.complex64),
            torch.zeros(1, dtype=torch.int64), torch.zeros(1, dtype=torch.int64),
            torch.zeros(1, dtype=torch.int32))


def test_batch_refuses_host_buffers_that_do_not_match():
    # (not pinned: the size and type checks come first, so every case fails on them or
    # on the pinning, never reaching the library)
    _raises(lambda: A.Batch([_item()], host=[]), "host dicts")
    _raises(lambda: A.Batch([_item()], host=[dict(y=torch.zeros(1))]), "unknown host buffer")
    _raises(lambda: A.Batch([_item()], host=[dict(x=torch.zeros(512, dtype=torch.complex64))]),
            "hold 1024 elements")
    _raises(lambda: A.Batch([_item()], host=[dict(loc=torch.zeros(8, dtype=torch.int64))]),
            "at least 16")
    _raises(lambda: A.Batch([_item()], host=[dict(status=torch.zeros(1, dtype=torch.int64))]),
            "torch.int32")
    _raises(lambda: A.Batch([_item()], host=[dict(x=torch.zeros(1 << 10, dtype=torch.complex64))]),
            "pinned")


def _cpu_plan(shape, dtype=torch.complex64):
    """A Plan object without a library handle, its buffers checked against the CPU."""
    p = A.Plan.__new__(A.Plan)
    p.shape, p.ndim, p.dtype, p.device, p.handle = tuple(shape), len(shape), dtype, CPU, None
    return p


def _outs(cap, dtype=torch.complex64):
    return (torch.empty(cap, dtype=torch.int64), torch.empty(cap, dtype=dtype),
            torch.zeros(1, dtype=torch.int64), torch.zeros(1, dtype=torch.int64),
            torch.zeros(1, dtype=torch.int32))


def test_the_buffers_the_benchmark_and_tests_pass_are_accepted():
    # 1D and 2D inputs with the output set of the benchmark (capacity 2^14) and the FP64 path
    _cpu_plan((1 << 14,)).check_exec_buffers(
        "exec", torch.zeros(1 << 14, dtype=torch.complex64), *_outs(1 << 14))
    _cpu_plan((256, 256)).check_exec_buffers(
        "exec", torch.zeros(256, 256, dtype=torch.complex64), *_outs(1 << 12))
    _cpu_plan((1 << 14,), torch.complex128).check_exec_buffers(
        "exec", torch.zeros(1 << 14, dtype=torch.complex128), *_outs(16, torch.complex128))
    # a value buffer longer than the location buffer is fine; shorter is not
    loc, val, c, k, s = _outs(16)
    _cpu_plan((1 << 10,)).check_exec_buffers(
        "exec", torch.zeros(1 << 10, dtype=torch.complex64), loc, torch.zeros(32, dtype=torch.complex64), c, k, s)
    _raises(lambda: _cpu_plan((1 << 10,)).check_exec_buffers(
        "exec", torch.zeros(1 << 10, dtype=torch.complex64), loc, val[:8], c, k, s), "at least 16")
    _raises(lambda: _cpu_plan((1 << 10,)).check_exec_buffers(
        "exec", torch.zeros(1 << 11, dtype=torch.complex64), loc, val, c, k, s), "hold 1024")
    _raises(lambda: _cpu_plan((1 << 10,)).check_exec_buffers(
        "exec", torch.zeros(1 << 10, dtype=torch.complex64), loc.int(), val, c, k, s), "torch.int64")


def test_bucket_count_check_takes_python_and_numpy_integers():
    import numpy as np

    assert A._power_of_two(64) and A._power_of_two(np.int64(4096))
    assert not any(A._power_of_two(v) for v in (0, -8, 48, 64.0, "64"))


def test_noalloc_wrapper_refuses_buffers_before_the_library_call():
    """atsfft_hash_spectrum_noalloc takes raw pointers: the package's wrapper checks that
    the input holds n complex64 values and the output at least B, on the current CUDA
    device, before calling it (on this CPU-only host every CPU tensor is refused)."""
    n, B = 1 << 10, 64
    x = torch.zeros(n, dtype=torch.complex64)
    z = torch.zeros(B, dtype=torch.complex64)
    if torch.cuda.is_available():
        pytest.skip("CPU-only check")
    with pytest.raises(A.ArgumentError, match="must be on cuda"):
        A.atsfft_hash_spectrum_noalloc(x, n, B, 0, 1, 0, z)
    with pytest.raises(A.ArgumentError, match="hold 1024 elements"):
        A.atsfft_hash_spectrum_noalloc(x[:100], n, B, 0, 1, 0, z)
    assert A.atsfft_hash_spectrum_noalloc(x, 1000, B, 0, 1, 0, z) == A.E_INVALID_ARG
