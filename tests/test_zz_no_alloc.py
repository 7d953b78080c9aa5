"""The allocation-free bucket-spectrum call agrees with the plan-based one and with the
oracle.  Needs a GPU.

atsfft_hash_spectrum_noalloc serves callers that cannot allocate device memory when they
need a hash's bucket spectrum (see include/atsfft.h): its scratch is a fixed array in the
library instead of a plan.  This file is collected last so that a run stopping at the
first failure has already run every other test; it also passes on its own in a fresh
process.  Tolerance: the bucket-spectrum bound used by the other GPU tests,
max |difference| <= 2e-5 * max |reference|, against the plan-based entry point and
against the FP64 oracle's spectrum of the same hash.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def A():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1908_02461_gb300 as A

    A.build()
    return A


@pytest.mark.parametrize("n,B,phase,index", [(1 << 14, 512, 1, 2), (1 << 22, 65536, 2, 3),
                                             (1 << 22, 4096, 0, 12)])
def test_noalloc_matches_plan_and_oracle_twice(A, n, B, phase, index):
    import torch

    import oracle as O
    from synth import sparse_signal_1d

    seed = 5
    sig = sparse_signal_1d(n, 40, 9, snr_db=40)
    x = torch.from_numpy(sig.x).cuda()
    plan = A.Plan((n,), seed=seed)
    ref = plan.hash_spectrum(x, B, phase, index).cpu().numpy()
    plan.close()
    exact = O.hash_spectrum_1d(sig.x, B, seed, phase, index)
    assert np.max(np.abs(ref - exact)) <= 2e-5 * np.max(np.abs(exact))
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):   # two calls in a row share and reuse the fixed scratch
        out = torch.full((B,), float("nan"), dtype=torch.complex64, device="cuda")
        st = A.atsfft_hash_spectrum_noalloc(x, n, B, seed, phase, index, out, stream)
        assert st == A.OK, A.atsfft_status_string(st)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.max(np.abs(got - ref)) <= 2e-5 * np.max(np.abs(ref))
        assert np.max(np.abs(got - exact)) <= 2e-5 * np.max(np.abs(exact))


def test_noalloc_rejects_sizes_beyond_its_scratch(A):
    """The C entry point refuses sizes beyond its fixed array before any launch; the
    buffers passed are of the full size, so nothing could be read out of bounds even if
    it did not."""
    import torch

    from paper_1908_02461_gb300 import _lib

    def bufs(n, B):
        return (torch.zeros(n, dtype=torch.complex64, device="cuda"),
                torch.zeros(B, dtype=torch.complex64, device="cuda"))

    x, z = bufs(1 << 23, 1 << 16)
    assert _lib.atsfft_hash_spectrum_noalloc(x, 1 << 23, 1 << 16, 0, 1, 0, z) == A.E_INVALID_ARG
    x, z = bufs(1 << 14, 1 << 11)
    assert _lib.atsfft_hash_spectrum_noalloc(x, 1 << 14, 1 << 11, 0, 1, 0, z) == A.E_INVALID_ARG
    x, z = bufs(1 << 14, 8)
    assert _lib.atsfft_hash_spectrum_noalloc(x, 1 << 14, 8, 0, 1, 0, z) == A.E_INVALID_ARG
    x, z = bufs(1000, 16)
    assert _lib.atsfft_hash_spectrum_noalloc(x, 1000, 16, 0, 1, 0, z) == A.E_INVALID_ARG
    # the checked wrapper refuses buffers that do not hold n and B values
    x, z = bufs(1 << 14, 256)
    with pytest.raises(A.ArgumentError):
        A.atsfft_hash_spectrum_noalloc(x[:100], 1 << 14, 256, 0, 1, 0, z)
    with pytest.raises(A.ArgumentError):
        A.atsfft_hash_spectrum_noalloc(x, 1 << 14, 512, 0, 1, 0, z)
