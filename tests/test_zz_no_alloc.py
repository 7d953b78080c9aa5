"""The allocation-free bucket-spectrum call agrees with the plan-based one.  Needs a GPU.

atsfft_hash_spectrum_noalloc serves callers that cannot allocate device memory when they
need a hash's bucket spectrum (see include/atsfft.h): its scratch is a fixed array in the
library instead of a plan.  This file is collected last so that a run stopping at the
first failure has already run every other test; it also passes on its own in a fresh
process.  Tolerance: the bucket-spectrum bound used by the other GPU tests,
max |difference| <= 2e-5 * max |reference|.
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
def test_noalloc_matches_plan_twice(A, n, B, phase, index):
    import torch

    from synth import sparse_signal_1d

    seed = 5
    sig = sparse_signal_1d(n, 40, 9, snr_db=40)
    x = torch.from_numpy(sig.x).cuda()
    plan = A.Plan((n,), seed=seed)
    ref = plan.hash_spectrum(x, B, phase, index).cpu().numpy()
    plan.close()
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):   # two calls in a row share and reuse the fixed scratch
        out = torch.full((B,), float("nan"), dtype=torch.complex64, device="cuda")
        st = A.atsfft_hash_spectrum_noalloc(x, n, B, seed, phase, index, out, stream)
        assert st == A.OK, A.atsfft_status_string(st)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.max(np.abs(got - ref)) <= 2e-5 * np.max(np.abs(ref))


def test_noalloc_rejects_sizes_beyond_its_scratch(A):
    import torch

    x = torch.zeros(16, dtype=torch.complex64, device="cuda")
    z = torch.zeros(16, dtype=torch.complex64, device="cuda")
    assert A.atsfft_hash_spectrum_noalloc(x, 1 << 23, 1 << 16, 0, 1, 0, z) == A.E_INVALID_ARG
    assert A.atsfft_hash_spectrum_noalloc(x, 1 << 14, 1 << 11, 0, 1, 0, z) == A.E_INVALID_ARG
    assert A.atsfft_hash_spectrum_noalloc(x, 1 << 14, 8, 0, 1, 0, z) == A.E_INVALID_ARG
    assert A.atsfft_hash_spectrum_noalloc(x, 1000, 16, 0, 1, 0, z) == A.E_INVALID_ARG
