"""The largest 1D sizes, where sample indices no longer fit the 2^23 exponent trick of
the binning: n = 2^26 against the oracle run here (about half a minute of CPU time), and
the maximum n = 2^28 against the oracle's stored result (tests/golden/
oracle_1d_n2p28_k100.json, written by tests/golden/make_oracle_large.py: the oracle needs
minutes there) and against the exact spectrum.  At these sizes the vote rule keeps
coordinates outside the support (about n C(7,4) (k/B*)^4 of them; the oracle keeps the
same ones), whose estimates are zero to FP32 accuracy.  Needs a GPU."""

import json
import os

import numpy as np
import pytest

from _parity import BAND, check
from synth import sparse_signal_1d

pytestmark = pytest.mark.gpu

GOLDEN_28 = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                         "oracle_1d_n2p28_k100.json")


@pytest.fixture(scope="module")
def A():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1908_02461_gb300 as A

    A.build()
    return A


def _on_device(sig):
    import torch

    return torch.from_numpy(sig.x).cuda()


def test_n_2_26_matches_oracle(A):
    import oracle as O

    O.build()
    sig = sparse_signal_1d(1 << 26, 300, 26)
    plan = A.Plan((1 << 26,), seed=3)
    loc, val, kk, st, cnt = plan(_on_device(sig), capacity=1 << 12)
    trace = plan.last_trace()
    plan.close()
    loc = loc.cpu().numpy()
    val = val.cpu().numpy()
    ref, dec = O.atsfft_log(sig.x, seed=3, capacity=1 << 12, band=BAND)
    gpu = dict(trace=trace, k=kk, status=st, count=cnt, loc=loc, val=val)
    info = check(gpu, ref, dec, (1 << 26,), 3, capacity=1 << 12)
    print(f"[large] n=2^26 {info}")
    assert np.isin(sig.support, loc).all()


def test_maximum_n_2_28_matches_stored_oracle(A):
    with open(GOLDEN_28) as f:
        g = json.load(f)
    sig = sparse_signal_1d(1 << g["logn"], g["k"], g["signal_seed"])
    plan = A.Plan((1 << g["logn"],), seed=g["plan_seed"])
    loc, val, kk, st, cnt = plan(_on_device(sig), capacity=g["capacity"])
    trace = plan.last_trace()
    plan.close()
    loc = loc.cpu().numpy()
    val = val.cpu().numpy()
    print(f"[large] n=2^28 k*={kk} count={cnt} status={st} (oracle: k*={g['k_star']} "
          f"count={g['count']})")
    # the stored run is far from every decision boundary (relative margin ~2e-3 against
    # FP32 rounding of ~1e-6), so the trajectory and the kept set are the oracle's
    assert g["min_margin"] > 2e-4
    assert st == g["status"] == A.OK
    assert [list(t) for t in trace] == g["trials_B_k"]
    assert kk == g["k_star"] and cnt == g["count"]
    assert loc.tolist() == g["loc"]
    # values against the exact spectrum: support coefficients to FP32 accuracy, the
    # coordinates outside the support near zero (no estimation bucket of theirs holds a
    # support coefficient in a majority of the hashes: the oracle's are below 1e-8)
    assert g["max_abs_outside"] < 1e-6
    on = np.isin(loc, sig.support)
    assert on.sum() == len(sig.support)
    cs = sig.coeffs[np.searchsorted(sig.support, loc[on])]
    assert float(np.abs(val[on] - cs).max()) < 2e-3
    assert float(np.abs(val[~on]).max()) < 1e-3
