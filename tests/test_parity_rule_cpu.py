"""The GPU parity rule (tests/_parity.py) itself, on the CPU: a result equal to the
oracle's passes as exact; a difference behind a decision the oracle logged near its
boundary passes as attributed; a dropped or added location, a shifted count or k*, or a
value error with no logged decision behind it fails.  The "GPU" results here are the
oracle's own outputs with one planted difference each."""

import numpy as np
import pytest

import oracle as O
from _parity import BAND, bucket_in_hash, check
from synth import sparse_signal_1d, sparse_signal_2d


def _as_gpu(ref):
    return dict(trace=[(b, k) for b, k, _ in ref.trials], k=ref.k_star, status=ref.status,
                count=ref.count, loc=ref.loc.copy(), val=ref.val.astype(np.complex64))


@pytest.fixture(scope="module")
def near_case():
    """n = 2^14, k = 16, plan seed 7: one location hash holds a near dominance decision
    (the oracle logs it with the buckets its flip would move)."""
    sig = sparse_signal_1d(1 << 14, 16, 0)
    ref, dec = O.atsfft_log(sig.x, seed=7, band=BAND)
    assert any(d.phase == 1 for d in dec)
    return sig, ref, dec


def test_identical_result_is_exact(near_case):
    sig, ref, dec = near_case
    info = check(_as_gpu(ref), ref, dec, sig.x.shape, 7)
    assert info.get("exact")


def _free_and_near_locations(ref, dec, shape, seed):
    B = ref.trials[-1][0]
    touched = {}
    for d in dec:
        if d.phase == 1:
            touched.setdefault(d.hash, set()).update(c for c in (d.c, d.m) if c >= 0)
    near, free = [], []
    for i in ref.loc.tolist():
        hit = any(bucket_in_hash(i, l, seed, shape, B) in touched.get(l, ()) for l in range(7))
        (near if hit else free).append(i)
    return near, free


def test_dropped_location_without_a_near_decision_fails(near_case):
    sig, ref, dec = near_case
    _, free = _free_and_near_locations(ref, dec, sig.x.shape, 7)
    g = _as_gpu(ref)
    keep = g["loc"] != free[0]
    g.update(loc=g["loc"][keep], val=g["val"][keep], count=g["count"] - 1)
    with pytest.raises(AssertionError, match="no near decision"):
        check(g, ref, dec, sig.x.shape, 7)


def test_added_location_without_a_near_decision_fails(near_case):
    sig, ref, dec = near_case
    B = ref.trials[-1][0]
    touched = {d.hash: {d.c, d.m} for d in dec if d.phase == 1}
    extra = next(i for i in range(sig.x.size) if i not in set(ref.loc.tolist()) and not any(
        bucket_in_hash(i, l, 7, sig.x.shape, B) in touched.get(l, ()) for l in range(7)))
    g = _as_gpu(ref)
    pos = np.searchsorted(g["loc"], extra)
    g.update(loc=np.insert(g["loc"], pos, extra), val=np.insert(g["val"], pos, 0),
             count=g["count"] + 1)
    with pytest.raises(AssertionError, match="no near decision"):
        check(g, ref, dec, sig.x.shape, 7)


def test_difference_behind_a_near_decision_is_attributed(near_case):
    sig, ref, dec = near_case
    near, _ = _free_and_near_locations(ref, dec, sig.x.shape, 7)
    assert near
    g = _as_gpu(ref)
    keep = g["loc"] != near[0]
    g.update(loc=g["loc"][keep], val=g["val"][keep], count=g["count"] - 1)
    info = check(g, ref, dec, sig.x.shape, 7)
    assert info["attributed"] == "location" and info["only_ref"] == [near[0]]


def test_count_that_disagrees_with_the_set_fails(near_case):
    sig, ref, dec = near_case
    g = _as_gpu(ref)
    g["count"] += 1
    with pytest.raises(AssertionError):
        check(g, ref, dec, sig.x.shape, 7)


def test_tuning_count_off_by_one_needs_a_near_decision_in_that_trial():
    sig = sparse_signal_1d(1 << 16, 50, 1, snr_db=40)
    ref, dec = O.atsfft_log(sig.x, seed=1, band=BAND)
    assert not [d for d in dec if d.phase == 0]
    g = _as_gpu(ref)
    g["trace"][-1] = (g["trace"][-1][0], g["trace"][-1][1] + 1)
    g["k"] += 1
    with pytest.raises(AssertionError, match="tuning count differs"):
        check(g, ref, dec, sig.x.shape, 1)
    # the same difference with a logged decision in that trial is attributed
    fake = O.Decision(0, int(g["trace"][-1][0]).bit_length() - 1, "dominance", 1, 2, 1e-5)
    info = check(g, ref, dec + [fake], sig.x.shape, 1)
    assert info["attributed"] == "tuning"


def test_value_error_beyond_the_tolerance_fails(near_case):
    sig, ref, dec = near_case
    g = _as_gpu(ref)
    big = int(np.argmax(np.abs(g["val"])))
    g["val"][big] *= 1 + 2e-4
    with pytest.raises(AssertionError):
        check(g, ref, dec, sig.x.shape, 7)
    g["val"][big] = ref.val[big] * (1 + 5e-5)
    assert check(g, ref, dec, sig.x.shape, 7).get("exact")


def test_2d_buckets_of_a_location_are_per_axis():
    sig = sparse_signal_2d(64, 6, 2, snr_db=30)
    ref, dec = O.atsfft_log(sig.x, seed=2, band=BAND)
    assert check(_as_gpu(ref), ref, dec, sig.x.shape, 2).get("exact")
    B = ref.trials[-1][0]
    s1, _, s2, _ = O.hash_params(2, 1, 3, 64, 2)
    for coord in ref.loc.tolist():
        i, j = divmod(coord, 64)
        assert bucket_in_hash(coord, 3, 2, (64, 64), B) == \
            O.bucket_of(i, s1, 64, B) * B + O.bucket_of(j, s2, 64, B)
