"""Checks the oracle's stored result for n = 2^28 (tests/golden/oracle_1d_n2p28_k100.json)
against what the paper and the mathematics fix, without rerunning the oracle:

* the trial trace follows Algorithm 2 with Eqs. (12)-(14) as read here: B doubles from
  the smallest trial, every trial before the last has r = |1 - k_t / k_(t-1)| >= delta2
  (or a zero count), the last has r < delta2, and B*, k* are the last trial's;
* every location of the exact spectrum's support is kept (Section III-B: a support
  coefficient lies in a selected bucket of every location hash when nothing collides);
* the kept list is ascending, distinct, within the capacity;
* the number of kept coordinates outside the support matches the vote rule's
  expectation n P(Bin(L, p) >= ceil(L / 2)), p = k* / B* (each location hash selects
  k* of its B* buckets), within 10% (about five standard deviations here)."""

import json
import math
import os

import numpy as np

from synth import sparse_spectrum_1d

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                      "oracle_1d_n2p28_k100.json")
DELTA2 = 0.05          # Eq. (14): delta2 = 5%
L_LOC = 7


def _golden():
    with open(GOLDEN) as f:
        return json.load(f)


def test_trace_follows_the_controller():
    g = _golden()
    tr = g["trials_B_k"]
    assert tr[0][0] == 16
    for (b0, _), (b1, _) in zip(tr, tr[1:]):
        assert b1 == 2 * b0
    def r(prev, cur):
        return math.inf if prev == 0 or cur == 0 else abs(1.0 - cur / prev)
    for t in range(1, len(tr) - 1):
        assert r(tr[t - 1][1], tr[t][1]) >= DELTA2
    assert r(tr[-2][1], tr[-1][1]) < DELTA2
    assert (g["B_star"], g["k_star"]) == tuple(tr[-1])
    assert g["status"] == 0


def test_support_kept_and_list_well_formed():
    g = _golden()
    n = 1 << g["logn"]
    support, _ = sparse_spectrum_1d(n, g["k"], g["signal_seed"])
    loc = np.asarray(g["loc"], dtype=np.int64)
    assert len(loc) == g["count"] <= g["capacity"]
    assert (np.diff(loc) > 0).all() and loc[0] >= 0 and loc[-1] < n
    assert np.isin(support, loc).all()
    assert int((~np.isin(loc, support)).sum()) == g["outside_support"]


def test_outside_count_matches_the_vote_rule():
    g = _golden()
    n = 1 << g["logn"]
    p = g["k_star"] / g["B_star"]
    need = (L_LOC + 1) // 2
    prob = sum(math.comb(L_LOC, j) * p ** j * (1 - p) ** (L_LOC - j) for j in range(need, L_LOC + 1))
    expect = (n - g["k"]) * prob
    assert abs(g["outside_support"] - expect) < 0.1 * expect, (g["outside_support"], expect)
