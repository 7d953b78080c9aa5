"""Parameter autotuner for a workload of 1D signals (length n, sparsity in a range, noise
level): times candidate parameter sets on synthetic probe signals with a known sparse
spectrum and keeps the fastest whose accuracy meets a target.

The candidates vary what trades speed for robustness -- location and estimation loop
counts, the window tolerance and the window's transition width alpha (together they set
the window support, Eqs. (8)-(9)), the range of bucket counts the tuning walks (Eq. (14):
a smallest B sized to the smallest expected k skips trials that cannot hold it, a largest
B sized to the largest k skips the widest windows) -- and the launch knobs that do not
change results (tuning stages).  Accuracy is measured with Eq. (15) (the L1 error
per true coefficient over the whole grid) and the detected k* against the true k; the
transform itself always runs on the GPU through the C ABI.
"""

from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field

import numpy as np

DEFAULT_GRID = {
    "loops": [(7, 7), (5, 5)],
    "filter_tol": [1e-6, 1e-5],
    "filter_alpha": [0.5, 1.0],
    "b_range": ["default", "k_range"],
    "tune_stages": [3, 2],
}


def b_range_for(n: int, k_range, which: str):
    """(b_min_log2, b_max_log2) of a candidate: "default" keeps the plan's range
    ([4, log2 n - 4]); "k_range" starts at the smallest B >= 2 k_lo (the k-hint rule of
    Algorithm 2's initial B) and ends at the smallest B >= 128 k_hi (the walk stops near
    64 k: one doubling of room), both clamped to the default range."""
    logn = n.bit_length() - 1
    lo_d, hi_d = 4, logn - 4
    if which == "default":
        return 0, 0
    lo = max(lo_d, math.ceil(math.log2(2 * k_range[0])))
    hi = min(hi_d, max(lo + 1, math.ceil(math.log2(128 * k_range[1]))))
    return (lo if lo != lo_d else 0), (hi if hi != hi_d else 0)


@dataclass
class TuneResult:
    params: dict                      # the chosen overrides for paper_1908_02461_gb300.params
    ms_per_transform: float
    error: float                      # mean Eq. (15) error per coefficient on the probes
    k_ratio: float                    # median k* / k on the probes
    table: list = field(default_factory=list)   # (overrides, ms, error, k_ratio, ok) per candidate


def _probe(n, k, snr_db, rng):
    """x = IDFT of a k-sparse spectrum (unit magnitudes, uniform phases) + complex noise."""
    loc = np.sort(rng.choice(n, size=k, replace=False))
    coef = np.exp(2j * np.pi * rng.uniform(size=k))
    spec = np.zeros(n, complex)
    spec[loc] = coef
    x = np.fft.ifft(spec)
    if snr_db is not None:
        sd = math.sqrt(np.mean(np.abs(x) ** 2) * 10 ** (-snr_db / 10) / 2)
        x = x + sd * (rng.standard_normal(n) + 1j * rng.standard_normal(n))
    return x.astype(np.complex64), loc, coef


def _l1_error(loc, coef, got_loc, got_val):
    truth = dict(zip(loc.tolist(), coef.tolist()))
    err = 0.0
    for i, v in zip(got_loc.tolist(), got_val.tolist()):
        err += abs(v - truth.pop(i, 0.0))
    err += sum(abs(v) for v in truth.values())
    return err / len(loc)


def autotune(n: int, k_range=(10, 1000), snr_db: float | None = 40.0, error_target: float = 1e-2,
             probes: int = 4, reps: int = 3, seed: int = 0, grid: dict | None = None,
             capacity: int = 1 << 14) -> TuneResult:
    """Chooses plan parameters for 1D signals of length n with k in k_range."""
    import torch

    from . import Plan, params

    grid = grid or DEFAULT_GRID
    rng = np.random.default_rng(seed)
    # probe sparsities spread log-uniformly over the range, at most n / 64 (beyond it the
    # largest B = n / 16 leaves fewer than 4 buckets per coefficient)
    lo, hi = k_range
    hi = max(lo, min(hi, n // 64))
    ks = sorted({int(round(math.exp(u))) for u in np.linspace(math.log(lo), math.log(hi), probes)})
    sigs = [_probe(n, k, snr_db, rng) for k in ks]
    xs = [torch.from_numpy(x).cuda() for x, _, _ in sigs]
    table = []
    best = None
    seen = set()
    for (ll, le), tol, alpha, br, stages in itertools.product(
            grid["loops"], grid["filter_tol"], grid["filter_alpha"],
            grid.get("b_range", ["default"]), grid["tune_stages"]):
        b_lo, b_hi = b_range_for(n, k_range, br)
        over = dict(loops_loc=ll, loops_est=le, filter_tol=tol, filter_alpha=alpha,
                    b_min_log2=b_lo, b_max_log2=b_hi, tune_stages=stages)
        key = tuple(sorted(over.items()))
        if key in seen:   # a k-derived range equal to the default one
            continue
        seen.add(key)
        plan = Plan((n,), params=params(**over), seed=seed)
        errs, ratios = [], []
        for (x, loc, coef), xd, k in zip(sigs, xs, ks):
            # every status is a result (NOT_SPARSE / NOT_CONVERGED / CAPACITY still return
            # locations and values); Eq. (15) scores it
            gl, gv, kk, st, cnt = plan(xd, capacity=capacity)
            errs.append(_l1_error(loc, coef, gl.cpu().numpy(), gv.cpu().numpy().astype(complex)))
            ratios.append(kk / k)
        # time: every probe once per rep, after one warm-up round
        out = [dict(loc=torch.empty(capacity, dtype=torch.int64, device="cuda"),
                    val=torch.empty(capacity, dtype=torch.complex64, device="cuda"),
                    c=torch.zeros(1, dtype=torch.int64, device="cuda"),
                    k=torch.zeros(1, dtype=torch.int64, device="cuda"),
                    s=torch.zeros(1, dtype=torch.int32, device="cuda")) for _ in xs]
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for r in range(reps + 1):
            if r == 1:
                ev0.record()
            for xd, o in zip(xs, out):
                plan.exec_async(xd, o["loc"], o["val"], o["c"], o["k"], o["s"])
        ev1.record()
        ev1.synchronize()
        ms = ev0.elapsed_time(ev1) / (reps * len(xs))
        plan.close()
        err, ratio = float(np.mean(errs)), float(np.median(ratios))
        ok = err <= error_target and 0.9 <= ratio <= 1.1
        table.append((over, ms, err, ratio, ok))
        if ok and (best is None or ms < best[1]):
            best = (over, ms, err, ratio)
    if best is None:   # nothing met the target: the most accurate candidate
        over, ms, err, ratio, _ = min(table, key=lambda r: r[2])
        best = (over, ms, err, ratio)
    return TuneResult(params=best[0], ms_per_transform=best[1], error=best[2], k_ratio=best[3],
                      table=table)
