"""The parity rule of the GPU tests: a CUDA transform against the FP64 oracle.

The two sides must agree exactly -- the tuning trajectory (B and local-maximum count of
every trial, Eqs. (12)-(14)), k*, the status, the count and the set of kept locations --
and the values of the common locations must agree within 1e-4 (relative, or absolute at
1 % of the largest coefficient for noise-level candidates).  The only difference allowed
is one that traces back to a discrete decision the oracle logged as lying within BAND of
its boundary, where FP32 energies can decide otherwise than FP64 ones:

  * a tuning count that differs must belong to a trial with a logged decision, and then
    the walk after it is not compared (every later step depends on that count);
  * a location kept by one side only must lie, in some location hash, in a bucket named
    by a logged decision of that hash (its threshold, tie band or cutoff-band test, or a
    bucket whose selection a logged local-maximum flip would move).

Nothing else is tolerated: a dropped location or a k* off by one with no logged decision
behind it fails.
"""

from __future__ import annotations

import numpy as np

import oracle as O

BAND = 2e-4   # ~1000x the FP32 rounding of an energy
VALUE_TOL = 1e-4


def value_error(v_gpu, v_ref):
    """max |v_gpu - v_ref| / max(|v_ref|, max|v_ref| / 100)."""
    if len(v_ref) == 0:
        return 0.0
    scale = max(np.max(np.abs(v_ref)) / 100.0, 1e-30)
    return float((np.abs(v_gpu - v_ref) / np.maximum(np.abs(v_ref), scale)).max())


def _log2(v: int) -> int:
    return int(v).bit_length() - 1


def bucket_in_hash(coord: int, l: int, seed: int, shape, B: int) -> int:
    """The bucket of a location (linear index in 2D) in location hash l at B per axis."""
    n = shape[0]
    if len(shape) == 1:
        sigma, _ = O.hash_params(seed, 1, l, n, 1)
        return O.bucket_of(coord, sigma, n, B)
    s1, _, s2, _ = O.hash_params(seed, 1, l, n, 2)
    i, j = divmod(int(coord), n)
    return O.bucket_of(i, s1, n, B) * B + O.bucket_of(j, s2, n, B)


def check(gpu: dict, ref, decisions, shape, seed: int, loops_loc: int = 7,
          capacity: int | None = None) -> dict:
    """Asserts the parity rule.  gpu: trace [(B, k)], k, status, count, loc, val (numpy).
    Returns a summary dict ('exact' when the two agree in every discrete output)."""
    ref_trace = [(int(b), int(k)) for b, k, _ in ref.trials]
    trace = [(int(b), int(k)) for b, k in gpu["trace"]]
    info = dict(k=(gpu["k"], ref.k_star), count=(gpu["count"], ref.count),
                status=(gpu["status"], ref.status), margin=ref.min_margin,
                near=len(decisions))
    if trace != ref_trace:
        t = next(i for i in range(min(len(trace), len(ref_trace)) + 1)
                 if i >= len(trace) or i >= len(ref_trace) or trace[i] != ref_trace[i])
        assert t < len(trace) and t < len(ref_trace), ("trajectories end apart", trace, ref_trace)
        assert trace[t][0] == ref_trace[t][0], ("trial B differs", trace, ref_trace)
        b = _log2(trace[t][0])
        near = [d for d in decisions if d.phase == 0 and d.hash == b]
        assert near, ("tuning count differs with no near decision in that trial",
                      t, trace, ref_trace, info)
        # the GPU's own walk still follows Eq. (14) on its own counts: B doubles while
        # r >= delta2, and it stops at the first trial below
        for i in range(1, len(trace)):
            assert trace[i][0] == 2 * trace[i - 1][0], ("walk does not double", trace)
            if i < len(trace) - 1:
                assert O.controller_branch(trace[i - 1][1], trace[i][1]) == 1, ("walk", trace)
        info.update(attributed="tuning", trial=t, decisions=near)
        return info
    assert gpu["k"] == ref.k_star, info
    loc, rloc = np.asarray(gpu["loc"]), np.asarray(ref.loc)
    cap = capacity if capacity is not None else max(len(loc), len(rloc))
    if gpu["count"] > cap or ref.count > cap:
        # truncated outputs: the sets are only known below the smaller largest location
        lim = min(loc.max() if len(loc) else -1, rloc.max() if len(rloc) else -1)
        gl, rl = loc[loc <= lim], rloc[rloc <= lim]
    else:
        gl, rl = loc, rloc
    only_gpu = np.setdiff1d(gl, rl)
    only_ref = np.setdiff1d(rl, gl)
    diff = np.concatenate([only_gpu, only_ref])
    if len(diff):
        B = trace[-1][0] if trace else int(ref.B_star)
        affected = {}
        for d in decisions:
            if d.phase == 1:
                affected.setdefault(d.hash, set()).update(c for c in (d.c, d.m) if c >= 0)
        for coord in diff.tolist():
            ok = any(bucket_in_hash(coord, l, seed, shape, B) in affected.get(l, ())
                     for l in range(loops_loc))
            assert ok, ("location differs with no near decision behind it", coord, info)
        info.update(attributed="location", only_gpu=only_gpu.tolist(), only_ref=only_ref.tolist())
        if gpu["count"] <= cap and ref.count <= cap:
            assert gpu["count"] - ref.count == len(only_gpu) - len(only_ref), info
        if (gpu["count"] > cap) == (ref.count > cap):
            assert gpu["status"] == ref.status, info
    else:
        assert gpu["count"] == ref.count, info
        st_g, st_r = gpu["status"], ref.status
        assert st_g == st_r, info
        assert loc.tolist() == rloc.tolist(), info
    common, ig, ir = np.intersect1d(loc, rloc, return_indices=True)
    err = value_error(np.asarray(gpu["val"])[ig], np.asarray(ref.val)[ir])
    info["value_err"] = err
    assert err <= VALUE_TOL, info
    if not len(diff):
        info["exact"] = True
    return info
