"""The column form of the location binning (k_bin_cols): its decomposition of a hash's
window taps, checked against brute force on the CPU.

For a hash (sigma odd, tau) at B = n / D buckets, the form claims:
  * the samples of bucket b all lie in residue column r = (sigma b + tau) mod B;
  * bucket b's taps t = b + u B, u_lo <= u <= u_hi, reach rows j0 + (u - u_lo) sigma
    (mod D) of that column, j0 the row of the first tap;
  * the tiles (1024 samples: 1024 / D whole columns), the lanes of a warp (2^logLC
    columns side by side, lpc lanes per column dealing out the hashes) and the column
    slots of a lane visit every column of every hash exactly once.
Together: every (tap, sample) pair of the window with t mod B != 0 is visited exactly
once (bucket 0 takes only the centre tap, Section II-A-2: sin(pi t / B) vanishes on the
other taps of bucket 0).  The brute force is the window's definition: all |t| <= h with
sample a = (sigma t + tau) mod n.
"""

import random

import pytest

TILE_LOG = 10          # samples per warp tile: 2^10
MAX_LOG_D = 8          # the form takes D = n / B <= 256


def _visits(n, B, sigma, tau, h, nh_lanes=14):
    """(t, a) pairs the column form visits for one hash, plus the (column, hash) units."""
    logn, logB = n.bit_length() - 1, B.bit_length() - 1
    logD = logn - logB
    logTC = TILE_LOG - logD
    logLC = min(logTC, 5)
    lpc = 32 >> logLC
    cps = 1 << (logTC - logLC)
    sinv = pow(sigma, -1, 1 << 32)
    mask, Bm, Dm = n - 1, B - 1, (1 << logD) - 1
    pairs, units = [], []
    for tl in range(n >> TILE_LOG):
        col0 = tl << logTC
        for lane in range(32):
            cl, sub = lane & ((1 << logLC) - 1), lane >> logLC
            for sl in range(cps):
                c = cl + (sl << logLC)
                r = col0 + c
                # the kernel deals hashes g = sub, sub + lpc, ... to this lane; one hash
                # here, owned by the lanes with sub == 0
                for g in range(sub, nh_lanes, lpc):
                    if g != 0:
                        continue
                    units.append(r)
                    b = (sinv * ((r - tau) & 0xFFFFFFFF)) & Bm
                    if b == 0:
                        continue
                    u_lo, u_hi = -((h + b) >> logB), (h - b) >> logB
                    t0 = b + u_lo * B
                    j = (((sigma * t0 + tau) & 0xFFFFFFFF) & mask) >> logB
                    for u in range(u_lo, u_hi + 1):
                        t = b + u * B
                        pairs.append((t, r + (j << logB)))
                        j = (j + (sigma & Dm)) & Dm
    return pairs, units


@pytest.mark.parametrize("logn,logD", [(10, 4), (10, 5), (10, 6), (12, 4), (12, 5), (12, 6),
                                       (12, 7), (12, 8), (14, 6)])
def test_column_form_visits_every_window_pair_once(logn, logD):
    rng = random.Random(1000 * logn + logD)
    n, D = 1 << logn, 1 << logD
    B = n // D
    for _ in range(3):
        sigma = rng.randrange(n) | 1
        tau = rng.randrange(n)
        # a window inside the circle and one clamped to it (h = n/2 - 1)
        for h in (rng.randrange(B, n // 2 - 1), n // 2 - 1):
            pairs, units = _visits(n, B, sigma, tau, h)
            # every column of the hash exactly once
            assert sorted(units) == list(range(B))
            # every in-window (tap, sample) pair outside bucket 0 exactly once
            want = sorted((t, (sigma * t + tau) % n) for t in range(-h, h + 1) if t % B != 0)
            assert sorted(pairs) == want


def test_column_form_lane_mapping_shapes():
    """Lanes per column and columns per lane multiply to the tile's columns at every D."""
    for logD in range(4, MAX_LOG_D + 1):
        logTC = TILE_LOG - logD
        logLC = min(logTC, 5)
        lpc, cps = 32 >> logLC, 1 << (logTC - logLC)
        assert (32 // lpc) * cps == 1 << logTC
        assert lpc * (1 << logLC) == 32
