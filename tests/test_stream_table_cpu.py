"""Host check of the residue-stream binning's table indexing (CPU): for every window the
stream form can take (n = 2^8 .. 2^28), every thread offset rho of t' mod B and every
row index Q = t' >> log2 B, the entry index v (D + 2) + 1 - kappa' + Q stays inside the
two tables of 2 (D + 2) entries, and entry E_v[i] is nonzero exactly when the tap is in
the window (t' <= 2h), with R_u taken at u = floor((t' - h) / B).  This restates the
index arithmetic the kernel uses (window test folded into the table) and checks it
against the direct definition of the window and of u."""

import numpy as np

import bench


def _table_entry_in_window(i, v, H):
    # E_v[i] is R_u for u = i - (H + 1) <= H - 1 + v, zero beyond
    u = i - (H + 1)
    return u <= H - 1 + v, u


def test_stream_table_indexing_covers_the_window_exactly():
    rng = np.random.default_rng(0)
    for logn in range(8, 29):
        n = 1 << logn
        for logB in range(4, logn - 4 + 1):
            B = 1 << logB
            if not bench._stream(n, B):
                continue
            h = bench._window_h(n, B)
            D = n // B
            H = h >> logB
            hr = h & (B - 1)
            rhos = np.unique(np.concatenate([np.arange(min(B, 64)),
                                             rng.integers(0, B, size=64), [B - 1]]))
            for rho in rhos.tolist():
                k1 = 1 if rho < hr else 0
                delta = (B if k1 else 0) + rho - hr
                v = ((h - delta) >> logB) - (H - 1)
                assert v in (0, 1)
                base = v * (D + 2) + 1 - k1
                Qs = np.unique(np.concatenate([np.arange(min(D, 64)), [D - 1],
                                               rng.integers(0, D, size=64)]))
                for Q in Qs.tolist():
                    e = base + Q
                    assert 0 <= e < 2 * (D + 2), (logn, logB, rho, Q)
                    i = e - v * (D + 2)
                    inside, u = _table_entry_in_window(i, v, H)
                    tprime = Q * B + rho
                    assert inside == (tprime <= 2 * h), (logn, logB, rho, Q)
                    # the rotation index: u = floor((t' - h) / B)
                    assert u == (tprime - h) // B, (logn, logB, rho, Q)
