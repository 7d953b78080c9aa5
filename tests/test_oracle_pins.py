"""Pins of the FP64 oracle against things other than itself.

Each test checks the oracle against what the paper or the mathematics fixes:
published test vectors, the paper's worked example (Fig. 5 text), library
routines (numpy's FFT), closed forms of the window design, Lemmas 1-2 and the
convolution theorem, brute-force DFTs on tiny inputs, and the exactness of
Eq. (11) on isolated coefficients.  CPU only.
"""

import json
import math
import os

import numpy as np
import pytest
from scipy.special import erf

import oracle as O
from synth import sparse_signal_1d, sparse_signal_2d

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


# --------------------------------------------------------------------------
# Random numbers and modular arithmetic (Def. 1)
# --------------------------------------------------------------------------

def test_splitmix64_published_vectors():
    for v in _gold("splitmix64.json")["vectors"]:
        got = O.splitmix64_stream(v["seed"], len(v["outputs"]))
        assert got == [int(s) for s in v["outputs"]]


@pytest.mark.parametrize("n", [2 ** 8, 2 ** 14, 2 ** 22, 2 ** 31])
def test_inverse_mod_is_inverse(n):
    rng = np.random.default_rng(1)
    for s in rng.integers(0, n, size=200):
        s = int(s) | 1
        inv = O.inv_mod(s, n)
        assert 0 <= inv < n and (s * inv) % n == 1


def test_hash_params_odd_sigma_and_range():
    seen = set()
    for phase in range(3):
        for index in range(20):
            s1, t1, s2, t2 = O.hash_params(99, phase, index, 4096, ndim=2)
            for v in (s1, t1, s2, t2):
                assert 0 <= v < 4096
            assert s1 % 2 == 1 and s2 % 2 == 1
            seen.add((s1, t1))
    assert len(seen) == 60  # every (phase, index) draws its own permutation


# --------------------------------------------------------------------------
# DFT (the paper's unscaled convention, Eq. (1))
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 4, 8, 64, 1024, 4096])
def test_fft_matches_numpy(n):
    rng = np.random.default_rng(n)
    a = rng.normal(size=n) + 1j * rng.normal(size=n)
    assert np.allclose(O.fft(a), np.fft.fft(a), rtol=0, atol=1e-11 * max(1, np.sqrt(n)))


def test_fft_rejects_non_power_of_two():
    with pytest.raises(ValueError):
        O.fft(np.zeros(12))


# --------------------------------------------------------------------------
# Flat window (Section II-A-2): box car of one bucket width convolved with a Gaussian
# --------------------------------------------------------------------------

def _erf_profile(o, D, sf):
    """Continuous box of width D (edges +-D/2) convolved with a unit-area Gaussian of
    standard deviation sf: the closed form the window design approximates."""
    z = math.sqrt(2.0) * sf
    return 0.5 * (erf((D / 2 - o) / z) + erf((D / 2 + o) / z))


@pytest.mark.parametrize("n,B", [(2 ** 12, 64), (2 ** 14, 256), (2 ** 16, 512), (2 ** 14, 1024)])
def test_window_response_matches_box_conv_gaussian(n, B):
    h, s, taps = O.filter_taps(n, B)
    assert taps.shape == (2 * h + 1,)
    assert np.allclose(taps, taps[::-1])                 # real, symmetric
    assert abs(taps.sum() - n) < 1e-9 * n                # Ghat'(0) = 1 normalisation
    D = n // B
    sf = n / (2 * math.pi * s)                          # frequency-domain std of the Gaussian
    resp = O.filter_response(n, B)
    offs = np.arange(D) - D / 2 + 0.5
    ideal = np.array([_erf_profile(o, D, sf) for o in offs])
    assert np.max(np.abs(resp - ideal)) < 2e-5
    # symmetric in the offset and exactly one half at the bucket edge in the ideal
    assert np.allclose(resp, resp[::-1], atol=1e-12)
    assert resp.min() > 0.45 and resp.max() <= 1 + 1e-6


@pytest.mark.parametrize("n,B", [(2 ** 12, 64), (2 ** 13, 512)])
def test_window_response_equals_dft_of_taps(n, B):
    """Ghat' at the half-integer offsets o equals the (2n)-point DFT of the taps at the
    odd frequency 2o (numpy's FFT as the independent route)."""
    h, s, taps = O.filter_taps(n, B)
    buf = np.zeros(2 * n)
    for t in range(-h, h + 1):
        buf[t % (2 * n)] += taps[t + h]
    spec = np.fft.fft(buf).real / n
    D = n // B
    resp = O.filter_response(n, B)
    for j in range(D):
        o2 = 2 * j - D + 1
        assert abs(resp[j] - spec[o2 % (2 * n)]) < 1e-12


def test_window_stopband():
    n, B = 2 ** 14, 128
    h, s, taps = O.filter_taps(n, B)
    D = n // B
    buf = np.zeros(n)
    for t in range(-h, h + 1):
        buf[t % n] += taps[t + h]
    spec = np.abs(np.fft.fft(buf)) / n
    f = np.minimum(np.arange(n), n - np.arange(n))
    # beyond (1 + alpha) D / 2 from the centre the gain is at the tolerance level
    assert spec[f >= (1 + 0.5) * D / 2 + 1].max() < 1e-5
    # inside (1 - alpha) D / 2 it is flat
    assert np.all(np.abs(spec[f <= (1 - 0.5) * D / 2 - 1] - 1) < 1e-5)


# --------------------------------------------------------------------------
# Hash function (Lemma 1, Lemma 2, convolution theorem): the bucket spectrum
# --------------------------------------------------------------------------

def _response_at(taps, h, n, phi):
    t = np.arange(-h, h + 1)
    return float(np.sum(taps * np.cos(2 * np.pi * phi * t / n))) / n


@pytest.mark.parametrize("n,B,seed", [(256, 16, 0), (512, 32, 1), (1024, 64, 2)])
def test_hash_spectrum_brute_force(n, B, seed):
    """Zhat_c = sum_i xhat_i omega^{-tau i} Ghat'(c D - 1/2 - sigma i) for every bucket c,
    with xhat from numpy's FFT: Lemma 1 moves xhat_i to sigma i with phase omega^{-tau i},
    the window multiplies in time (convolution in frequency) and Lemma 2 samples every
    D-th frequency of the half-bin-shifted filtered spectrum."""
    rng = np.random.default_rng(seed)
    x = (rng.normal(size=n) + 1j * rng.normal(size=n)).astype(np.complex64).astype(np.complex128)
    xh = np.fft.fft(x)
    h, s, taps = O.filter_taps(n, B)
    D = n // B
    for phase, index in [(0, 3), (1, 0), (2, 5)]:
        sigma, tau = O.hash_params(seed, phase, index, n)
        Z = O.hash_spectrum_1d(x, B, seed, phase, index)
        i = np.arange(n)
        p = (sigma * i) % n
        ph = np.exp(2j * np.pi * ((tau * i) % n) / n)      # omega^{-tau i}
        expect = np.zeros(B, dtype=complex)
        for c in range(B):
            d = (c * D - 0.5 - p) % n
            d = np.where(d > n / 2, d - n, d)
            g = np.array([_response_at(taps, h, n, dd) for dd in d])
            expect[c] = np.sum(xh * ph * g)
        assert np.max(np.abs(Z - expect)) < 1e-9 * np.max(np.abs(expect))


def test_hash_spectrum_2d_brute_force():
    N, B, seed = 32, 8, 4
    rng = np.random.default_rng(seed)
    x = rng.normal(size=(N, N)) + 1j * rng.normal(size=(N, N))
    xh = np.fft.fft2(x)
    h, s, taps = O.filter_taps(N, B)
    D = N // B
    s1, t1, s2, t2 = O.hash_params(seed, 1, 2, N, ndim=2)
    Z = O.hash_spectrum_2d(x, B, seed, 1, 2)
    i = np.arange(N)
    g1 = {}
    expect = np.zeros((B, B), dtype=complex)
    for c1 in range(B):
        for c2 in range(B):
            acc = 0
            for a in range(N):
                d1 = (c1 * D - 0.5 - s1 * a) % N
                d1 = d1 - N if d1 > N / 2 else d1
                if (c1, a) not in g1:
                    g1[(c1, a)] = _response_at(taps, h, N, d1)
                d2 = (c2 * D - 0.5 - s2 * i) % N
                d2 = np.where(d2 > N / 2, d2 - N, d2)
                gg = np.array([_response_at(taps, h, N, dd) for dd in d2])
                ph = np.exp(2j * np.pi * ((t1 * a + t2 * i) % N) / N)
                acc += np.sum(xh[a, :] * ph * g1[(c1, a)] * gg)
            expect[c1, c2] = acc
    assert np.max(np.abs(Z - expect)) < 1e-9 * np.max(np.abs(expect))


def test_lemma1_and_lemma2_conventions():
    """The identities the oracle's hash relies on, checked with numpy alone:
    Lemma 1 (permutation) and Lemma 2 (aliasing), in the paper's DFT convention."""
    n, B = 256, 16
    rng = np.random.default_rng(0)
    x = rng.normal(size=n) + 1j * rng.normal(size=n)
    sigma, tau = 77, 13
    Px = x[(sigma * np.arange(n) + tau) % n]
    lhs = np.fft.fft(Px)[(sigma * np.arange(n)) % n]
    rhs = np.fft.fft(x) * np.exp(2j * np.pi * tau * np.arange(n) / n)
    assert np.allclose(lhs, rhs, atol=1e-9)
    y = x.reshape(n // B, B).sum(axis=0)
    assert np.allclose(np.fft.fft(y), np.fft.fft(x)[:: n // B], atol=1e-9)


# --------------------------------------------------------------------------
# Estimator (Eq. (11)) exactness on isolated coefficients
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n,B", [(1024, 32), (4096, 256)])
def test_isolated_coefficient_estimate_exact(n, B):
    D = n // B
    resp = O.filter_response(n, B)
    for f, val in [(0, 1.0), (5, 0.3 - 0.4j), (n // 2, -1j), (n - 1, 2.0 + 0.5j), (777 % n, 1j)]:
        xh = np.zeros(n, complex)
        xh[f] = val
        x = np.fft.ifft(xh)
        for l in range(4):
            sigma, tau = O.hash_params(3, 2, l, n)
            Z = O.hash_spectrum_1d(x, B, 3, 2, l)
            p = (sigma * f) % n
            q = (2 * p + 1 + D) // (2 * D)
            hb, o2 = q % B, 2 * p + 1 - 2 * q * D
            est = Z[hb] * np.exp(-2j * np.pi * ((tau * f) % n) / n) / resp[(o2 + D - 1) // 2]
            assert abs(est - val) < 1e-9
            others = np.delete(np.abs(Z), hb)
            assert others.max() <= 0.5 * abs(val) + 1e-9   # only neighbours see leakage


# --------------------------------------------------------------------------
# Local maxima (Section III-A) and the controller (Eqs. (12)-(14))
# --------------------------------------------------------------------------

def test_fig5_worked_example():
    g = _gold("fig5_local_maxima.json")
    N, B, k = g["N"], g["B"], g["k"]
    hits = 0
    for seed in range(4):
        sig = sparse_signal_2d(N, k, seed)
        Z = O.hash_spectrum_2d(sig.x, B, seed, 0, 0)
        lm, T, _ = O.local_maxima(np.abs(Z) ** 2, ndim=2)
        hits += len(lm) == g["local_maxima"]
    assert hits == 4


def test_local_maxima_synthetic_1d():
    B = 64
    E = np.full(B, 1e-6)
    spikes = [3, 10, 40, 63]
    for c in spikes:
        E[c] = 1.0
    E[11] = 0.3                          # shoulder next to a spike: not a maximum
    E[0] = 0.9                           # cyclic neighbour of 63: 63 dominates it
    lm, T, _ = O.local_maxima(E)
    assert lm.tolist() == [3, 10, 40, 63]
    # exact tie between neighbours: the later bucket (cyclically) wins, one maximum
    E2 = np.full(B, 1e-6)
    E2[20] = E2[21] = 1.0
    E2[63] = E2[0] = 0.5
    lm2, _, _ = O.local_maxima(E2)
    assert lm2.tolist() == [0, 21]
    # below the threshold max(thr_rel * max, thr_med * median) nothing counts
    E3 = np.full(B, 1.0)
    E3[5] = 15.0
    lm3, T3, _ = O.local_maxima(E3)
    assert T3 == pytest.approx(20.0) and lm3.tolist() == []
    # the median is the element of rank floor(B/2) of the ascending energies (the upper of
    # the two middle ones for even B): half the buckets at 1, half at 2, so the median is 2
    # and T = 40; a spike of 30 lies between 20 * 1 and 20 * 2 and is not a maximum
    E4 = np.where(np.arange(B) % 2 == 0, 1.0, 2.0)
    E4[9] = 30.0
    lm4, T4, _ = O.local_maxima(E4)
    assert T4 == 20.0 * np.sort(E4)[B // 2] == 40.0 and lm4.tolist() == []
    E4[9] = 50.0
    assert O.local_maxima(E4)[0].tolist() == [9]


def test_local_maxima_synthetic_2d():
    B = 16
    E = np.full((B, B), 1e-6)
    E[2, 3] = 1.0
    E[2, 4] = 0.8                        # 8-neighbour, smaller
    E[9, 9] = 0.5
    E[10, 10] = 0.5                      # diagonal exact tie: (10,10) is later, wins
    E[15, 0] = 0.7
    E[0, 15] = 0.6                       # diagonal across both wraps: (15,0) and (0,15) are neighbours
    lm, _, _ = O.local_maxima(E, ndim=2)
    assert sorted(lm.tolist()) == sorted([2 * B + 3, 10 * B + 10, 15 * B + 0])


def test_controller_branches_eq14():
    g = _gold("eq14_controller.json")
    for kp, kc, br in g["cases_k_prev_k_cur_branch"]:
        assert O.controller_branch(kp, kc, g["delta1"], g["delta2"]) == br, (kp, kc)
    assert O.controller_branch(0, 5) == 1 and O.controller_branch(7, 0) == 1


def test_default_parameters_are_the_papers_and_the_readings():
    """The defaults of a whole transform: Eq. (14)'s constants as the paper prints them
    (golden file), and where the paper leaves a value open the readings taken for it:
    threshold T = max(1e-3 max E, 20 median E) and a 1 % tie band for Section III-A's
    undefined `threshold` and ties, seven location and seven estimation hashes for the
    unstated `loops`, and the window tolerance 1e-6 with alpha = 1/2 for the flat window
    whose parameters Eqs. (8)-(9) leave open."""
    g = _gold("eq14_controller.json")
    p = O.default_params()
    assert (p.delta1, p.delta2, p.eps1, p.eps2) == (g["delta1"], g["delta2"], g["eps1"], g["eps2"])
    assert (p.thr_rel, p.thr_med, p.tie_eta) == (1e-3, 20.0, 1e-2)
    assert (p.loops_loc, p.loops_est) == (7, 7)
    assert (p.filter_tol, p.filter_alpha) == (1e-6, 0.5)
    assert (p.b_min_log2, p.b_max_log2, p.fixed_k, p.est_reuse_loc) == (0, 0, 0, 0)


@pytest.mark.parametrize("logn,k,seed", [(14, 32, 3), (13, 32, 0)])
def test_transform_walk_stops_at_the_first_ratio_below_delta2(logn, k, seed):
    """Eqs. (12)-(14) in a whole transform: B doubles from 16 while r = |1 - k_t/k_(t-1)|
    >= delta2 (a zero count reads as an unbounded change) and the walk stops at the first
    r < delta2.  These seeds end on the keep branch (delta1 <= r < delta2), where a walk
    that stopped only below delta1 would go on."""
    sig = sparse_signal_1d(1 << logn, k, seed)
    res = O.atsfft_1d(sig.x, seed=seed)
    Bs = [int(t[0]) for t in res.trials]
    ks = [int(t[1]) for t in res.trials]
    assert res.status == 0
    assert Bs == [16 << t for t in range(len(Bs))]

    def ratio(prev, cur):
        return math.inf if prev == 0 or cur == 0 else abs(1.0 - cur / prev)

    rs = [ratio(ks[t - 1], ks[t]) for t in range(1, len(ks))]
    assert all(r >= 0.05 for r in rs[:-1]) and rs[-1] < 0.05, rs
    assert rs[-1] >= 0.02, rs   # the keep branch
    assert (res.B_star, res.k_star) == (Bs[-1], ks[-1])


def test_top_num_keeps_the_num_largest_when_energies_are_apart():
    """Algorithm 1 "find num largest": with energies more than the tie band apart the
    cutoff is the num largest local maxima, by brute force."""
    rng = np.random.default_rng(3)
    for trial in range(20):
        nb = 256
        lm = np.sort(rng.choice(nb, size=int(rng.integers(1, 60)), replace=False))
        E = np.zeros(nb)
        E[lm] = 1.1 ** rng.permutation(len(lm))   # distinct, 10 % apart
        for num in (1, 3, len(lm) // 2 + 1, len(lm), len(lm) + 5):
            want = np.sort(lm[np.argsort(-E[lm], kind="stable")[:num]])
            assert O.top_num(E, lm, num).tolist() == want.tolist(), (trial, num)


def test_top_num_fills_the_tie_band_in_ascending_bucket_order():
    """Energies within the relative band eta of the num-th largest count as tied and the
    lower bucket index wins (the reading of the ties).  Worked case, eta = 1 %, num = 3:
    energies 2.0 (bucket 20), 1.005 (11), 1.000 (3), 0.995 (7), 0.5 (25); the pivot is
    the third largest, 1.000; 2.0 lies above the band [0.99, 1.01] and is kept; the band
    holds buckets 3, 7 and 11, of which the two lowest, 3 and 7, fill the cut."""
    E = np.zeros(32)
    E[[3, 7, 11, 20, 25]] = [1.000, 0.995, 1.005, 2.0, 0.5]
    assert O.top_num(E, [3, 7, 11, 20, 25], 3, eta=1e-2).tolist() == [3, 7, 20]
    # without a tie band the three largest energies
    assert O.top_num(E, [3, 7, 11, 20, 25], 3, eta=0.0).tolist() == [3, 11, 20]
    # all equal: the num lowest buckets; at most num kept: all of them
    F = np.zeros(16)
    F[[2, 4, 6, 8, 10]] = 1.0
    assert O.top_num(F, [2, 4, 6, 8, 10], 2).tolist() == [2, 4]
    assert O.top_num(F, [2, 4, 6, 8, 10], 9).tolist() == [2, 4, 6, 8, 10]


# --------------------------------------------------------------------------
# Decision margins and the near-decision log (the switch of the GPU parity rule)
# --------------------------------------------------------------------------

def _rel(a, b):
    return abs(a - b) / max(abs(a), abs(b))


def test_margin_of_a_threshold_decision_worked_case():
    """Section III-A local maxima, threshold T = max(thr_rel maxE, thr_med medianE).
    Worked case: 64 buckets at 1e-9 (median term 2e-8), a spike of 1 at bucket 10
    (T = 1e-3) and an isolated bucket 30 at T (1 + 3e-5).  The only comparison near its
    boundary is E_30 against T, relative margin 3e-5 / (1 + 3e-5); the noise buckets tie
    within the band but are below T, so reversing their pairs changes nothing and is not
    a deciding comparison."""
    E = np.full(64, 1e-9)
    E[10] = 1.0
    E[30] = 1e-3 * (1 + 3e-5)
    for mode in (0, 1):
        lm, T, m, dec = O.local_maxima_log(E, mode=mode, band=1e-3)
        assert lm.tolist() == [10, 30] and T == pytest.approx(1e-3, rel=1e-15)
        assert m == pytest.approx(_rel(E[30], 1e-3), rel=1e-9)
        assert [(d.kind, d.c, d.m) for d in dec] == [("threshold", 30, -1)]
        assert dec[0].margin == pytest.approx(m, rel=1e-12)
    # just below T: the same margin, bucket 30 no longer a maximum
    E[30] = 1e-3 * (1 - 3e-5)
    lm, _, m, dec = O.local_maxima_log(E, band=1e-3)
    assert lm.tolist() == [10] and m == pytest.approx(_rel(E[30], 1e-3), rel=1e-9)
    assert [(d.kind, d.c) for d in dec] == [("threshold", 30)]


def test_margin_of_a_dominance_decision_depends_on_what_the_outcome_is():
    """Two neighbours 0.5 and 0.5 (1 + eta)(1 + 2e-5): the later one dominates by a
    relative 2e-5 beyond the tie band.  Reversing the pair swaps which bucket is the
    maximum: that changes the maxima set (location, mode 1: logged, margin 2e-5/(1+2e-5))
    but not their number (tuning, mode 0: not a deciding comparison)."""
    eta = 1e-2
    E = np.full(64, 1e-9)
    E[10] = 1.0
    E[40] = 0.5
    E[41] = 0.5 * (1 + eta) * (1 + 2e-5)
    lm, _, m1, dec1 = O.local_maxima_log(E, mode=1, band=1e-3)
    assert lm.tolist() == [10, 41]
    assert [(d.kind, d.c, d.m) for d in dec1] == [("dominance", 40, 41)]
    assert m1 == pytest.approx(_rel(E[41], (1 + eta) * E[40]), rel=1e-9)
    lm0, _, m0, dec0 = O.local_maxima_log(E, mode=0, band=1e-3)
    assert lm0.tolist() == [10, 41] and dec0 == [] and m0 > 1e-3
    # the same pair reversed in position: the earlier bucket dominates; still logged
    E[40], E[41] = E[41], E[40]
    lm, _, m, dec = O.local_maxima_log(E, mode=1, band=1e-3)
    assert lm.tolist() == [10, 40] and [(d.kind, d.c, d.m) for d in dec] == [("dominance", 40, 41)]


def test_margin_of_the_cutoff_band_worked_case():
    """Algorithm 1 "find num largest" with the tie band: maxima 1.0 (bucket 5), 0.9 (15),
    0.5 (25) and 0.9 (1 - eta)(1 - 4e-5) (35), num = 2.  The pivot is 0.9, the band
    [0.891, 0.909]; bucket 35 lies just below its lower edge (relative 4e-5) and is the
    only comparison near a boundary; the cut keeps 5 and 15."""
    eta = 1e-2
    E = np.full(64, 1e-9)
    E[[5, 15, 25]] = [1.0, 0.9, 0.5]
    E[35] = 0.9 * (1 - eta) * (1 - 4e-5)
    sel, m, dec = O.location_select_log(E, 2, band=1e-3)
    assert sel.tolist() == [5, 15]
    assert [(d.kind, d.c) for d in dec] == [("topnum", 35)]
    assert m == pytest.approx(_rel(E[35], 0.9 * (1 - eta)), rel=1e-9)


def test_a_near_local_maximum_flip_logs_the_buckets_whose_selection_it_moves():
    """A near dominance decision in a location hash moves the cut: maxima 1.0 (bucket 5),
    0.935 (15) and the pair 34 < 35 with E_35 = 0.95 just beyond the tie band above E_34.
    num = 2: the pivot is E_35, the band [0.9405, 0.9595], the cut {5, 35}.  Were the pair
    reversed, 34 would be the maximum instead, the pivot E_34 = 0.9406 and its band
    [0.9312, 0.9500] would hold 15 and 34, of which the lower bucket fills the cut: {5, 15}.
    So the log names the pair and, as moved by that flip, buckets 15 and 35 (bucket 15 is
    nowhere near a boundary itself)."""
    eta = 1e-2
    E = np.full(64, 1e-9)
    E[5], E[15] = 1.0, 0.935
    E[35] = 0.95
    E[34] = 0.95 / ((1 + eta) * (1 + 2e-5))
    sel, m, dec = O.location_select_log(E, 2, band=1e-3)
    assert sel.tolist() == [5, 35]
    got = sorted((d.kind, d.c, d.m) for d in dec)
    assert got == [("dominance", 34, 35), ("pivot", 15, 34), ("pivot", 35, 34)], got
    assert m == pytest.approx(_rel(E[35], (1 + eta) * E[34]), rel=1e-9)
    # the flipped hash, computed directly (bucket 35 no longer a maximum), has the cut
    # the log predicts
    G = np.full(64, 1e-9)
    G[5], G[15], G[34] = 1.0, 0.935, E[34]
    assert O.location_select_log(G, 2, band=1e-3)[0].tolist() == [5, 15]


def test_margin_bounds_every_outcome_change_under_perturbation():
    """The margin is the smallest relative distance of a deciding comparison from its
    boundary, so scaling every energy by its own factor within (1 +- margin/3) can change
    neither the count (tuning) nor the maxima set (location) nor the cut; energies drawn
    from a few levels make exact and near ties frequent."""
    rng = np.random.default_rng(11)
    for trial in range(40):
        ndim = 1 if trial % 2 == 0 else 2
        side = 128 if ndim == 1 else 12
        shape = (side,) if ndim == 1 else (side, side)
        levels = np.array([1e-9, 1e-4, 1e-3, 1.02e-3, 0.3, 0.302, 0.5, 0.505, 1.0])
        E = levels[rng.integers(0, len(levels), size=shape)] * (1 + 1e-4 * rng.random(shape))
        for mode in (0, 1):
            lm, _, m, _ = O.local_maxima_log(E, ndim=ndim, mode=mode, band=0.0)
            if not np.isfinite(m) or m <= 0:
                continue
            for _ in range(10):
                P = E * (1 + (m / 3) * rng.uniform(-1, 1, size=shape))
                lp, _, _, _ = O.local_maxima_log(P, ndim=ndim, mode=mode, band=0.0)
                if mode == 0:
                    assert len(lp) == len(lm), (trial, m)
                else:
                    assert lp.tolist() == lm.tolist(), (trial, m)
        num = max(1, len(O.local_maxima(E, ndim=ndim)[0]) // 2)
        sel, m, _ = O.location_select_log(E, num, ndim=ndim, band=0.0)
        for _ in range(10):
            P = E * (1 + (m / 3) * rng.uniform(-1, 1, size=shape))
            assert O.location_select_log(P, num, ndim=ndim, band=0.0)[0].tolist() == sel.tolist()


@pytest.mark.parametrize("ndim,seed", [(1, 4), (1, 18), (2, 2), (2, 6)])
def test_logged_transform_margins_agree_with_the_result(ndim, seed):
    """Whole transforms (Algorithm 2): the log with an unbounded band holds every
    deciding comparison, so its smallest margin is the result's min_margin; a narrower
    band keeps exactly those below it; and logging changes no output.  (Seeds 4 and 2
    have their smallest margin in a location hash, 18 and 6 in a tuning trial.)"""
    if ndim == 1:
        sig = sparse_signal_1d(1 << 12, 12, seed, snr_db=30)
    else:
        sig = sparse_signal_2d(64, 6, seed, snr_db=30)
    ref = (O.atsfft_1d if ndim == 1 else O.atsfft_2d)(sig.x, seed=seed)
    r_all, d_all = O.atsfft_log(sig.x, seed=seed, band=np.inf)
    r_cut, d_cut = O.atsfft_log(sig.x, seed=seed, band=3e-2)
    for r in (r_all, r_cut):
        assert r.loc.tolist() == ref.loc.tolist() and r.k_star == ref.k_star
        assert r.min_margin == ref.min_margin
    base = [d for d in d_all if d.kind != "pivot"]
    assert {d.phase for d in base} == {0, 1}
    assert min(d.margin for d in base) == ref.min_margin
    key = lambda d: (d.phase, d.hash, d.kind, d.c, d.m)
    assert sorted(map(key, (d for d in d_cut if d.kind != "pivot"))) == \
        sorted(map(key, (d for d in base if d.margin < 3e-2)))
    # tuning records name the trials' log2 B, location records the hash index
    tB = {int(b).bit_length() - 1 for b, _, _ in ref.trials}
    assert {d.hash for d in base if d.phase == 0} <= tB
    assert {d.hash for d in base if d.phase == 1} <= set(range(7))


def test_bucket_of_matches_the_reverse_hash_preimages():
    """Eq. (10): coordinate i lies in bucket h(i) exactly when sigma i mod n is one of the
    D permuted positions [c D - D/2, c D + D/2) the reverse hash visits."""
    n, B = 1 << 10, 32
    D = n // B
    sigma = O.hash_params(5, 1, 0, n)[0]
    for i in range(n):
        c = O.bucket_of(i, sigma, n, B)
        p = sigma * i % n
        assert (p - (c * D - D // 2)) % n < D


def test_median_componentwise_matches_numpy():
    rng = np.random.default_rng(5)
    for L in (1, 3, 5, 7, 9):
        v = rng.normal(size=L) + 1j * rng.normal(size=L)
        m = O.median_componentwise(v)
        assert m == complex(np.median(v.real), np.median(v.imag))


# --------------------------------------------------------------------------
# Whole transform against a brute-force DFT on tiny inputs
# --------------------------------------------------------------------------

CASES_1D = [(1024, 1, 0), (1024, 2, 0), (1024, 4, 2), (4096, 2, 2), (4096, 4, 1), (4096, 6, 0),
            (4096, 6, 3), (16384, 16, 0), (16384, 16, 1)]


@pytest.mark.parametrize("n,k,seed", CASES_1D)
def test_atsfft_1d_brute_force(n, k, seed):
    sig = sparse_signal_1d(n, k, seed)
    xh = np.fft.fft(sig.x.astype(np.complex128))          # exact DFT of the given input
    r = O.atsfft_1d(sig.x, seed=seed)
    assert r.status == 0
    assert set(sig.support.tolist()) <= set(r.loc.tolist())
    assert np.all(np.diff(r.loc) > 0)
    got = dict(zip(r.loc.tolist(), r.val.tolist()))
    for i in range(n):
        if i in got:
            assert abs(got[i] - xh[i]) < 1e-5
    assert r.k_star <= k


CASES_2D = [(64, 1, 0), (128, 3, 1), (128, 6, 2), (256, 10, 0)]


@pytest.mark.parametrize("N,k,seed", CASES_2D)
def test_atsfft_2d_brute_force(N, k, seed):
    sig = sparse_signal_2d(N, k, seed)
    xh = np.fft.fft2(sig.x.astype(np.complex128)).ravel()
    r = O.atsfft_2d(sig.x, seed=seed)
    assert r.status in (0, 5)
    assert r.loc.tolist() == sig.support.tolist()
    assert np.max(np.abs(r.val - xh[r.loc])) < 1e-5


def test_2d_transposed_support_is_distinguished():
    """A support that is not symmetric under transposition must come back untransposed."""
    N = 128
    xh = np.zeros((N, N), complex)
    xh[3, 70] = 1.0
    xh[100, 5] = 0.5j
    x = np.fft.ifft2(xh).astype(np.complex64)
    r = O.atsfft_2d(x, seed=1)
    got = dict(zip(r.loc.tolist(), r.val.tolist()))
    assert abs(got[3 * N + 70] - 1.0) < 1e-5 and abs(got[100 * N + 5] - 0.5j) < 1e-5
    assert 70 * N + 3 not in got and 5 * N + 100 not in got
    extras = [abs(v) for i, v in got.items() if i not in (3 * N + 70, 100 * N + 5)]
    assert max(extras, default=0.0) < 1e-5


# --------------------------------------------------------------------------
# Degenerate cases and limits
# --------------------------------------------------------------------------

def test_zero_signal_gives_empty_output():
    r = O.atsfft_1d(np.zeros(4096, np.complex64))
    assert r.status == 0 and r.count == 0 and r.k_star == 0
    r2 = O.atsfft_2d(np.zeros((64, 64), np.complex64))
    assert r2.status == 0 and r2.count == 0


def test_capacity_reports_needed_count():
    sig = sparse_signal_1d(4096, 4, 1)
    r = O.atsfft_1d(sig.x, seed=1, capacity=2)
    assert r.status == 6 and r.count >= 4 and len(r.loc) == 2
    # exactly enough room is no error; one less is
    c = O.atsfft_1d(sig.x, seed=1).count
    r = O.atsfft_1d(sig.x, seed=1, capacity=c)
    assert r.status == 0 and r.count == c and len(r.loc) == c
    r = O.atsfft_1d(sig.x, seed=1, capacity=c - 1)
    assert r.status == 6 and r.count == c and len(r.loc) == c - 1


def test_trial_cap_not_converged():
    sig = sparse_signal_1d(1 << 16, 50, 3, 40)
    r = O.atsfft_1d(sig.x, seed=3, params=O.default_params(tune_max=2))
    assert r.status == 4 and len(r.trials) == 2


def test_pure_noise_is_not_sparse():
    rng = np.random.default_rng(0)
    x = (rng.normal(size=1 << 14) + 1j * rng.normal(size=1 << 14)).astype(np.complex64)
    r = O.atsfft_1d(x, seed=0)
    assert r.status == 5 and r.B_star == (1 << 14) // 16


def test_invalid_arguments():
    r = O.atsfft_1d(np.zeros(1000, np.complex64))
    assert r.status == 1
    r = O.atsfft_1d(np.zeros(4096, np.complex64), params=O.default_params(eps1=0.3))
    assert r.status == 1
    r = O.atsfft_1d(np.zeros(4096, np.complex64), params=O.default_params(delta1=0.06))
    assert r.status == 1


def test_k_hint_starts_higher():
    sig = sparse_signal_1d(1 << 16, 50, 3, 40)
    r = O.atsfft_1d(sig.x, seed=3, k_hint=50)
    assert r.trials[0][0] == 128


def test_vote_rule_single_and_three_loops():
    """Section II-B keeps coordinates found in at least half of the location loops.
    With one loop that is exactly the union of the preimages of the selected buckets
    (D = n/B coordinates each, disjoint); with three loops a coordinate needs two votes.
    Seed 3 is a case where no location hash has more local maxima than k*, so every
    local maximum is selected."""
    n, seed = 1 << 14, 3
    sig = sparse_signal_1d(n, 16, seed)
    r1 = O.atsfft_1d(sig.x, seed=seed, params=O.default_params(loops_loc=1))
    B, D = r1.B_star, n // r1.B_star
    Z = O.hash_spectrum_1d(sig.x, B, seed, 1, 0)
    lm, _, _ = O.local_maxima(np.abs(Z) ** 2)
    assert r1.count == min(len(lm), r1.k_star) * D
    sigma, _ = O.hash_params(seed, 1, 0, n)
    p = (sigma * r1.loc) % n
    assert set(((2 * p + 1 + D) // (2 * D)) % B) <= set(lm.tolist())
    r3 = O.atsfft_1d(sig.x, seed=seed, params=O.default_params(loops_loc=3))
    assert r3.B_star == B
    votes = np.zeros(n, int)
    for l in range(3):
        Z = O.hash_spectrum_1d(sig.x, B, seed, 1, l)
        lm, _, _ = O.local_maxima(np.abs(Z) ** 2)
        assert len(lm) <= r3.k_star
        sigma, _ = O.hash_params(seed, 1, l, n)
        q = ((2 * ((sigma * np.arange(n)) % n) + 1 + D) // (2 * D)) % B
        votes += np.isin(q, lm)
    assert r3.loc.tolist() == np.flatnonzero(votes >= 2).tolist()


def test_fixed_support_estimates_are_linear_and_equal_the_dft_on_sparse_inputs():
    """Eq. (11) at a fixed support: every loop's estimate is a linear functional of the
    signal (superposition), and on an exactly sparse signal it equals the DFT value at
    each support point wherever the coefficient is alone in its bucket (window gain
    divided out), so the componentwise median is the DFT value."""
    import oracle as O
    from synth import sparse_signal_1d

    n, B = 1 << 12, 256
    sig = sparse_signal_1d(n, 8, 3)
    loc = sig.support
    X = np.fft.fft(sig.x.astype(np.complex128))
    est = O.estimates_1d(sig.x, B, loc, seed=5)
    assert est.shape == (8, 7)
    # each loop is exact unless another coefficient shares its bucket; the median is exact
    exact = np.abs(est - X[loc][:, None]) < 1e-7
    assert exact.mean() > 0.9
    med = np.sort(est.real, axis=1)[:, 3] + 1j * np.sort(est.imag, axis=1)[:, 3]
    assert np.abs(med - X[loc]).max() < 1e-7
    rng = np.random.default_rng(0)
    u = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    v = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    a, b = 0.7 - 0.2j, -1.3 + 0.4j
    lhs = O.estimates_1d(a * u + b * v, B, loc, seed=5)
    rhs = a * O.estimates_1d(u, B, loc, seed=5) + b * O.estimates_1d(v, B, loc, seed=5)
    assert np.abs(lhs - rhs).max() < 1e-9 * np.abs(rhs).max()


def test_fixed_k_bucket_count_by_brute_force():
    """Fixed-k mode's B is the smallest power of two with B^2 >= n k in 1D and B^4 >= N^2 k
    in 2D (the bucket count of the SFFT setting, per axis), within the B range: found here
    by doubling B until the inequality holds."""
    def smallest(side_pow, total, lo, hi):
        B = 1
        while B ** side_pow < total:
            B *= 2
        return min(max(B, lo), hi)

    for n in (1 << 12, 1 << 16):
        for k in (1, 2, 3, 16, 17, 100, 1000):
            r = O.atsfft_1d(np.zeros(n, np.complex64), k_hint=k, seed=1,
                            params=O.default_params(fixed_k=1))
            assert r.B_star == smallest(2, n * k, 16, n // 16), (n, k)
    for N in (64, 256):
        for k in (1, 2, 3, 4, 5, 10, 100, 1000):
            r = O.atsfft_2d(np.zeros((N, N), np.complex64), k_hint=k, seed=1,
                            params=O.default_params(fixed_k=1))
            assert r.B_star == smallest(4, N * N * k, 8, N // 4), (N, k)


def test_a_single_trial_range_is_not_an_error():
    """With one B to try (n = 256: B in [16, 16]; or a hint that starts at the largest B)
    Eq. (12) has no previous count, so Eq. (14) never asks to double past the range: the
    transform ends OK at that B (the reading of the stop rule), and exactly sparse inputs
    are recovered."""
    sig = sparse_signal_1d(256, 2, 0)
    r = O.atsfft_1d(sig.x, seed=0)
    assert r.status == 0 and [int(t[0]) for t in r.trials] == [16] and r.B_star == 16
    assert r.loc.tolist() == sorted(sig.support.tolist())
    sig = sparse_signal_1d(1 << 14, 16, 1)
    r = O.atsfft_1d(sig.x, seed=1, k_hint=600)   # ceil(log2(1200)) = 11 > n/16 = 2^10
    assert r.status == 0 and [int(t[0]) for t in r.trials] == [1 << 10]
    assert r.loc.tolist() == sorted(sig.support.tolist())


@pytest.mark.parametrize("N,k,seed,status", [(256, 10, 0, 0), (512, 40, 1, 0), (256, 20, 3, 5)])
def test_2d_walk_starts_at_8_and_follows_eq14(N, k, seed, status):
    """2D: B (per axis) doubles from 8 while r >= delta2 and stops at the first r < delta2;
    a walk that would double past N/4 ends NOT_SPARSE (status 5) there."""
    sig = sparse_signal_2d(N, k, seed)
    res = O.atsfft_2d(sig.x, seed=seed)
    Bs = [int(t[0]) for t in res.trials]
    ks = [int(t[1]) for t in res.trials]
    assert Bs == [8 << t for t in range(len(Bs))]
    rs = [math.inf if a == 0 or b == 0 else abs(1.0 - b / a) for a, b in zip(ks, ks[1:])]
    assert all(r >= 0.05 for r in rs[:-1])
    assert res.status == status
    if status == 0:
        assert rs[-1] < 0.05
    else:
        assert rs[-1] >= 0.05 and Bs[-1] == N // 4


def test_fixed_k_mode_bucket_count_and_recovery():
    """Fixed-k mode (no tuning): B is the smallest power of two with B^2 >= n k (2D:
    B^4 >= N^2 k), k* = the hint, and an exactly sparse input is recovered exactly."""
    import oracle as O
    from synth import sparse_signal_1d, sparse_signal_2d

    for n, k, want in [(1 << 14, 16, 9), (1 << 14, 17, 10), (1 << 20, 1000, 15)]:
        x = np.zeros(n, np.complex64)
        r = O.atsfft_1d(x, k_hint=k, seed=1, params=O.default_params(fixed_k=1))
        assert r.B_star == 1 << want and r.k_star == k and len(r.trials) == 0
    r = O.atsfft_2d(np.zeros((256, 256), np.complex64), k_hint=10, seed=1,
                    params=O.default_params(fixed_k=1))
    assert r.B_star == 1 << 5   # N^2 k = 655360 -> ceil(log2) = 20 -> ceil(20/4) = 5
    sig = sparse_signal_1d(1 << 12, 8, 5)
    r = O.atsfft_1d(sig.x, k_hint=8, seed=5, params=O.default_params(fixed_k=1))
    X = np.fft.fft(sig.x.astype(np.complex128))
    assert r.loc.tolist() == sorted(sig.support.tolist())
    assert np.abs(r.val - X[r.loc]).max() < 1e-6
    sig2 = sparse_signal_2d(64, 5, 6)
    r2 = O.atsfft_2d(sig2.x, k_hint=5, seed=6, params=O.default_params(fixed_k=1))
    X2 = np.fft.fft2(sig2.x.astype(np.complex128)).ravel()
    # the small fixed B of 2D (16 x 16 buckets for k = 5) lets a few preimages collect
    # the votes too; the true support is all there, with exact values
    true = np.isin(r2.loc, sig2.support)
    assert true.sum() == len(sig2.support)
    assert np.abs(r2.val - X2[r2.loc])[true].max() < 1e-6
    assert O.atsfft_1d(sig.x, k_hint=0, seed=5, params=O.default_params(fixed_k=1)).status == 1


def test_estimation_reusing_location_hashes():
    """With est_reuse_loc the estimates come from the location hashes: an exactly sparse
    input is still recovered exactly, the location stage is unchanged, and more
    estimation than location loops is rejected."""
    import oracle as O
    from synth import sparse_signal_1d

    sig = sparse_signal_1d(1 << 12, 8, 9)
    a = O.atsfft_1d(sig.x, seed=9)
    b = O.atsfft_1d(sig.x, seed=9, params=O.default_params(est_reuse_loc=1))
    X = np.fft.fft(sig.x.astype(np.complex128))
    assert a.loc.tolist() == b.loc.tolist() and a.k_star == b.k_star
    # within the window's stop-band leakage (tolerance 1e-6 per neighbour coefficient)
    assert np.abs(b.val - X[b.loc]).max() < 1e-5
    # the reused estimates are exactly the location hashes' Eq. (11) values
    est_loc = O.estimates_1d(sig.x, a.trials[-1][0], b.loc, seed=9,
                             params=O.default_params(est_reuse_loc=1))
    est_new = O.estimates_1d(sig.x, a.trials[-1][0], b.loc, seed=9)
    assert not np.allclose(est_loc, est_new, atol=0, rtol=0)
    bad = O.default_params(est_reuse_loc=1, loops_loc=5, loops_est=7)
    assert O.atsfft_1d(sig.x, seed=9, params=bad).status == 1   # invalid argument


# --------------------------------------------------------------------------
# The ctypes wrapper against the oracle's C prototypes
# --------------------------------------------------------------------------

def test_wrapper_argument_and_return_types_match_the_prototypes():
    """Each ctypes declaration of the oracle's wrapper has its C prototype's parameter
    count and kinds (pointer, int, int64, uint64, double) and return kind."""
    import ctypes as C
    import re

    hdr = os.path.join(os.path.dirname(O.__file__), "atsfft_oracle.h")
    txt = re.sub(r"/\*.*?\*/", " ", open(hdr).read(), flags=re.S)
    protos = re.findall(r"^(void|int|int64_t|uint64_t)\s+(orc_[a-z0-9_]+)\s*\(([^;]*?)\)\s*;",
                        txt, flags=re.M | re.S)
    assert len(protos) >= 15

    def kind_of_decl(d):
        d = d.strip()
        if "*" in d:
            return "ptr"
        for t, k in (("uint64_t", "u64"), ("int64_t", "i64"), ("double", "f64"), ("int", "i32")):
            if re.match(rf"(const\s+)?{t}\b", d):
                return k
        raise AssertionError(d)

    def kind_of_ctype(a):
        if a is None:
            return "void"
        if isinstance(a, type) and issubclass(a, C._Pointer) or a in (C.c_void_p, C.c_char_p):
            return "ptr"
        return {C.c_int: "i32", C.c_int64: "i64", C.c_uint64: "u64", C.c_double: "f64"}[a]

    lib = O.lib()
    for ret, name, params in protos:
        fn = getattr(lib, name)
        decls = [p for p in params.split(",") if p.strip() and p.strip() != "void"]
        if fn.argtypes is not None or decls:
            assert fn.argtypes is not None, name
            assert [kind_of_ctype(a) for a in fn.argtypes] == [kind_of_decl(d) for d in decls], name
        want_ret = {"void": ("void", "i32"), "int": ("i32",), "int64_t": ("i64",),
                    "uint64_t": ("u64",)}[ret]
        assert kind_of_ctype(fn.restype) in want_ret, (name, ret, fn.restype)
