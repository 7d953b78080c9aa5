"""The seeded input generator produces what its recipe says (CPU only)."""

import numpy as np

from synth import l1_error_per_coefficient, sparse_signal_1d, sparse_signal_2d


def test_1d_exactly_sparse_and_seeded():
    s = sparse_signal_1d(4096, 12, 5)
    xh = np.fft.fft(s.x.astype(np.complex128))
    assert np.all(np.diff(s.support) > 0) and len(s.support) == 12
    assert np.allclose(xh[s.support], s.coeffs, atol=1e-5)
    off = np.delete(xh, s.support)
    assert np.max(np.abs(off)) < 1e-5
    assert np.allclose(np.abs(s.coeffs), 1.0)
    s2 = sparse_signal_1d(4096, 12, 5)
    assert np.array_equal(s.x, s2.x)


def test_noise_level_matches_snr():
    s = sparse_signal_1d(1 << 16, 50, 1, snr_db=40)
    xh = np.zeros(1 << 16, complex)
    xh[s.support] = s.coeffs
    clean = np.fft.ifft(xh)
    noise = s.x.astype(np.complex128) - clean
    snr = 10 * np.log10(np.mean(np.abs(clean) ** 2) / np.mean(np.abs(noise) ** 2))
    assert abs(snr - 40) < 0.2


def test_2d_loguniform_magnitudes():
    s = sparse_signal_2d(128, 40, 2, mag=("loguniform", 0.1, 1.0))
    xh = np.fft.fft2(s.x.astype(np.complex128)).ravel()
    assert np.allclose(xh[s.support], s.coeffs, atol=1e-5)
    m = np.abs(s.coeffs)
    assert m.min() >= 0.1 - 1e-12 and m.max() <= 1.0 + 1e-12


def test_l1_error_metric():
    s = sparse_signal_1d(1024, 3, 0)
    assert l1_error_per_coefficient(s, s.support, s.coeffs) == 0.0
    assert abs(l1_error_per_coefficient(s, s.support[:2], s.coeffs[:2]) - 1 / 3) < 1e-12
    e = l1_error_per_coefficient(s, np.r_[s.support, [0]], np.r_[s.coeffs, [0.5]])
    assert abs(e - (0.5 / 3 if 0 not in s.support else e)) < 1e-12


def test_spectrum_alone_is_the_signals_spectrum():
    from synth import sparse_spectrum_1d

    for n, k, seed, kw in [(4096, 12, 5, {}), (1 << 14, 40, 2, {"mag": ("loguniform", 0.1, 1.0)})]:
        s = sparse_signal_1d(n, k, seed, snr_db=30.0, **kw)
        support, coeffs = sparse_spectrum_1d(n, k, seed, **kw)
        assert np.array_equal(support, s.support) and np.array_equal(coeffs, s.coeffs)
