"""Seeded k-sparse test signals in the shape of the paper's workloads.

Section IV of the paper draws k frequencies at random, gives them magnitude 1
and leaves every other frequency at 0; the workloads here extend that recipe
with log-uniform magnitudes and complex Gaussian noise at a given SNR.

Conventions (Section II): the forward DFT is unscaled,
    xhat[f] = sum_t x[t] * exp(-2*pi*i*f*t/n),
so the time signal is x = ifft(xhat) = (1/n) sum_f xhat[f] exp(+2*pi*i*f*t/n).
Signals are produced in FP64 and returned as complex64 (what the GPU path
consumes); the FP64 oracle reads those same complex64 values widened to FP64.
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class SparseSignal:
    x: np.ndarray            # complex64, shape (n,) or (N, N)
    support: np.ndarray      # int64, ascending linear indices of the nonzero DFT bins
    coeffs: np.ndarray       # complex128, DFT values at `support` (noise-free spectrum)
    noise_var: float         # per-sample complex noise variance added in time domain


def _magnitudes(rng, k, mag):
    if mag == "unit":
        return np.ones(k)
    if isinstance(mag, tuple) and mag[0] == "loguniform":
        lo, hi = mag[1], mag[2]
        return np.exp(rng.uniform(np.log(lo), np.log(hi), size=k))
    raise ValueError(f"unknown magnitude law {mag!r}")


def _add_noise(rng, x, snr_db):
    if snr_db is None:
        return x, 0.0
    power = float(np.mean(np.abs(x) ** 2))
    var = power * 10.0 ** (-snr_db / 10.0)
    noise = rng.normal(0.0, np.sqrt(var / 2.0), size=x.shape + (2,))
    return x + (noise[..., 0] + 1j * noise[..., 1]), var


def _spectrum(rng, size, k, mag):
    support = np.sort(rng.choice(size, size=k, replace=False)).astype(np.int64)
    phases = rng.uniform(0.0, 2.0 * np.pi, size=k)
    mags = _magnitudes(rng, k, mag)
    return support, mags * np.exp(1j * phases)


def sparse_spectrum_1d(n: int, k: int, seed: int, mag="unit"):
    """(support, coeffs) of `sparse_signal_1d(n, k, seed, mag=mag)` without forming the
    signal (the same draws, so the same spectrum)."""
    return _spectrum(np.random.default_rng(seed), n, k, mag)


def sparse_signal_1d(n: int, k: int, seed: int, snr_db: float | None = None,
                     mag="unit", dtype=np.complex64) -> SparseSignal:
    """n-sample signal whose DFT has exactly k nonzero bins (plus optional noise).

    Locations: k distinct values drawn uniformly from [0, n); phases uniform in
    [0, 2*pi); magnitudes 1 ("unit") or ("loguniform", lo, hi).  The samples are
    computed in FP64 and stored as `dtype` (complex64 by default).
    """
    rng = np.random.default_rng(seed)
    support, coeffs = _spectrum(rng, n, k, mag)
    xhat = np.zeros(n, dtype=np.complex128)
    xhat[support] = coeffs
    x = np.fft.ifft(xhat)
    x, var = _add_noise(rng, x, snr_db)
    return SparseSignal(x.astype(dtype), support, coeffs, var)


def sparse_signal_2d(N: int, k: int, seed: int, snr_db: float | None = None,
                     mag="unit", dtype=np.complex64) -> SparseSignal:
    """N x N image whose 2D DFT has exactly k nonzero bins at distinct (u, v).

    The support is returned as linear indices u*N + v (row-major); the pixels are
    computed in FP64 and stored as `dtype` (complex64 by default).
    """
    rng = np.random.default_rng(seed)
    support, coeffs = _spectrum(rng, N * N, k, mag)
    xhat = np.zeros(N * N, dtype=np.complex128)
    xhat[support] = coeffs
    x = np.fft.ifft2(xhat.reshape(N, N))
    x, var = _add_noise(rng, x, snr_db)
    return SparseSignal(x.astype(dtype), support, coeffs, var)


def l1_error_per_coefficient(sig: SparseSignal, loc: np.ndarray, val: np.ndarray) -> float:
    """Eq. (15): (1/k) * sum over the whole grid of |xhat' - xhat|.

    xhat is the generator's noise-free sparse spectrum; xhat' is zero outside
    the reported locations.
    """
    k = len(sig.support)
    truth = dict(zip(sig.support.tolist(), sig.coeffs.tolist()))
    err = 0.0
    seen = set()
    for i, v in zip(np.asarray(loc).tolist(), np.asarray(val).tolist()):
        err += abs(v - truth.get(i, 0.0))
        seen.add(i)
    for i, c in truth.items():
        if i not in seen:
            err += abs(c)
    return err / max(k, 1)
