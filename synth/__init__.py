"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke run.

This module only draws test signals: a k-sparse spectrum (distinct random
locations, chosen magnitudes, uniform phases), its inverse DFT, and additive
complex Gaussian noise at a stated SNR.  It holds none of the sparse-FFT
arithmetic, so both the CUDA path and the FP64 oracle can consume its output
without sharing any of the method's code.
"""

from .signals import (  # noqa: F401
    SparseSignal,
    sparse_signal_1d,
    sparse_spectrum_1d,
    sparse_signal_2d,
    l1_error_per_coefficient,
)
