"""CPU check of the location tail's fixed-width index arithmetic at every size the plan
accepts (1D n up to 2^28, 2D N up to 2^14): the kernel's 32-bit forms (products wrap
mod 2^32, which n divides) against exact integer arithmetic, and the property the votes
rest on: every preimage of bucket c hashes back to c (Section II-B reverse hash; Eq.
(10) with the half-bin reading)."""

import random

import pytest

M32 = 0xFFFFFFFF


def bucket_of_u32(i, sigma, logn, logB):
    """The kernel's bucket of coordinate i: round((sigma i mod n + 1/2) / D) mod B in
    32-bit unsigned arithmetic."""
    nmask, D = (1 << logn) - 1, 1 << (logn - logB)
    p = ((sigma * i) & M32) & nmask
    t = (2 * p + 1 + D) & M32
    assert t == 2 * p + 1 + D          # no wrap: 2p + 1 + D < 2^30 for n <= 2^28
    return (t >> (logn - logB + 1)) & ((1 << logB) - 1)


def bucket_shift_u32(i, sigma, logn, logB):
    """The votes kernel's form of the same bucket: ((sigma i + D/2) mod n) >> log2 D in
    32-bit unsigned arithmetic (floor((2p + 1 + D) / 2D) = floor((p + D/2) / D) for
    integers p, D >= 2, and the reduction mod n commutes with the shift mod B, n = B D)."""
    nmask, logD = (1 << logn) - 1, logn - logB
    return ((((sigma * i) & M32) + (1 << (logD - 1))) & M32 & nmask) >> logD


def preimage_u32(c, q, sinv, logn, logB):
    """The kernel's q-th preimage of bucket c: sigma^{-1} (c D - D/2 + q) mod n, 32-bit."""
    nmask, logD = (1 << logn) - 1, logn - logB
    D = 1 << logD
    pp = (((c << logD) & M32) - (D >> 1) + q) & M32 & nmask
    return ((sinv * pp) & M32) & nmask


def _inv(sigma, n):
    return pow(sigma, -1, n)


@pytest.mark.parametrize("logn", [8, 14, 22, 26, 28])
def test_1d_bucket_and_preimages_match_exact_arithmetic(logn):
    rng = random.Random(logn)
    n = 1 << logn
    for logB in sorted({4, (4 + logn - 4) // 2, logn - 4}):
        B, D = 1 << logB, 1 << (logn - logB)
        for _ in range(200):
            sigma = rng.randrange(n) | 1
            sinv = _inv(sigma, n)
            i = rng.randrange(n)
            p = sigma * i % n
            assert bucket_of_u32(i, sigma, logn, logB) == ((2 * p + 1 + D) // (2 * D)) % B
            assert bucket_shift_u32(i, sigma, logn, logB) == ((2 * p + 1 + D) // (2 * D)) % B
            c, q = rng.randrange(B), rng.randrange(D)
            coord = preimage_u32(c, q, sinv, logn, logB)
            assert coord == sinv * ((c * D - D // 2 + q) % n) % n
            assert bucket_of_u32(coord, sigma, logn, logB) == c
            assert bucket_shift_u32(coord, sigma, logn, logB) == c
        # the D preimages of a bucket are distinct and all hash back to it (small D only)
        if D <= 4096:
            sigma = rng.randrange(n) | 1
            sinv = _inv(sigma, n)
            c = rng.randrange(B)
            pre = {preimage_u32(c, q, sinv, logn, logB) for q in range(D)}
            assert len(pre) == D
            assert all(bucket_of_u32(x, sigma, logn, logB) == c for x in pre)
            assert all(bucket_shift_u32(x, sigma, logn, logB) == c for x in pre)


@pytest.mark.parametrize("logN", [5, 10, 14])
def test_2d_coordinates_fit_and_hash_back(logN):
    """2D: coordinate i N + j < 2^28 packed in 32 bits; each axis's preimage hashes back."""
    rng = random.Random(100 + logN)
    N = 1 << logN
    for logB in sorted({3, logN - 2}):
        B, D = 1 << logB, 1 << (logN - logB)
        for _ in range(200):
            s1, s2 = rng.randrange(N) | 1, rng.randrange(N) | 1
            c1, c2, q1, q2 = rng.randrange(B), rng.randrange(B), rng.randrange(D), rng.randrange(D)
            i = preimage_u32(c1, q1, _inv(s1, N), logN, logB)
            j = preimage_u32(c2, q2, _inv(s2, N), logN, logB)
            coord = ((i << logN) | j) & M32
            assert coord == i * N + j < 1 << 28
            assert bucket_of_u32(coord >> logN, s1, logN, logB) == c1
            assert bucket_of_u32(coord & (N - 1), s2, logN, logB) == c2
            assert bucket_shift_u32(coord >> logN, s1, logN, logB) == c1
            assert bucket_shift_u32(coord & (N - 1), s2, logN, logB) == c2


def test_shift_form_equals_half_bin_rule_exhaustively_small_n():
    """Every coordinate, odd sigma and bucket count at n = 2^8: the two bucket forms agree."""
    logn = 8
    n = 1 << logn
    for logB in range(1, logn):
        for sigma in range(1, n, 2):
            for i in range(n):
                assert bucket_shift_u32(i, sigma, logn, logB) == bucket_of_u32(i, sigma, logn, logB)
