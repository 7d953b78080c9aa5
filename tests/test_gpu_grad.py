"""Gradients through the transform at a fixed recovered support (1D): the forward map of
Eq. (11) against the FP64 oracle, the adjoint against the forward map (dot products),
autograd against FP64 central differences, and the dense-DFT rows at the support.
Needs a GPU."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def A():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1908_02461_gb300 as A

    A.build()
    return A


@pytest.fixture(scope="module")
def O():
    import oracle

    oracle.build()
    return oracle


def _case(A, n, k, seed, snr=None):
    import torch

    from synth import sparse_signal_1d

    sig = sparse_signal_1d(n, k, seed, snr_db=snr)
    plan = A.Plan((n,), seed=seed)
    x = torch.from_numpy(sig.x).cuda()
    loc, val, msel, B, kk, st, cnt = plan.exec_sel(x, capacity=1 << 12)
    assert cnt == loc.numel() and cnt > 0
    return sig, plan, x, loc, val, msel, B


def _rand_c(rng, shape, dtype=np.complex128):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(dtype)


def _selected(est, msel):
    """(Re est[lr], Im est[li]) per coordinate from the oracle's [count, L] estimates."""
    r = np.arange(len(est))
    return est[r, msel[:, 0]].real + 1j * est[r, msel[:, 1]].imag


CASES = [(1 << 12, 8, 3, None), (1 << 14, 16, 4, 40.0), (1 << 18, 60, 5, 40.0)]


@pytest.mark.parametrize("n,k,seed,snr", CASES)
def test_exec_sel_and_apply_reproduce_the_transform(A, n, k, seed, snr):
    import torch

    sig, plan, x, loc, val, msel, B = _case(A, n, k, seed, snr)
    loc2, val2, k2, st2, cnt2 = plan(x, capacity=1 << 12)
    assert torch.equal(loc, loc2) and torch.equal(val, val2)
    m = msel.cpu().numpy()
    assert m.min() >= 0 and m.max() < 7
    y = plan.estimate_apply(B, x, loc, msel)
    ref = val.cpu().numpy()
    err = np.abs(y.cpu().numpy() - ref).max() / np.abs(ref).max()
    assert err < 1e-5, err
    plan.close()


@pytest.mark.parametrize("n,k,seed,snr", CASES)
def test_apply_matches_fp64_oracle(A, O, n, k, seed, snr):
    import torch

    sig, plan, x, loc, val, msel, B = _case(A, n, k, seed, snr)
    rng = np.random.default_rng(seed)
    u = _rand_c(rng, n)
    got = plan.estimate_apply(B, torch.from_numpy(u.astype(np.complex64)).cuda(), loc, msel)
    est = O.estimates_1d(u.astype(np.complex64), B, loc.cpu().numpy(), seed=seed)
    ref = _selected(est, msel.cpu().numpy())
    err = np.abs(got.cpu().numpy() - ref).max() / np.abs(ref).max()
    assert err < 1e-4, err
    plan.close()


@pytest.mark.parametrize("n,k,seed,snr", CASES)
def test_adjoint_dot_product(A, n, k, seed, snr):
    import torch

    sig, plan, x, loc, val, msel, B = _case(A, n, k, seed, snr)
    rng = np.random.default_rng(seed + 1)
    for _ in range(3):
        u = torch.from_numpy(_rand_c(rng, n, np.complex64)).cuda()
        g = torch.from_numpy(_rand_c(rng, loc.numel(), np.complex64)).cuda()
        Ju = plan.estimate_apply(B, u, loc, msel).cpu().numpy().astype(np.complex128)
        JTg = plan.estimate_adjoint(B, loc, msel, g).cpu().numpy().astype(np.complex128)
        lhs = np.real(np.vdot(g.cpu().numpy().astype(np.complex128), Ju))
        rhs = np.real(np.vdot(JTg, u.cpu().numpy().astype(np.complex128)))
        scale = np.linalg.norm(Ju) * np.linalg.norm(g.cpu().numpy())
        assert abs(lhs - rhs) <= 1e-5 * scale, (lhs, rhs, scale)
    plan.close()


def test_autograd_against_fp64_central_differences(A, O):
    """n = 2^12, k = 8: L(x) = sum |y(x) - t|^2, y the transform's values; the autograd
    gradient's directional derivatives against central differences of the FP64 oracle's
    estimates at the same support and selections."""
    import torch

    n, k, seed = 1 << 12, 8, 3
    sig, plan, x, loc, val, msel, B = _case(A, n, k, seed)
    rng = np.random.default_rng(9)
    t = _rand_c(rng, loc.numel()) * 0.5
    xr = x.clone().requires_grad_(True)
    loc_a, y = A.sparse_fft(xr, plan, 1 << 12)
    assert torch.equal(loc_a, loc)
    tt = torch.from_numpy(t.astype(np.complex64)).cuda()
    L = ((y - tt).abs() ** 2).sum()
    (gx,) = torch.autograd.grad(L, xr)
    gx = gx.cpu().numpy().astype(np.complex128)
    m = msel.cpu().numpy()
    lc = loc.cpu().numpy()
    x64 = sig.x.astype(np.complex128)

    def loss64(z):
        est = O.estimates_1d(z, B, lc, seed=seed)   # FP64 (the input widened)
        return float(np.sum(np.abs(_selected(est, m) - t) ** 2))

    for _ in range(3):
        d = _rand_c(rng, n)
        eps = 1e-3
        fd = (loss64(x64 + eps * d) - loss64(x64 - eps * d)) / (2 * eps)
        an = float(np.real(np.vdot(gx, d)))
        assert abs(an - fd) <= 1e-3 * max(abs(fd), 1e-3 * np.linalg.norm(gx) * np.linalg.norm(d)), (an, fd)
    plan.close()


def test_rows_at_the_support_are_dft_rows_on_sparse_inputs(A):
    """For an exactly sparse signal the estimate at its support equals the dense DFT
    there (Jx = F_S x), and so does the map applied to another signal with the same
    support."""
    import torch

    from synth import sparse_signal_1d

    n, k, seed = 1 << 14, 16, 7
    sig, plan, x, loc, val, msel, B = _case(A, n, k, seed)
    lc = loc.cpu().numpy()
    true = np.isin(lc, sig.support)          # recovered points on the true support
    assert true.sum() >= 0.9 * k
    X = np.fft.fft(sig.x.astype(np.complex128))
    y = plan.estimate_apply(B, x, loc, msel).cpu().numpy()
    assert np.abs(y - X[lc])[true].max() <= 1e-4 * np.abs(X[lc]).max()
    # a different signal on the same support
    rng = np.random.default_rng(1)
    spec = np.zeros(n, complex)
    spec[sig.support] = _rand_c(rng, k)
    u = np.fft.ifft(spec)
    yu = plan.estimate_apply(B, torch.from_numpy(u.astype(np.complex64)).cuda(), loc, msel)
    assert np.abs(yu.cpu().numpy() - spec[lc])[true].max() <= 1e-4 * np.abs(spec).max()
    plan.close()
