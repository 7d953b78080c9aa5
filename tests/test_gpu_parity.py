"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.  Needs a GPU.

Tolerances (the 1e-4 value bar of the hot path, and FP32 arithmetic):
  * window tables Ghat': both sides FP64, 1e-9 absolute;
  * bucket spectra (permute + window + bin + bucket FFT, FP32 on the GPU):
    max |Zhat_gpu - Zhat_oracle| <= 2e-5 * max |Zhat_oracle| (errors of FP32 taps and
    sums scale with the bucket energies, not with each bucket);
  * whole transforms (tests/_parity.py): the tuning trajectory, k*, status, count and
    locations identical, values |v_gpu - v_oracle| <= 1e-4 * max(|v_oracle|,
    max_i |v_oracle_i|/100); a discrete difference passes only when it traces back to a
    decision the oracle logged within 2e-4 of its boundary (where FP32 and FP64 energies
    can decide differently).
"""

import numpy as np
import pytest

from _parity import BAND, check, value_error

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


def _cuda(x):
    import torch

    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _check_transform(A, O, x, seed, ndim, params_kw=None, capacity=1 << 16, k_hint=0):
    params_kw = params_kw or {}
    shape = x.shape
    plan = A.Plan(shape, k_hint=k_hint, params=A.params(**params_kw), seed=seed)
    loc, val, k, status, count = plan(_cuda(x), capacity=capacity)
    trace = plan.last_trace()
    plan.close()
    ref, dec = O.atsfft_log(x, k_hint=k_hint, params=O.default_params(**params_kw), seed=seed,
                            capacity=capacity, band=BAND)
    gpu = dict(trace=trace, k=k, status=status, count=count, loc=loc.cpu().numpy(),
               val=val.cpu().numpy())
    info = check(gpu, ref, dec, shape, seed, loops_loc=params_kw.get("loops_loc", 7),
                 capacity=capacity)
    info.update(k_gpu=k, k_ref=ref.k_star, count_gpu=count, count_ref=ref.count)
    info["status"] = (status, ref.status)
    print(f"[{'exact' if info.get('exact') else 'attributed'}] {shape} {info}")
    return info, info.get("value_err")


# --------------------------------------------------------------------------
# a0: window tables
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n,Bs", [(1 << 14, [16, 64, 256, 1024]), (1 << 22, [4096, 65536, 262144])])
def test_window_response_tables(A, O, n, Bs):
    plan = A.Plan((n,), seed=0)
    for B in Bs:
        got = plan.window_response(B)
        ref = O.filter_response(n, B)
        assert np.max(np.abs(got - ref)) < 1e-9, B
    plan.close()


def test_window_response_tables_2d(A, O):
    plan = A.Plan((256, 256), seed=0)
    for B in (8, 16, 64):
        assert np.max(np.abs(plan.window_response(B) - O.filter_response(256, B))) < 1e-9
    plan.close()


# --------------------------------------------------------------------------
# a1-a3: permute + window + bin + bucket FFT, per hash
# --------------------------------------------------------------------------

def _spectrum_case(A, O, x, B, seed, phase, index, ndim):
    plan = A.Plan(x.shape, seed=seed)
    got = plan.hash_spectrum(_cuda(x), B, phase, index).cpu().numpy()
    plan.close()
    fn = O.hash_spectrum_1d if ndim == 1 else O.hash_spectrum_2d
    ref = fn(x, B, seed, phase, index)
    return float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))


@pytest.mark.parametrize("B", [16, 32, 128, 512, 1024])
def test_hash_spectrum_small(A, O, B):
    from synth import sparse_signal_1d

    sig = sparse_signal_1d(1 << 14, 16, 3)
    for phase, index in [(0, int(np.log2(B))), (1, 0), (1, 5), (2, 3)]:
        rel = _spectrum_case(A, O, sig.x, B, 3, phase, index, 1)
        assert rel < 2e-5, (B, phase, index, rel)


@pytest.mark.parametrize("B", [16, 4096, 16384, 65536, 262144])
def test_hash_spectrum_full_size(A, O, B):
    """n = 2^22 (the bench size): gather form below, residue stream above a fifth of n."""
    from synth import sparse_signal_1d

    sig = sparse_signal_1d(1 << 22, 1000, 11, snr_db=40)
    rel = _spectrum_case(A, O, sig.x, B, 11, 1, 2, 1)
    assert rel < 2e-5, (B, rel)


@pytest.mark.parametrize("N,B", [(64, 8), (256, 16), (256, 64), (1024, 256)])
def test_hash_spectrum_2d(A, O, N, B):
    from synth import sparse_signal_2d

    sig = sparse_signal_2d(N, 20, 4, snr_db=30, mag=("loguniform", 0.1, 1.0))
    for phase, index in [(0, int(np.log2(B))), (1, 1), (2, 0)]:
        rel = _spectrum_case(A, O, sig.x, B, 4, phase, index, 2)
        assert rel < 2e-5, (N, B, phase, rel)


# --------------------------------------------------------------------------
# whole transforms
# --------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(6))
def test_config1_exactly_sparse(A, O, seed):
    """n = 2^14, k = 16, unit magnitudes, no noise; k unknown to the solver."""
    from synth import sparse_signal_1d

    sig = sparse_signal_1d(1 << 14, 16, seed)
    _check_transform(A, O, sig.x, seed, 1)


@pytest.mark.parametrize("n,k,seed", [(1 << 16, 50, 1), (1 << 18, 200, 2), (1 << 12, 4, 3)])
def test_noisy_1d_mid(A, O, n, k, seed):
    from synth import sparse_signal_1d

    sig = sparse_signal_1d(n, k, seed, snr_db=40)
    _check_transform(A, O, sig.x, seed, 1)


@pytest.mark.parametrize("k,seed,D", [(250, 52, 128), (400, 57, 64), (800, 54, 32), (1500, 56, 16)])
def test_location_binning_forms(A, O, k, seed, D):
    """n = 2^20, 40 dB, signals whose B* (the oracle's) puts D = n / B* at 128, 64, 32 and
    16: the column form of the location pass, whose tile holds 1024 / D whole columns (8,
    16, 32 and 64: four lanes per column, two, one, and two columns per lane).  The whole
    transform against the oracle, and B* as the oracle's."""
    from synth import sparse_signal_1d

    n = 1 << 20
    sig = sparse_signal_1d(n, k, seed, snr_db=40)
    plan = A.Plan((n,), params=A.params(), seed=5)
    plan(_cuda(sig.x), capacity=1 << 16)
    b_star = plan.last_trace()[-1][0]
    plan.close()
    assert n // b_star == D
    _check_transform(A, O, sig.x, 5, 1)


@pytest.mark.parametrize("k", [50, 200, 1000, 2000])
def test_config2_full_size(A, O, k):
    """n = 2^22, 40 dB, the sweep of the benchmark."""
    from synth import sparse_signal_1d

    sig = sparse_signal_1d(1 << 22, k, 100 + k, snr_db=40)
    _check_transform(A, O, sig.x, 7, 1)


@pytest.mark.parametrize("N,k,seed", [(128, 6, 2), (256, 10, 0), (1024, 100, 5)])
def test_2d_small(A, O, N, k, seed):
    from synth import sparse_signal_2d

    sig = sparse_signal_2d(N, k, seed, snr_db=30, mag=("loguniform", 0.1, 1.0))
    _check_transform(A, O, sig.x, seed, 2)


def test_config3_full_size(A, O):
    """4096 x 4096, k = 1000, log-uniform magnitudes, 30 dB."""
    from synth import sparse_signal_2d

    sig = sparse_signal_2d(4096, 1000, 5, snr_db=30, mag=("loguniform", 0.1, 1.0))
    _check_transform(A, O, sig.x, 7, 2)


# --------------------------------------------------------------------------
# degenerate cases and limits
# --------------------------------------------------------------------------

def test_zero_signal(A, O):
    x = np.zeros(1 << 14, np.complex64)
    plan = A.Plan(x.shape, seed=0)
    loc, val, k, status, count = plan(_cuda(x))
    assert (k, status, count) == (0, 0, 0)
    plan.close()
    x2 = np.zeros((64, 64), np.complex64)
    plan2 = A.Plan(x2.shape, seed=0)
    loc, val, k, status, count = plan2(_cuda(x2))
    assert (k, status, count) == (0, 0, 0)
    plan2.close()


def test_capacity_too_small(A, O):
    from synth import sparse_signal_1d

    sig = sparse_signal_1d(1 << 14, 16, 1)
    info, _ = _check_transform(A, O, sig.x, 1, 1, capacity=3)
    assert info["status"] == (6, 6) and info["count_gpu"] >= 16


def test_capacity_zero(A, O):
    from synth import sparse_signal_1d

    sig = sparse_signal_1d(1 << 14, 16, 1)
    plan = A.Plan(sig.x.shape, seed=1)
    loc, val, k, status, count = plan(_cuda(sig.x), capacity=0)
    assert status == 6 and count >= 16 and len(loc) == 0
    plan.close()


def test_not_converged_and_hint(A, O):
    from synth import sparse_signal_1d

    sig = sparse_signal_1d(1 << 16, 50, 3, snr_db=40)
    info, _ = _check_transform(A, O, sig.x, 3, 1, params_kw={"tune_max": 2})
    assert info["status"] == (4, 4)
    _check_transform(A, O, sig.x, 3, 1, k_hint=50)


def test_pure_noise_not_sparse(A, O):
    rng = np.random.default_rng(0)
    x = (rng.normal(size=1 << 14) + 1j * rng.normal(size=1 << 14)).astype(np.complex64)
    info, _ = _check_transform(A, O, x, 0, 1)
    assert info["status"] == (5, 5)


def test_smallest_and_custom_range(A, O):
    from synth import sparse_signal_1d

    sig = sparse_signal_1d(256, 2, 0)
    _check_transform(A, O, sig.x, 0, 1)
    sig = sparse_signal_1d(1 << 15, 20, 9, snr_db=40)
    _check_transform(A, O, sig.x, 9, 1, params_kw={"b_min_log2": 6, "b_max_log2": 10,
                                                   "loops_loc": 5, "loops_est": 9})


def test_exec_argument_errors(A):
    import torch

    plan = A.Plan((1 << 14,), seed=0)
    x = torch.zeros(1 << 14, dtype=torch.complex64, device="cuda")
    out = torch.zeros(4, dtype=torch.int64, device="cuda")
    assert A.atsfft_exec(plan.handle, x, out, out, -1, out, out, out, None) == A.E_INVALID_ARG
    assert A.atsfft_exec_2d(plan.handle, x, out, out, 4, out, out, out, None) == A.E_INVALID_ARG
    assert A.atsfft_exec(plan.handle, 0, out, out, 4, out, out, out, None) == A.E_INVALID_ARG
    plan.close()


# --------------------------------------------------------------------------
# Modes: fixed-k (no tuning) and estimation reusing the location hashes
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n,k,seed,snr", [(1 << 14, 16, 2, None), (1 << 22, 1000, 2000, 40.0)])
def test_fixed_k_mode(A, O, n, k, seed, snr):
    from synth import sparse_signal_1d

    sig = sparse_signal_1d(n, k, seed, snr_db=snr)
    info, _ = _check_transform(A, O, sig.x, 7, 1, params_kw={"fixed_k": 1}, k_hint=k)
    assert info["k_gpu"] == k


def test_fixed_k_mode_2d(A, O):
    from synth import sparse_signal_2d

    sig = sparse_signal_2d(256, 10, 4)
    info, _ = _check_transform(A, O, sig.x, 4, 2, params_kw={"fixed_k": 1}, k_hint=10)
    assert info["k_gpu"] == 10


@pytest.mark.parametrize("n,k,seed,snr", [(1 << 14, 16, 3, None), (1 << 22, 200, 1200, 40.0)])
def test_estimation_reusing_location_hashes(A, O, n, k, seed, snr):
    from synth import sparse_signal_1d

    sig = sparse_signal_1d(n, k, seed, snr_db=snr)
    _check_transform(A, O, sig.x, 7, 1, params_kw={"est_reuse_loc": 1})


# --------------------------------------------------------------------------
# FP64 path (precision 1): complex128 input, values to ~1e-12 of the FP64 oracle
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n,k,seed,snr", [(1 << 14, 16, 2, None), (1 << 16, 40, 21, 40.0),
                                          (1 << 20, 300, 5, 40.0)])
def test_fp64_path_values(A, O, n, k, seed, snr):
    import torch

    from synth import sparse_signal_1d

    sig = sparse_signal_1d(n, k, seed, snr_db=snr, dtype=np.complex128)
    plan = A.Plan((n,), params=A.params(precision=1), seed=7)
    x = torch.from_numpy(sig.x).cuda()
    loc, val, kk, st, cnt = plan(x, capacity=1 << 14)
    assert val.dtype == torch.complex128
    trace = plan.last_trace()
    plan.close()
    ref = O.atsfft_1d(sig.x, seed=7, capacity=1 << 14)
    # decisions as in the FP32 path (on the input rounded to complex64), by the parity rule
    x32 = sig.x.astype(np.complex64)
    ref32, dec = O.atsfft_log(x32, seed=7, capacity=1 << 14, band=BAND)
    loc = loc.cpu().numpy()
    v = val.cpu().numpy()
    gpu = dict(trace=trace, k=kk, status=st, count=cnt, loc=loc, val=v.astype(np.complex64))
    info = check(gpu, ref32, dec, (n,), 7, capacity=1 << 14)
    # values: the FP64 oracle on the complex128 input; its decisions are those of the
    # FP64 energies, so the comparison is over the locations both kept
    assert ref.loc.tolist() == ref32.loc.tolist() or "attributed" in info
    common, ig, ir = np.intersect1d(loc, ref.loc, return_indices=True)
    assert len(common) > 0
    err = np.abs(v[ig] - ref.val[ir]).max() / np.abs(ref.val).max()
    print(f"[fp64] n={n} k*={kk} count={cnt} value err={err:.1e} {info}")
    assert err < 1e-10, err


@pytest.mark.parametrize("N,k,seed,snr", [(256, 10, 4, None), (1024, 100, 5, 30.0)])
def test_fp64_path_values_2d(A, O, N, k, seed, snr):
    """The FP64 path on images: locations by the FP32 stages on the rounded input (the
    parity rule against the oracle on that input), values within 1e-10 of the FP64
    oracle's on the complex128 input (Eq. (11) in 2D with the separable window)."""
    import torch

    from synth import sparse_signal_2d

    sig = sparse_signal_2d(N, k, seed, snr_db=snr, mag=("loguniform", 0.1, 1.0),
                           dtype=np.complex128)
    plan = A.Plan((N, N), params=A.params(precision=1), seed=7)
    loc, val, kk, st, cnt = plan(torch.from_numpy(sig.x).cuda(), capacity=1 << 14)
    assert val.dtype == torch.complex128
    trace = plan.last_trace()
    plan.close()
    ref = O.atsfft_2d(sig.x, seed=7, capacity=1 << 14)
    ref32, dec = O.atsfft_log(sig.x.astype(np.complex64), seed=7, capacity=1 << 14, band=BAND)
    loc = loc.cpu().numpy()
    v = val.cpu().numpy()
    gpu = dict(trace=trace, k=kk, status=st, count=cnt, loc=loc, val=v.astype(np.complex64))
    info = check(gpu, ref32, dec, (N, N), 7, capacity=1 << 14)
    common, ig, ir = np.intersect1d(loc, ref.loc, return_indices=True)
    assert len(common) > 0
    err = np.abs(v[ig] - ref.val[ir]).max() / np.abs(ref.val).max()
    print(f"[fp64 2d] N={N} k*={kk} count={cnt} value err={err:.1e} {info}")
    assert err < 1e-10, err


def test_fp64_plan_rejects_fp32_entries(A):
    """hash_spectrum and the fixed-support estimate map read complex64 input: an FP64
    plan refuses them with an argument error before any launch."""
    import torch

    n = 1 << 14
    plan = A.Plan((n,), params=A.params(precision=1), seed=7)
    x = torch.zeros(n, dtype=torch.complex64, device="cuda")
    loc = torch.zeros(1, dtype=torch.int64, device="cuda")
    msel = torch.zeros(2, dtype=torch.uint8, device="cuda")
    with pytest.raises(A.ATSFFTError):
        plan.hash_spectrum(x, 64, 1, 0)
    with pytest.raises(A.ATSFFTError):
        plan.estimate_apply(64, x, loc, msel)
    with pytest.raises(A.ATSFFTError):
        plan.estimate_adjoint(64, loc, msel, torch.zeros(1, dtype=torch.complex64, device="cuda"))
    plan.close()


@pytest.mark.parametrize("n,k,seed", [(1 << 20, 50, 41), (1 << 20, 4000, 42), (1 << 22, 2000, 43),
                                      (1 << 16, 1500, 44)])
def test_tuning_stages_give_identical_transforms(A, n, k, seed):
    """One, two or three tuning batches (Algorithm 2's trials evaluated up front, or in
    stages that run only while the controller has not stopped) give bit-identical
    trajectories and outputs; the cases walk to the last trial or stop before it."""
    from synth import sparse_signal_1d

    sig = sparse_signal_1d(n, k, seed, snr_db=40.0)
    x = _cuda(sig.x)
    res = []
    for stages in (1, 2, 3):
        plan = A.Plan((n,), params=A.params(tune_stages=stages), seed=5)
        loc, val, kk, st, cnt = plan(x, capacity=1 << 14)
        res.append((plan.last_trace(), kk, st, cnt, loc.cpu().numpy(), val.cpu().numpy()))
        plan.close()
    for r in res[1:]:
        assert r[:4] == res[0][:4]
        assert np.array_equal(r[4], res[0][4])
        assert np.array_equal(r[5], res[0][5])
    print(f"[stages] n={n} k={k} trials={len(res[0][0])} last B={res[0][0][-1][0]} status={res[0][2]}")
