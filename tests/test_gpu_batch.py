"""Batched execution through one CUDA graph (atsfft_batch_*): every branch gives exactly
the outputs of the plain exec of its plan, and relaunches re-read the inputs.  Needs a GPU."""

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


def _outputs(torch, cap):
    return dict(loc=torch.empty(cap, dtype=torch.int64, device="cuda"),
                val=torch.empty(cap, dtype=torch.complex64, device="cuda"),
                count=torch.zeros(1, dtype=torch.int64, device="cuda"),
                k=torch.zeros(1, dtype=torch.int64, device="cuda"),
                status=torch.zeros(1, dtype=torch.int32, device="cuda"))


def _result(o):
    n = int(o["count"].item())
    m = min(n, o["loc"].numel())
    return (n, int(o["k"].item()), int(o["status"].item()), o["loc"][:m].cpu().numpy(),
            o["val"][:m].cpu().numpy())


def _same(a, b):
    assert a[:3] == b[:3]
    assert np.array_equal(a[3], b[3])
    assert np.array_equal(a[4], b[4])


def test_batch_matches_plain_execs_and_relaunches(A):
    import torch

    from synth import sparse_signal_1d, sparse_signal_2d

    cases = [((1 << 14,), sparse_signal_1d(1 << 14, 16, 11).x),
             ((1 << 18,), sparse_signal_1d(1 << 18, 200, 12, snr_db=40.0).x),
             ((256, 256), sparse_signal_2d(256, 10, 13).x)]
    cap = 1 << 12
    plans, xs, outs, refs = [], [], [], []
    for shape, x in cases:
        p = A.Plan(shape, seed=5)
        xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
        o = _outputs(torch, cap)
        p.exec_async(xd, o["loc"], o["val"], o["count"], o["k"], o["status"])
        torch.cuda.synchronize()
        refs.append(_result(o))
        plans.append(p)
        xs.append(xd)
        outs.append(_outputs(torch, cap))
    batch = A.Batch([(p, x, o["loc"], o["val"], o["count"], o["k"], o["status"])
                     for p, x, o in zip(plans, xs, outs)])
    assert batch.kernels() > 0
    for _ in range(2):
        batch.launch()
        torch.cuda.synchronize()
        for o, ref in zip(outs, refs):
            _same(_result(o), ref)
    # new input in place: the next launch transforms it
    x2 = sparse_signal_1d(1 << 14, 16, 99).x
    xs[0].copy_(torch.from_numpy(x2))
    o = _outputs(torch, cap)
    plans[0].exec_async(xs[0], o["loc"], o["val"], o["count"], o["k"], o["status"])
    torch.cuda.synchronize()
    ref2 = _result(o)
    batch.launch()
    torch.cuda.synchronize()
    _same(_result(outs[0]), ref2)
    batch.close()
    for p in plans:
        p.close()


def test_batch_rejects_duplicate_plans_and_profiling(A):
    import torch

    p = A.Plan((1 << 14,), seed=1)
    x = torch.zeros(1 << 14, dtype=torch.complex64, device="cuda")
    o = _outputs(torch, 16)
    item = (p, x, o["loc"], o["val"], o["count"], o["k"], o["status"])
    with pytest.raises(A.ATSFFTError):
        A.Batch([item, item])
    p.set_profiling(True)
    with pytest.raises(A.ATSFFTError):
        A.Batch([item])
    p.set_profiling(False)
    p.close()


def test_clone_gives_identical_transforms(A):
    import torch

    from synth import sparse_signal_1d, sparse_signal_2d

    for shape, x in [((1 << 16,), sparse_signal_1d(1 << 16, 40, 21, snr_db=40.0).x),
                     ((128, 128), sparse_signal_2d(128, 6, 22).x)]:
        p = A.Plan(shape, k_hint=8, seed=9)
        c = p.clone()
        xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
        ra = p(xd, capacity=1 << 10)
        p.close()   # the clone owns its tables
        rb = c(xd, capacity=1 << 10)
        assert ra[2:] == rb[2:]
        assert np.array_equal(ra[0].cpu().numpy(), rb[0].cpu().numpy())
        assert np.array_equal(ra[1].cpu().numpy(), rb[1].cpu().numpy())
        c.close()


def test_autotune_meets_the_error_target(A):
    """The candidate grid spans the loop counts, the window's alpha and the tuning's B
    range (Eqs. (8), (9), (14)); the choice is the fastest candidate that meets the Eq. (15)
    error target with k*/k in [0.9, 1.1]."""
    from paper_1908_02461_gb300.autotune import autotune, b_range_for

    n, kr = 1 << 16, (20, 64)
    assert b_range_for(n, kr, "k_range") == (6, 0)   # B from 2^6 >= 2 k_lo; top as default
    grid = {"loops": [(7, 7), (5, 5)], "filter_tol": [1e-6], "filter_alpha": [0.5, 1.0],
            "b_range": ["default", "k_range"], "tune_stages": [3]}
    res = autotune(n, k_range=kr, snr_db=40.0, error_target=1e-2, probes=2, reps=1, grid=grid)
    assert len(res.table) == 8
    assert {r[0]["filter_alpha"] for r in res.table} == {0.5, 1.0}
    assert {r[0]["b_min_log2"] for r in res.table} == {0, 6}
    assert res.error <= 1e-2 and 0.9 <= res.k_ratio <= 1.1
    assert res.ms_per_transform == min(r[1] for r in res.table if r[4])
    p = A.Plan((n,), params=A.params(**res.params))
    p.close()


def test_tail_grid_size_does_not_change_results(A):
    """The coop_* launch parameters (accepted for the ABI, without effect since the tail
    kernels stopped being cooperative grids) leave transforms bit-identical, also inside a
    batch graph."""
    import torch

    from synth import sparse_signal_1d, sparse_signal_2d

    cases = [((1 << 16,), sparse_signal_1d(1 << 16, 40, 31, snr_db=40.0).x),
             ((1 << 20,), sparse_signal_1d(1 << 20, 500, 32, snr_db=40.0).x),
             ((256, 256), sparse_signal_2d(256, 12, 33).x)]
    cap = 1 << 12
    small = A.params(coop_blocks_per_sm=1, coop_sms=19)
    plans, xs, outs, refs = [], [], [], []
    for shape, x in cases:
        xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
        ref = A.Plan(shape, seed=3)
        o = _outputs(torch, cap)
        ref.exec_async(xd, o["loc"], o["val"], o["count"], o["k"], o["status"])
        torch.cuda.synchronize()
        refs.append(_result(o))
        ref.close()
        p = A.Plan(shape, params=small, seed=3)
        o = _outputs(torch, cap)
        p.exec_async(xd, o["loc"], o["val"], o["count"], o["k"], o["status"])
        torch.cuda.synchronize()
        _same(_result(o), refs[-1])
        plans.append(p)
        xs.append(xd)
        outs.append(_outputs(torch, cap))
    batch = A.Batch([(p, x, o["loc"], o["val"], o["count"], o["k"], o["status"])
                     for p, x, o in zip(plans, xs, outs)])
    batch.launch()
    torch.cuda.synchronize()
    for o, ref in zip(outs, refs):
        _same(_result(o), ref)
    batch.close()
    for p in plans:
        p.close()
    with pytest.raises(A.ATSFFTError):
        A.Plan((1 << 14,), params=A.params(coop_sms=-1))


def test_io_batch_copies_and_matches_plain_execs(A):
    """atsfft_batch_create_io: the graph copies the inputs from pinned host memory (one
    chain, item order), runs the transforms and copies the outputs back; they equal the
    plain execs' outputs, and a relaunch transforms new host data written in place."""
    import torch

    from synth import sparse_signal_1d

    cases = [((1 << 16,), sparse_signal_1d(1 << 16, 30, 61, snr_db=40.0).x),
             ((1 << 18,), sparse_signal_1d(1 << 18, 300, 62, snr_db=40.0).x),
             ((1 << 14,), sparse_signal_1d(1 << 14, 16, 63).x)]
    cap = 1 << 12
    plans, xs, outs, host, refs = [], [], [], [], []
    for shape, x in cases:
        p = A.Plan(shape, seed=4)
        ref = p(torch.from_numpy(x).cuda(), capacity=cap)
        refs.append((ref[0].cpu().numpy(), ref[1].cpu().numpy(), ref[2], ref[3], ref[4]))
        plans.append(p)
        xs.append(torch.zeros(shape, dtype=torch.complex64, device="cuda"))
        outs.append(_outputs(torch, cap))
        host.append(dict(x=torch.from_numpy(x).pin_memory(),
                         loc=torch.zeros(cap, dtype=torch.int64).pin_memory(),
                         val=torch.zeros(cap, dtype=torch.complex64).pin_memory(),
                         count=torch.zeros(1, dtype=torch.int64).pin_memory(),
                         k=torch.zeros(1, dtype=torch.int64).pin_memory(),
                         status=torch.zeros(1, dtype=torch.int32).pin_memory()))
    batch = A.Batch([(p, x, o["loc"], o["val"], o["count"], o["k"], o["status"])
                     for p, x, o in zip(plans, xs, outs)], host=host)
    for _ in range(2):
        batch.launch()
        torch.cuda.synchronize()
        for h, (loc, val, k, st, cnt) in zip(host, refs):
            m = min(cnt, cap)
            assert int(h["count"][0]) == cnt and int(h["k"][0]) == k and int(h["status"][0]) == st
            assert np.array_equal(h["loc"][:m].numpy(), loc[:m])
            assert np.array_equal(h["val"][:m].numpy(), val[:m])
    # new host input in place: the next launch copies and transforms it
    x2 = sparse_signal_1d(1 << 14, 16, 99).x
    ref2 = plans[2](torch.from_numpy(x2).cuda(), capacity=cap)
    host[2]["x"].copy_(torch.from_numpy(x2))
    batch.launch()
    torch.cuda.synchronize()
    m = min(ref2[4], cap)
    assert int(host[2]["count"][0]) == ref2[4]
    assert np.array_equal(host[2]["loc"][:m].numpy(), ref2[0][:m].cpu().numpy())
    batch.close()
    with pytest.raises(ValueError):
        A.Batch([(plans[0], xs[0], outs[0]["loc"], outs[0]["val"], outs[0]["count"],
                  outs[0]["k"], outs[0]["status"])], host=[dict(x=torch.zeros(1 << 16, dtype=torch.complex64))])
    for p in plans:
        p.close()
