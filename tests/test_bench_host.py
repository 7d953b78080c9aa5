"""Host-side logic of bench.py: the max-over-ranks aggregation (gloo, two ranks on CPU)
and the roofline model's bookkeeping."""

import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    v = bench.aggregate(10.0 + 5.0 * rank, world)
    q.put((rank, v))
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_max_over_two_gloo_ranks():
    import multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    got = dict(q.get(timeout=10) for _ in range(2))
    assert got == {0: 15.0, 1: 15.0}


def test_aggregate_single_rank_is_identity():
    import bench

    assert bench.aggregate(3.5, 1) == 3.5


def test_roofline_model_picks_dominant_phase():
    import bench

    n = 1 << 22
    ph = {"tune1_bin": 0.02, "tune1_fft": 0.01, "tune1_tail": 0.02, "tune2_bin": 0.03,
          "tune2_fft": 0.03, "tune2_tail": 0.02, "tune3_bin": 0.01, "tune3_fft": 0.01,
          "tune3_tail": 0.01, "le_bin_stream": 0.06, "le_bin_gather": 0.006,
          "le_fft": 0.035, "loc_tail": 0.12}
    traces = {2000: [(16, 0), (65536, 1900)]}
    roof, rows = bench.roofline({2000: ph}, traces, n)
    assert roof["kernel"] == "loc_tail" and roof["bound"] == "hbm"
    assert roof["kernels"] == "k_loc_select + k_loc_votes + k_loc_finish"
    # the location tail: 8 B* per location hash, 4 k* D per location hash for the votes,
    # 8 bytes per kept coordinate and estimation hash
    B = 65536
    loc_bytes = 7 * B * 8 + 7 * 4 * 1900 * (n // B)
    assert rows["loc_tail"]["achieved"] == pytest.approx(loc_bytes / 0.12e-3 / 1e9)
    _, rows_k = bench.roofline({2000: ph}, traces, n, kept={2000: 2100})
    assert rows_k["loc_tail"]["achieved"] == pytest.approx((loc_bytes + 8 * 7 * 2100) / 0.12e-3 / 1e9)
    assert rows["le_bin_stream"]["bound"] == "alu"
    # the column form at B* = 2^16 (D = 64): 14 hashes x the window's 2h + 1 taps, with
    # h = 1152809 at the default alpha = 0.5, tol = 1e-6 (Eqs. (8)-(9)), in 0.06 ms
    assert rows["le_bin_stream"]["achieved"] == pytest.approx(14 * 2305619 / 0.06e-3 / 1e9)
    # at B* = 2^18 (D = 16) the window is clamped to n - 1 taps: every sample meets every
    # hash's window
    tr16 = {2000: [(16, 0), (1 << 18, 1900)]}
    _, rows16 = bench.roofline({2000: ph}, tr16, n)
    assert rows16["le_bin_stream"]["achieved"] == pytest.approx(14 * n / 0.06e-3 / 1e9)
    # the second tuning stage ran (the walk reached B = 2^16, past the gather trials), the
    # third (the largest trial, 2^18) did not
    assert rows["tune2_bin"]["bound"] == "alu"
    assert rows["tune2_bin"]["achieved"] == pytest.approx(3 * n / 0.03e-3 / 1e9)
    assert "tune3_bin" not in rows
    # a walk to 2^18: the third stage's pass (one trial, n pairs) counts too
    _, rows = bench.roofline({2000: ph}, {2000: [(16, 0), (1 << 18, 1900)]}, n)
    assert rows["tune3_bin"]["achieved"] == pytest.approx(n / 0.01e-3 / 1e9)


def test_roofline_model_skips_unused_second_stage():
    import bench

    n = 1 << 22
    ph = {nm: 0.01 for nm in ("tune1_bin", "tune1_fft", "tune1_tail", "tune2_bin", "tune2_fft",
                              "tune2_tail", "tune3_bin", "tune3_fft", "tune3_tail",
                              "le_bin_stream", "le_bin_gather", "le_fft", "loc_tail")}
    traces = {50: [(16, 0), (4096, 49)]}
    _, rows = bench.roofline({50: ph}, traces, n)
    assert "tune2_bin" not in rows and "tune2_fft" not in rows and "tune3_bin" not in rows


def test_all_cores_oracle_baseline_runs_in_spawned_processes():
    import bench

    r = bench.cpu_baseline_all_cores(max_procs=2)
    assert r["kind"] == "oracle" and r["cores"] == 2 and r["value"] > 0


def test_reference_arm_prints_one_contract_line(capsys):
    """--impl reference: the oracle in spawned single-threaded processes (two here, on
    n = 2^12 signals instead of the bench's 2^22), one JSON line with the reference
    arm's keys."""
    import argparse
    import json

    import bench

    args = argparse.Namespace(gpus=1, steps=6, warmup=2)
    bench.run_reference(args, n_log2=12, max_procs=2)
    out = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert out["impl"] == "reference" and out["metric"] == "transforms/s"
    assert out["steps"] == 6 and out["warmup"] == 2 and out["value"] > 0
    assert out["cpu_baseline"]["kind"] == "oracle" and out["cpu_baseline"]["cores"] == 2
    assert out["cpu_baseline"]["value"] == out["value"]
    assert out["e2e"] == {"value": out["value"], "unit": "transforms/s",
                          "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import argparse

    import bench

    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    assert bench.run_reference(argparse.Namespace(gpus=2, steps=1, warmup=0), n_log2=12) is None
    assert capsys.readouterr().out == ""


def test_reference_worker_setup_failure_is_raised_not_respawned(monkeypatch):
    """A failing worker setup surfaces as an error from the first task (an initializer
    that raised would make the pool respawn workers forever)."""
    import bench

    monkeypatch.setattr(bench, "KS", ())   # no signals to build: setup succeeds
    bench._ref_init(8)
    assert bench._REF_ERR is None and bench._REF_SIGS == []
    monkeypatch.setattr(bench, "_REF_ERR", "ImportError: no oracle")
    with pytest.raises(RuntimeError, match="setup failed"):
        bench._ref_ready(0)
    with pytest.raises(RuntimeError, match="setup failed"):
        bench._ref_step(0)
