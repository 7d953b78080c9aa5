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
    ph = {"tune_gather": 0.02, "tune_stream": 0.03, "tune_fft": 0.06, "tune_tail": 0.05,
          "le_bin_stream": 0.06, "le_bin_gather": 0.006, "le_fft": 0.07, "loc_tail": 0.12}
    traces = {2000: [(16, 0), (65536, 1900)]}
    roof, rows = bench.roofline({2000: ph}, traces, n)
    assert roof["kernel"] == "loc_tail" and roof["bound"] == "hbm"
    assert rows["le_bin_stream"]["bound"] == "alu"
    # 14 hashes x n pairs in 0.06 ms
    assert rows["le_bin_stream"]["achieved"] == pytest.approx(14 * n / 0.06e-3 / 1e9)
