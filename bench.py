#!/usr/bin/env python
"""ATSFFT throughput on GB300: transforms/s and Gsamples/s at n = 2^22.

Workload (a "step"): one sparse FFT with sparsity detection of each of four synthetic
signals of n = 2^22 complex64 samples whose DFTs have k in {50, 200, 1000, 2000}
nonzeros (uniform distinct locations, unit magnitudes, uniform phases) plus complex
Gaussian noise at 40 dB SNR; k is unknown to the solver.  Signals are generated
from fixed seeds and resident in HBM when the timed region starts; L2 is flushed
(256 MiB write) between steps, outside the timed brackets.

value  = transforms / s over the whole job (all ranks), device time (CUDA events);
e2e    = the same through the C ABI with host buffers: each step copies the four
         signals from pinned host memory, runs the transforms and reads the outputs
         back, all inside the timed region (one graph, atsfft_batch_create_io);
roofline = the dominant kernel of the step, timed by the library's phase events on
         its launch stream during the timed steps;
cpu_baseline = the FP64 oracle on the host cores, on a bounded sample.
Multi-GPU: replicas only (each rank transforms its own copies; no collective on the
data path), "scaling": "weak".
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_LOG2 = 22
KS = (50, 200, 1000, 2000)
SNR_DB = 40.0
SEED = 7
CAPACITY = 1 << 14
FLUSH_BYTES = 256 << 20
WORKLOAD = ("1D ATSFFT, n=2^22 complex64, k in {50,200,1000,2000} unknown to the solver, "
            "unit magnitudes, 40 dB complex Gaussian noise; one step = 4 transforms")


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


# DRAM bytes of one launch of a phase's kernels, from one ncu capture of the current
# kernels (dram__bytes_read.sum + dram__bytes_write.sum); None once a kernel changes.
NCU_TRAFFIC = {}

# The kernels of each profiled phase (the location tail is three kernels chained with
# programmatic dependent launch; its phase time covers all three).
PHASE_KERNELS = {
    "tune1_bin": "k_bin_gather_tune", "tune1_fft": "k_fft_batch x2", "tune1_tail": "k_tune_tail",
    "tune2_bin": "k_bin_stream<3,0>", "tune2_fft": "k_fft_batch x2", "tune2_tail": "k_tune_tail",
    "tune3_bin": "k_bin_stream<1,0>", "tune3_fft": "k_fft_batch x2", "tune3_tail": "k_tune_tail",
    "le_bin_stream": "k_bin_cols (D = n / B* <= 256; else k_bin_stream<14,1>)",
    "le_bin_gather": "k_bin_gather_1d",
    "le_fft": "k_fft_pass x2", "loc_tail": "k_loc_select + k_loc_votes + k_loc_finish",
}


def _signals():
    from synth import sparse_signal_1d

    return [sparse_signal_1d(1 << N_LOG2, k, 1000 + k, snr_db=SNR_DB) for k in KS]


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                    rows.append(parts)
        except Exception:
            pass
        finally:
            try:
                os.unlink(self.path)
            except Exception:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][2]),
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())}


def aggregate(local_ms, world_size, device=None):
    """Max over ranks of a rank's device time (ms); identity for one rank."""
    if world_size <= 1:
        return float(local_ms)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def cufft_reference_ms(n, dev, reps=20):
    """Dense cuFFT C2C complex64 of length n (torch.fft), median of `reps` event timings
    with L2 flushed in between -- a comparison only, not part of the method."""
    import torch

    x = torch.randn(n, dtype=torch.complex64, device=dev)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    for _ in range(3):
        torch.fft.fft(x)
    ts = []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(reps):
        flush.zero_()
        e0.record()
        torch.fft.fft(x)
        e1.record()
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return float(statistics.median(ts))


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


_REF_SIGS = None
_REF_ERR = None


def _ref_init(n_log2):
    """Worker of the reference arm: builds the oracle and its own copy of the step's
    signals before any step is timed.  A failure is kept and raised by the worker's
    first task (an initializer that raises makes the pool respawn workers forever)."""
    global _REF_SIGS, _REF_ERR
    try:
        import oracle
        from synth import sparse_signal_1d

        oracle.build()
        _REF_SIGS = [sparse_signal_1d(1 << n_log2, k, 1000 + k, snr_db=SNR_DB).x for k in KS]
    except Exception as exc:
        _REF_ERR = f"{type(exc).__name__}: {exc}"


def _ref_ready(_):
    if _REF_ERR:
        raise RuntimeError(f"reference worker setup failed: {_REF_ERR}")
    time.sleep(0.05)
    return os.getpid()


def _ref_step(i):
    """One reference step: the oracle transform of the step's signal i."""
    import oracle

    if _REF_ERR:
        raise RuntimeError(f"reference worker setup failed: {_REF_ERR}")
    oracle.atsfft_1d(_REF_SIGS[i], seed=SEED, capacity=CAPACITY)
    return i


def run_reference(args, n_log2=N_LOG2, max_procs=16):
    """The oracle (plain FP64 C) on the host cores, same metric: a step is one transform
    of the step's signals (k cycling), and the steps run as single-threaded processes,
    one per core, so that K steps take about K / cores transforms' time."""
    ws, rank, _ = _dist()
    if rank != 0:
        return None
    import multiprocessing as mp

    procs = max(1, min(max_procs, os.cpu_count() or 1))
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs, initializer=_ref_init, initargs=(n_log2,)) as pool:
        seen = set()
        for _ in range(100):   # every worker has built the oracle and its signals
            seen.update(pool.map(_ref_ready, range(procs), chunksize=1))
            if len(seen) >= procs:
                break
        pool.map(_ref_step, [i % len(KS) for i in range(args.warmup)], chunksize=1)
        steps = max(1, args.steps)
        t0 = time.perf_counter()
        pool.map(_ref_step, [i % len(KS) for i in range(steps)], chunksize=1)
        total = time.perf_counter() - t0
    v = steps / total
    line = {"impl": "reference", "metric": "transforms/s", "value": v, "unit": "transforms/s",
            "n_gpus": args.gpus, "steps": steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": 1 << n_log2, "ks": list(KS),
                       "reference_step": "one transform, cycling through the four k"},
            "cpu_baseline": {"value": v, "unit": "transforms/s", "cores": procs, "kind": "oracle",
                             "sample": f"{steps} transforms (k cycling over {list(KS)}), "
                                       f"{procs} single-threaded FP64 processes at once"},
            "e2e": {"value": v, "unit": "transforms/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return line


def cpu_baseline(sigs, budget_s=20.0):
    import oracle

    oracle.build()
    done, t0 = 0, time.perf_counter()
    while True:
        s = sigs[done % len(sigs)]
        oracle.atsfft_1d(s.x, seed=SEED, capacity=CAPACITY)
        done += 1
        if time.perf_counter() - t0 > budget_s or done >= 2 * len(sigs):
            break
    dt = time.perf_counter() - t0
    return {"value": done / dt, "unit": "transforms/s", "cores": 1, "kind": "oracle",
            "sample": f"{done} transforms of the step's signals (k cycling), single-threaded FP64"}


def _oracle_worker(k):
    """One oracle transform of the step's signal for k (a separate process)."""
    import oracle
    from synth import sparse_signal_1d

    oracle.build()
    x = sparse_signal_1d(1 << N_LOG2, k, 1000 + k, snr_db=SNR_DB).x
    t0 = time.perf_counter()
    oracle.atsfft_1d(x, seed=SEED, capacity=CAPACITY)
    return time.perf_counter() - t0


def cpu_baseline_all_cores(max_procs=16):
    """The same oracle, one single-threaded process per host core, all at once
    (independent transforms, k cycling): transforms/s = processes / the longest
    transform's time (each process times its own oracle call, after generating its
    signal)."""
    import multiprocessing as mp

    procs = max(1, min(max_procs, os.cpu_count() or 1))
    ks = [KS[i % len(KS)] for i in range(procs)]
    ctx = mp.get_context("spawn")   # spawned, not forked: the parent holds a CUDA context
    with ctx.Pool(procs) as pool:
        times = pool.map(_oracle_worker, ks, chunksize=1)
    return {"value": procs / max(times), "unit": "transforms/s", "cores": procs,
            "kind": "oracle",
            "sample": f"{procs} transforms of the step's signals (k cycling) at once, one "
                      f"single-threaded FP64 process per core"}


# ---- roofline model ---------------------------------------------------------------------
# Algorithmic bytes (or sample-hash pairs) per launch of each single-kernel phase, from
# the plan's defaults (alpha 0.5, tol 1e-6, 7 + 7 hashes, B range [2^4, n/16]): each value
# read and written once per launch (roofline() below lists the terms).
L_LOC, L_EST, NH = 7, 7, 14
# MUFU (XU pipe) results per clock per SM: ncu rates the XU pipe at one warp instruction
# per 4 cycles per SM sub-partition (4 x 32 / 4 = 32 lanes per clock per SM)
SFU_PER_SM_CLK, SMS, SM_MAX_MHZ = 32, 152, 2070.0


def _window_h(n, B, alpha=0.5, tol=1e-6):
    import math

    q = math.sqrt(2 * math.log(1 / tol))
    s = B * q / (math.pi * alpha)
    h = math.ceil(s * q)
    return min(h, n // 2 - 1)


def _chunks(n, B):
    return max(1, min((1 << 16) // B, n // B))


def _stream(n, B):
    return 5 * (2 * _window_h(n, B) + 1) >= n and n // B <= 4096


def _column_form(n, B):
    """The location pass at B takes the column form (only its in-window taps)."""
    return n >= 1024 and n // B <= 256


def mufu_pair_peak(stream=None):
    """Sample-hash pairs per second the MUFU pipe allows, measured: atsfft_mufu_probe
    times independent ex2.approx + rcp.approx chains on every SM (two operations per
    pair).  Returns (pairs/s, source string); the derived figure if the probe fails."""
    import paper_1908_02461_gb300 as A

    st, ops = A.atsfft_mufu_probe(4096, stream)
    if st == A.OK and ops > 0:
        return ops / 2.0, ("measured: atsfft_mufu_probe (ex2.approx + rcp.approx chains on "
                           f"every SM) {ops / 1e12:.2f} Tops/s / 2 ops per sample-hash pair")
    return SFU_PER_SM_CLK * SMS * SM_MAX_MHZ * 1e6 / 2.0, (
        "derived: 32 SFU ops/clk/SM x 152 SMs x 2070 MHz / 2 SFU ops per sample-hash pair")


def roofline(per_signal, traces, n, stages=3, pair_peak=None, pair_src=None, kept=None):
    """Algorithmic work of each profiled phase per launch, achieved rate, fraction of peak.

    Bytes (HBM-bound phases) count each input and output value once; pairs (the
    stream-form binning, bound by its two MUFU operations per (sample, hash) pair) count
    the in-window taps x hashes in the column form of the location pass, samples x hashes
    in the residue stream.  The tuning stages split the trials at the last one binned in
    the gather form and (three stages) before the largest; a later stage only counts for
    transforms whose controller walked past the previous stage's last trial (its kernels
    exit at once otherwise)."""
    peaks, src = _peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    if pair_peak is None:
        pair_peak = SFU_PER_SM_CLK * SMS * SM_MAX_MHZ * 1e6 / 2.0   # 2 SFU ops per pair
        pair_src = "derived: 32 SFU ops/clk/SM x 152 SMs x 2070 MHz / 2 SFU ops per sample-hash pair"
    logn = n.bit_length() - 1
    Bs = [1 << b for b in range(4, logn - 4 + 1)]
    gB = [B for B in Bs if not _stream(n, B)]
    sB = [B for B in Bs if _stream(n, B)]
    split = max(gB) if gB else 0
    s2B = sB[:-1] if stages == 3 and len(sB) >= 2 else sB
    s3B = sB[-1:] if stages == 3 and len(sB) >= 2 else []
    split2 = max(s2B) if s2B else split

    def fft_bytes(B, chunks):
        return 8 * B * chunks + 8 * B + 4 * B + (16 * B if B > 1024 else 0)

    rows = {}
    for k, ph in per_signal.items():
        # the trace's last trial is B*; an empty trace (fixed-k mode) carries B* alone
        Bstar = traces[k][-1][0]
        walked = max(b for b, _ in traces[k]) if len(traces[k]) > 1 else 0
        stage2 = walked > split
        stage3 = walked > split2
        tuned = len(traces[k]) > 1 or traces[k][0][1] is not None
        model = {}
        if tuned:
            model["tune1_bin"] = ("hbm", sum(8 * (2 * _window_h(n, B) + 1) + 8 * B for B in gB))
            model["tune1_fft"] = ("hbm", sum(fft_bytes(B, 1) for B in gB))
            model["tune1_tail"] = ("hbm", sum(4 * B + 4 * B for B in gB))
        for nm, tB, on in (("tune2", s2B, stage2), ("tune3", s3B, stage3)):
            if tB and on:
                R = max(tB)
                model[nm + "_bin"] = ("alu", len(tB) * n)
                model[nm + "_fft"] = ("hbm", sum(fft_bytes(B, _chunks(n, R) * R // B) for B in tB))
                model[nm + "_tail"] = ("hbm", sum(4 * B + 4 * B for B in tB))
        if _stream(n, Bstar):
            taps = min(2 * _window_h(n, Bstar) + 1, n) if _column_form(n, Bstar) else n
            model["le_bin_stream"] = ("alu", NH * taps)
        else:
            model["le_bin_gather"] = ("hbm", NH * 8 * (2 * _window_h(n, Bstar) + 1) + 8 * NH * Bstar)
        ch = _chunks(n, Bstar) if _stream(n, Bstar) else 1
        model["le_fft"] = ("hbm", sum(fft_bytes(Bstar, ch) for _ in range(NH)))
        # local maxima and cutoff: energies and lists, 8 B* per location hash; votes: at
        # most 4 k* D bytes per location hash (k* selected buckets of D = n / B*
        # preimages); estimates: 8 bytes per kept coordinate and estimation hash
        k_star = traces[k][-1][1] or 0
        model["loc_tail"] = ("hbm", L_LOC * Bstar * (4 + 4) + L_LOC * 4 * k_star * (n // Bstar)
                             + 8 * L_EST * ((kept or {}).get(k) or 0))
        for nm, (bound, units) in model.items():
            t = ph[nm] / 1e3
            if t <= 0:
                continue
            ach = units / t / 1e9
            frac = ach / (pair_peak / 1e9) if bound == "alu" else ach / hbm
            rows.setdefault(nm, []).append((t, ach, frac, units, bound))
    out = {"_alu_peak": {"pairs_per_s": pair_peak, "source": pair_src}}
    for nm, lst in rows.items():
        t = float(np.mean([r[0] for r in lst]))
        ach = float(np.mean([r[1] for r in lst]))
        out[nm] = {"bound": lst[0][4], "ms_per_launch": 1e3 * t, "achieved": ach,
                   "unit": "Gpair/s" if lst[0][4] == "alu" else "GB/s",
                   "frac": float(np.mean([r[2] for r in lst])), "launches_per_step": len(lst)}
    # dominant single-kernel phase: largest total time per step
    dom = max((nm for nm in out if not nm.startswith("_")),
              key=lambda nm: out[nm]["ms_per_launch"] * out[nm]["launches_per_step"])
    d = out[dom]
    peak = pair_peak / 1e9 if d["bound"] == "alu" else hbm
    roof = {"kernel": dom, "kernels": PHASE_KERNELS.get(dom, dom), "bound": d["bound"],
            "achieved": d["achieved"], "peak": peak,
            "unit": d["unit"], "frac": d["achieved"] / peak,
            "traffic": NCU_TRAFFIC[dom][0] if dom in NCU_TRAFFIC else None,
            "traffic_launch": NCU_TRAFFIC[dom][1] if dom in NCU_TRAFFIC else None,
            "peak_source": pair_src if d["bound"] == "alu" else f"{src} hbm_gbs",
            "ms_per_launch": d["ms_per_launch"]}
    return roof, out


def accuracy(sig, loc, val, k_star):
    """Eq. (15) against the generator's noise-free spectrum, k*/k, and how many kept
    coordinates lie outside the true support (the vote rule's noise floor)."""
    from synth import l1_error_per_coefficient

    on = np.isin(loc, sig.support)
    return {"l1_err_per_coef": float(l1_error_per_coefficient(sig, loc, val.astype(complex))),
            "k_star_over_k": k_star / len(sig.support), "kept": int(len(loc)),
            "kept_outside_support": int((~on).sum()),
            "support_found": float(on.sum() / len(sig.support))}


IMG_N, IMG_K, IMG_SNR, IMG_SEED = 4096, 1000, 30.0, 5
IMG_WORKLOAD = ("2D-SFFT, 4096x4096 complex64, k=1000 unknown to the solver, magnitudes "
                "log-uniform in [0.1,1], 30 dB complex Gaussian noise; one step = 1 transform")


def cufft2_reference_ms(N, dev, reps=20):
    """Dense 2D cuFFT C2C complex64 of N x N (torch.fft.fft2), median of event timings with
    L2 flushed in between -- a comparison only."""
    import torch

    x = torch.randn(N, N, dtype=torch.complex64, device=dev)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    for _ in range(3):
        torch.fft.fft2(x)
    ts = []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(reps):
        flush.zero_()
        e0.record()
        torch.fft.fft2(x)
        e1.record()
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return float(statistics.median(ts))


def image_summary(dev, steps, warmup):
    """The 2D workload (4096 x 4096, k = 1000, 30 dB) on the plain per-image path: device
    time per transform (CUDA events, L2 flushed between transforms; the 128 MiB input is
    larger than L2 anyway), the dense 2D cuFFT of the same size, and the accuracy."""
    import torch

    import paper_1908_02461_gb300 as A
    from synth import sparse_signal_2d

    sig = sparse_signal_2d(IMG_N, IMG_K, IMG_SEED, snr_db=IMG_SNR, mag=("loguniform", 0.1, 1.0))
    x = torch.from_numpy(sig.x).to(dev)
    plan = A.Plan((IMG_N, IMG_N), seed=SEED)
    o = dict(loc=torch.empty(CAPACITY, dtype=torch.int64, device=dev),
             val=torch.empty(CAPACITY, dtype=torch.complex64, device=dev),
             count=torch.zeros(1, dtype=torch.int64, device=dev),
             k=torch.zeros(1, dtype=torch.int64, device=dev),
             status=torch.zeros(1, dtype=torch.int32, device=dev))
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(max(3, warmup)):
        plan.exec_async(x, o["loc"], o["val"], o["count"], o["k"], o["status"], stream.cuda_stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms = []
    for _ in range(steps):
        flush.zero_()
        e0.record(stream)
        plan.exec_async(x, o["loc"], o["val"], o["count"], o["k"], o["status"], stream.cuda_stream)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    count, kstar, status = int(o["count"].item()), int(o["k"].item()), int(o["status"].item())
    m = min(count, CAPACITY)
    loc = o["loc"][:m].cpu().numpy()
    val = o["val"][:m].cpu().numpy()
    B, _ = plan.last_trace()[-1]
    plan.close()
    cu = cufft2_reference_ms(IMG_N, dev)
    t = float(np.mean(ms))
    return {"workload": IMG_WORKLOAD, "transforms_per_s": 1e3 / t, "ms_per_transform": t,
            "gsamples_per_s": IMG_N * IMG_N / (t * 1e-3) / 1e9,
            "cufft2d_c2c_ms": cu, "cufft2d_transforms_per_s": 1e3 / cu, "vs_cufft2d": cu / t,
            "status": status, "k_star": kstar, "B_star_per_axis": B,
            "accuracy": accuracy(sig, loc, val, kstar), "steps": steps}


def image_workload(args):
    """--workload image4096: the 2D line on its own (one JSON line)."""
    import torch

    import paper_1908_02461_gb300 as A

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    A.build()
    dev = torch.device("cuda", local)
    steps = max(5, min(args.steps, 200))
    with ClockSampler(local) as clk:
        r = image_summary(dev, steps, args.warmup)
    if rank != 0:
        return
    print(json.dumps({
        "metric": "transforms/s", "value": r["transforms_per_s"], "unit": "transforms/s",
        "n_gpus": 1, "steps": steps, "warmup": args.warmup, "ms_per_step": r["ms_per_transform"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic", "config": dict(r, l2="flushed between steps (256 MiB write)"),
        "clocks": clk.summary()}))


def ncu_case(k):
    """Small fixed case for ncu captures: no timing, no other kernels than the exec's."""
    import torch

    import paper_1908_02461_gb300 as A
    from synth import sparse_signal_1d

    A.build()
    sig = sparse_signal_1d(1 << N_LOG2, k, 1000 + k, snr_db=SNR_DB)
    x = torch.from_numpy(sig.x).cuda()
    plan = A.Plan((1 << N_LOG2,), seed=SEED)
    for _ in range(3):
        loc, val, kk, st, cnt = plan(x, capacity=CAPACITY)
    torch.cuda.synchronize()
    print(json.dumps({"ncu_case": k, "k_star": kk, "status": st, "count": cnt}))
    plan.close()


def ncu_image():
    """Small fixed 2D case for ncu captures: one plan, the 4096^2 headline image, three
    transforms, no timing."""
    import torch

    import paper_1908_02461_gb300 as A
    from synth import sparse_signal_2d

    A.build()
    sig = sparse_signal_2d(IMG_N, IMG_K, IMG_SEED, snr_db=IMG_SNR, mag=("loguniform", 0.1, 1.0))
    x = torch.from_numpy(sig.x).cuda()
    plan = A.Plan((IMG_N, IMG_N), seed=SEED)
    for _ in range(3):
        loc, val, kk, st, cnt = plan(x, capacity=CAPACITY)
    torch.cuda.synchronize()
    print(json.dumps({"ncu_image": IMG_N, "k_star": kk, "status": st, "count": cnt}))
    plan.close()


MIXED_SIGNALS = 512
MIXED_LOGN = (16, 18, 20, 22)
MIXED_BRANCHES = 64      # graph branches per batch


def mixed_workload(args):
    """512 independent signals, n uniform over {2^16, 2^18, 2^20, 2^22}, k log-uniform in
    [10, 1000], 40 dB noise: one plan per signal (clones of one template per size), the
    transforms recorded into CUDA graphs of MIXED_BRANCHES branches; a step transforms all
    512 signals.  Prints one JSON line (transforms/s and Gsamples/s)."""
    import torch

    import paper_1908_02461_gb300 as A

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    A.build()
    dev = torch.device("cuda", local)
    rng = np.random.default_rng(4242 + rank)
    sizes = [1 << int(rng.choice(MIXED_LOGN)) for _ in range(MIXED_SIGNALS)]
    ks = [int(round(np.exp(rng.uniform(np.log(10), np.log(1000))))) for _ in range(MIXED_SIGNALS)]
    gen = torch.Generator(device=dev)
    gen.manual_seed(777 + rank)
    xs = []
    for n, k in zip(sizes, ks):
        # x = IDFT of a k-sparse spectrum (unit magnitudes, uniform phases) + complex
        # Gaussian noise at 40 dB of the signal power, synthesised on the device
        loc = rng.choice(n, size=k, replace=False)
        spec = torch.zeros(n, dtype=torch.complex128, device=dev)
        spec[torch.from_numpy(loc).to(dev)] = torch.from_numpy(
            np.exp(2j * np.pi * rng.uniform(size=k))).to(dev)
        x = torch.fft.ifft(spec)
        p_sig = float((x.abs() ** 2).mean())
        sd = np.sqrt(p_sig * 10 ** (-SNR_DB / 10) / 2)
        noise = torch.complex(torch.randn(n, generator=gen, device=dev, dtype=torch.float64),
                              torch.randn(n, generator=gen, device=dev, dtype=torch.float64)) * sd
        xs.append((x + noise).to(torch.complex64).contiguous())
    # per size: parameters from the autotuner (probe signals of the same family)
    from paper_1908_02461_gb300.autotune import autotune

    tuned, t_tune = {}, time.perf_counter()
    for n in sorted(set(sizes)):
        res = autotune(n, k_range=(10, 1000), snr_db=SNR_DB, probes=3, reps=2, seed=SEED)
        tuned[n] = res
    t_tune = time.perf_counter() - t_tune
    templates = {n: A.Plan((n,), params=A.params(**tuned[n].params), seed=SEED)
                 for n in sorted(set(sizes))}
    t0 = time.perf_counter()
    plans = [templates[n].clone() for n in sizes]
    t_clone = time.perf_counter() - t0
    outs = [dict(loc=torch.empty(CAPACITY, dtype=torch.int64, device=dev),
                 val=torch.empty(CAPACITY, dtype=torch.complex64, device=dev),
                 count=torch.zeros(1, dtype=torch.int64, device=dev),
                 k=torch.zeros(1, dtype=torch.int64, device=dev),
                 status=torch.zeros(1, dtype=torch.int32, device=dev)) for _ in sizes]
    batches = []
    for b0 in range(0, MIXED_SIGNALS, MIXED_BRANCHES):
        items = [(plans[i], xs[i], outs[i]["loc"], outs[i]["val"], outs[i]["count"],
                  outs[i]["k"], outs[i]["status"]) for i in range(b0, min(b0 + MIXED_BRANCHES, MIXED_SIGNALS))]
        batches.append(A.Batch(items))
    stream = torch.cuda.current_stream()
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def step():
        for bt in batches:
            bt.launch(stream.cuda_stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    steps = max(1, args.steps // 100)
    ms = []
    if ws > 1:
        torch.distributed.barrier()
    with ClockSampler(local) as clk:
        for _ in range(steps):
            flush.zero_()
            ev0.record(stream)
            step()
            ev1.record(stream)
            ev1.synchronize()
            ms.append(ev0.elapsed_time(ev1))
    total_ms = aggregate(sum(ms), ws, dev)
    ntrans = MIXED_SIGNALS * steps * ws
    status = [int(o["status"].item()) for o in outs]
    kstar = [int(o["k"].item()) for o in outs]
    samples = sum(sizes) * steps * ws
    launches = sum(bt.kernels() for bt in batches) * steps
    for bt in batches:
        bt.close()
    for p in plans + list(templates.values()):
        p.close()
    if rank != 0:
        return
    print(json.dumps({
        "metric": "transforms/s", "value": ntrans / (total_ms / 1e3), "unit": "transforms/s",
        "n_gpus": ws, "steps": steps, "warmup": args.warmup, "ms_per_step": total_ms / steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "512 signals, n uniform in {2^16,2^18,2^20,2^22}, k log-uniform "
                               "in [10,1000], 40 dB noise; one step = 512 transforms",
                   "gsamples_per_s": samples / (total_ms / 1e3) / 1e9,
                   "graphs": len(batches), "branches_per_graph": MIXED_BRANCHES,
                   "autotune_s": t_tune,
                   "autotuned": {str(n): dict(r.params, ms=r.ms_per_transform, err=r.error)
                                 for n, r in tuned.items()},
                   "clone_s": t_clone, "status_counts": {str(v): status.count(v) for v in sorted(set(status))},
                   "k_star_vs_k_median_ratio": float(np.median(np.array(kstar) / np.array(ks))),
                   "l2": "flushed between steps (256 MiB write)"},
        "gpu_launches": launches,
        "clocks": clk.summary(),
    }))


GRAD_SIGNALS, GRAD_LOGN, GRAD_K = 64, 20, 256


def grad_workload(args):
    """64 signals, n = 2^20, k = 256, 40 dB noise; loss = sum |xhat_S - target|^2 with
    Gaussian targets: a step is the forward transform of every signal (with the median
    selections) and the gradient of the loss with respect to every input
    (atsfft_estimate_adjoint).  Prints one JSON line (transforms/s, forward + gradient)."""
    import torch

    import paper_1908_02461_gb300 as A
    from paper_1908_02461_gb300 import _lib as L

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    A.build()
    dev = torch.device("cuda", local)
    from synth import sparse_signal_1d

    n = 1 << GRAD_LOGN
    sigs = [sparse_signal_1d(n, GRAD_K, 9000 + i, snr_db=SNR_DB) for i in range(GRAD_SIGNALS)]
    xs = [torch.from_numpy(sg.x).to(dev) for sg in sigs]
    tmpl = A.Plan((n,), seed=SEED)
    plans = [tmpl.clone() for _ in sigs]
    cap = 1 << 12
    bufs = [dict(loc=torch.empty(cap, dtype=torch.int64, device=dev),
                 val=torch.empty(cap, dtype=torch.complex64, device=dev),
                 msel=torch.empty(cap, 2, dtype=torch.uint8, device=dev),
                 count=torch.zeros(1, dtype=torch.int64, device=dev),
                 k=torch.zeros(1, dtype=torch.int64, device=dev),
                 status=torch.zeros(1, dtype=torch.int32, device=dev),
                 gx=torch.empty(n, dtype=torch.complex64, device=dev)) for _ in sigs]
    gen = torch.Generator(device=dev)
    gen.manual_seed(5)
    targets = torch.randn(GRAD_SIGNALS, cap, dtype=torch.complex64, device=dev, generator=gen)
    stream = torch.cuda.current_stream()
    s = stream.cuda_stream

    def step():
        for p, x, b in zip(plans, xs, bufs):
            L.atsfft_exec_sel(p.handle, x, b["loc"], b["val"], b["msel"], cap, b["count"], b["k"],
                              b["status"], s)
        counts = [min(int(b["count"].item()), cap) for b in bufs]   # (synchronises)
        Bs = [L.atsfft_last_result(p.handle, s)[1] for p in plans]
        for p, b, c, B, t in zip(plans, bufs, counts, Bs, targets):
            g = 2.0 * (b["val"][:c] - t[:c])          # dL/dRe y + i dL/dIm y
            L.atsfft_estimate_adjoint(p.handle, B, b["loc"], b["msel"], c, g, b["gx"], s)
        return counts

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    steps = max(2, args.steps // 100)
    t_all = []
    if ws > 1:
        torch.distributed.barrier()
    with ClockSampler(local) as clk:
        for _ in range(steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            counts = step()
            torch.cuda.synchronize()
            t_all.append((time.perf_counter() - t0) * 1e3)
    total_ms = aggregate(sum(t_all), ws, dev)
    ntrans = GRAD_SIGNALS * steps * ws
    for p in plans:
        p.close()
    tmpl.close()
    if rank != 0:
        return
    print(json.dumps({
        "metric": "transforms/s", "value": ntrans / (total_ms / 1e3), "unit": "transforms/s",
        "n_gpus": ws, "steps": steps, "warmup": args.warmup, "ms_per_step": total_ms / steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "64 signals, n=2^20, k=256, 40 dB; forward transform + gradient "
                               "of sum |xhat_S - target|^2 (Gaussian targets) w.r.t. the input",
                   "timing": "host wall clock around each step (two device syncs per step: "
                             "the counts and B* of the forward pass set the adjoint's sizes)",
                   "mean_count": float(np.mean(counts))},
        "clocks": clk.summary(),
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--phases", action="store_true", help="print per-phase times to stderr")
    ap.add_argument("--streams", type=int, default=4,
                    help="without --no-graph: ignored; with it, run the step's transforms on "
                         "this many CUDA streams (1 = in order)")
    ap.add_argument("--tune-stages", type=int, default=3, choices=[1, 2, 3],
                    help="1D tuning in one batch (1), small-window trials first (2), and "
                         "the largest trial last (3)")
    ap.add_argument("--est-reuse-loc", action="store_true",
                    help="estimation loops reuse the location hashes (off: fresh hashes)")
    ap.add_argument("--fixed-k", action="store_true",
                    help="no tuning: B from the true k given as the hint (the SFFT setting)")
    ap.add_argument("--no-graph", action="store_true",
                    help="time per-signal execs on streams instead of one graph launch per step")
    ap.add_argument("--no-image", action="store_true",
                    help="skip the 2D (4096x4096) summary in the headline line")
    ap.add_argument("--workload", default="headline",
                    choices=["headline", "mixed512", "grad64", "image4096"],
                    help="mixed512: the 512-signal mixed-size batch; grad64: 64 transforms with "
                         "the gradient of a loss at their supports (instead of the headline)")
    ap.add_argument("--ncu-case", type=int, default=0, metavar="K",
                    help="profiling case for ncu: one plan, the k=K signal, three transforms")
    ap.add_argument("--ncu-image", action="store_true",
                    help="profiling case for ncu: one plan, the 4096^2 image, three transforms")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.ncu_image:
        ncu_image()
        return
    if args.ncu_case:
        ncu_case(args.ncu_case)
        return
    if args.workload == "mixed512":
        mixed_workload(args)
        return
    if args.workload == "grad64":
        grad_workload(args)
        return
    if args.workload == "image4096":
        image_workload(args)
        return

    import torch

    import paper_1908_02461_gb300 as A

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    A.build()
    dev = torch.device("cuda", local)
    sigs = _signals()
    n = 1 << N_LOG2
    host = [torch.from_numpy(s.x).pin_memory() for s in sigs]
    xs = [h.to(dev) for h in host]
    nstreams = max(1, min(args.streams, len(sigs)))
    use_graph = not args.no_graph
    common = dict(tune_stages=args.tune_stages, est_reuse_loc=int(args.est_reuse_loc),
                  fixed_k=int(args.fixed_k))
    pp = A.params(**common)
    plans = [A.Plan((n,), params=pp, seed=SEED, k_hint=k if args.fixed_k else 0) for k in KS]
    # the plain path (one transform at a time): its own plans, profiled per phase
    plain_plans = [A.Plan((n,), params=A.params(**common), seed=SEED,
                          k_hint=k if args.fixed_k else 0) for k in KS]
    outs = []
    for _ in sigs:
        outs.append(dict(loc=torch.empty(CAPACITY, dtype=torch.int64, device=dev),
                         val=torch.empty(CAPACITY, dtype=torch.complex64, device=dev),
                         count=torch.zeros(1, dtype=torch.int64, device=dev),
                         k=torch.zeros(1, dtype=torch.int64, device=dev),
                         status=torch.zeros(1, dtype=torch.int32, device=dev)))
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    side = [stream] + [torch.cuda.Stream(device=dev) for _ in range(nstreams - 1)]
    batch = None
    if use_graph:
        # the step's transforms as one CUDA graph with a branch per signal
        batch = A.Batch([(p, x, o["loc"], o["val"], o["count"], o["k"], o["status"])
                         for p, x, o in zip(plans, xs, outs)])

    def step():
        if batch is not None:
            batch.launch(stream.cuda_stream)
            return
        # transforms on `nstreams` streams, joined back into the timing stream
        if nstreams == 1:
            for p, x, o in zip(plans, xs, outs):
                p.exec_async(x, o["loc"], o["val"], o["count"], o["k"], o["status"], stream.cuda_stream)
            return
        start = torch.cuda.Event()
        start.record(stream)
        for i, (p, x, o) in enumerate(zip(plans, xs, outs)):
            st = side[i % nstreams]
            st.wait_event(start)
            p.exec_async(x, o["loc"], o["val"], o["count"], o["k"], o["status"], st.cuda_stream)
        for st in side[1:]:
            ev = torch.cuda.Event()
            ev.record(st)
            stream.wait_event(ev)

    def plain_step():
        for p, x, o in zip(plain_plans, xs, outs):
            p.exec_async(x, o["loc"], o["val"], o["count"], o["k"], o["status"], stream.cuda_stream)

    for _ in range(args.warmup):
        flush.zero_()
        step()
        flush.zero_()
        plain_step()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    # ---- plain per-signal path, in order, with per-kernel phase events -----------------
    for p in plain_plans:
        p.set_profiling(True)
    plain_ms, phase_acc, stamp_acc = [], [], []
    for _ in range(max(3, args.steps // 4)):
        flush.zero_()
        ev0.record(stream)
        plain_step()
        ev1.record(stream)
        ev1.synchronize()
        plain_ms.append(ev0.elapsed_time(ev1))
        for p in plain_plans:
            ph, _ = p.phase_times()
            phase_acc.append(ph)
            if args.phases:
                st_ = p.tail_stamps()
                stamp_acc.append([(b - st_[0]) / 1e3 for b in st_])
    for p in plain_plans:
        p.set_profiling(False)
    plain_value = len(sigs) * len(plain_ms) / (sum(plain_ms) / 1e3)

    # ---- timed region: the step on `nstreams` streams ----------------------------------
    step_ms, launches = [], 0
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.zero_()
            ev0.record(stream)
            step()
            ev1.record(stream)
            ev1.synchronize()
            step_ms.append(ev0.elapsed_time(ev1))
            launches += batch.kernels() if batch is not None else sum(p.phase_times()[1] for p in plans)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if ws > 1:
        torch.distributed.barrier()
    total_ms = aggregate(sum(step_ms), ws, dev)
    ntrans = len(sigs) * args.steps * ws
    value = ntrans / (total_ms / 1e3)

    status = [int(o["status"].item()) for o in outs]
    kstar = [int(o["k"].item()) for o in outs]
    counts = [int(o["count"].item()) for o in outs]

    # ---- dominant kernel of the plain step and its roofline -------------------------
    names = list(phase_acc[0].keys())
    mean_phase = {nm: float(np.mean([ph[nm] for ph in phase_acc])) for nm in names}
    per_signal = {}
    for i, k in enumerate(KS):
        rows = phase_acc[i::len(KS)]
        per_signal[k] = {nm: float(np.mean([r[nm] for r in rows])) for nm in names}
    bin_ms = {k: per_signal[k]["le_bin_stream"] + per_signal[k]["le_bin_gather"] for k in KS}
    tune_stage2 = {k: sum(per_signal[k][f"tune{st}_{ph}"] for st in (2, 3) for ph in ("bin", "fft", "tail"))
                   for k in KS}
    traces = {}
    for k, p in zip(KS, plans):
        tr = p.last_trace()
        if not tr:   # fixed-k mode: no trials, B* from the plan's last result
            tr = [(A._lib.atsfft_last_result(p.handle)[1], None)]
        traces[k] = tr
    pair_peak, pair_src = mufu_pair_peak(stream.cuda_stream)
    kept = {k: min(int(o["count"].item()), CAPACITY) for k, o in zip(KS, outs)}
    roof, phase_rooflines = roofline(per_signal, traces, n, stages=args.tune_stages,
                                     pair_peak=pair_peak, pair_src=pair_src, kept=kept)
    acc = {}
    for k, sg, o in zip(KS, sigs, outs):
        m = min(int(o["count"].item()), CAPACITY)
        acc[str(k)] = accuracy(sg, o["loc"][:m].cpu().numpy(), o["val"][:m].cpu().numpy(),
                               int(o["k"].item()))

    # ---- end to end through the C ABI with host buffers -----------------------------
    host_out = [dict(loc=torch.empty(CAPACITY, dtype=torch.int64).pin_memory(),
                     val=torch.empty(CAPACITY, dtype=torch.complex64).pin_memory()) for _ in sigs]

    # largest k first: its transform is the longest, and the last input to land should be
    # followed by the shortest one.  One graph (atsfft_batch_create_io): the inputs are
    # copied one after another from pinned host memory, each transform starts as soon as
    # its input has landed, its outputs come back after it.
    order = sorted(range(len(sigs)), key=lambda i: -KS[i])
    host_scal = [dict(count=torch.zeros(1, dtype=torch.int64).pin_memory(),
                      k=torch.zeros(1, dtype=torch.int64).pin_memory(),
                      status=torch.zeros(1, dtype=torch.int32).pin_memory()) for _ in sigs]
    io_batch = A.Batch([(plans[i], xs[i], outs[i]["loc"], outs[i]["val"], outs[i]["count"],
                         outs[i]["k"], outs[i]["status"]) for i in order],
                       host=[dict(x=host[i], loc=host_out[i]["loc"], val=host_out[i]["val"],
                                  **host_scal[i]) for i in order])

    def e2e_step():
        io_batch.launch(stream.cuda_stream)

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    e2e_ms = []
    for _ in range(args.steps):
        flush.zero_()
        ev0.record(stream)
        e2e_step()
        ev1.record(stream)
        ev1.synchronize()
        e2e_ms.append(ev0.elapsed_time(ev1))
    e2e_total = aggregate(sum(e2e_ms), ws, dev)
    cufft_ms = cufft_reference_ms(n, dev) if rank == 0 else None
    h2d = sum(h.numel() * 8 for h in host)
    d2h = len(sigs) * (CAPACITY * 8 + CAPACITY * 8 + 8 + 8 + 4)

    image = None
    if rank == 0 and not args.no_image:
        try:
            image = image_summary(dev, 20, 3)
        except Exception as exc:   # the 1D line stands on its own
            image = {"unavailable": f"{type(exc).__name__}: {exc}"}

    cpu = cpu_all = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(sigs)
        try:
            cpu_all = cpu_baseline_all_cores()
        except Exception as exc:   # the single-threaded figure stands on its own
            cpu_all = {"unavailable": f"{type(exc).__name__}: {exc}"}

    clocks = clk.summary()
    if args.phases and rank == 0:
        print(json.dumps({"per_signal_phase_ms": per_signal, "mean_phase_ms": mean_phase},
                         indent=1), file=sys.stderr)
        for i, k in enumerate(KS):
            if stamp_acc:
                print("tail stamps us k=%d:" % k, [round(v, 1) for v in stamp_acc[-len(KS) + i]],
                      file=sys.stderr)
    io_batch.close()
    if batch is not None:
        batch.close()
    for p in plans + plain_plans:
        p.close()
    if ws > 1:
        torch.distributed.destroy_process_group()
    if rank != 0:
        return
    line = {
        "metric": "transforms/s", "value": value, "unit": "transforms/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": n, "ks": list(KS), "snr_db": SNR_DB,
                   "parallelism": f"replicas x{ws}", "l2": "flushed between steps (256 MiB write)",
                   "gsamples_per_s": value * n / 1e9,
                   "plain_path_transforms_per_s": plain_value,
                   "plain_path_ms_per_step": float(np.mean(plain_ms)),
                   "k_star": kstar, "counts": counts, "status": status,
                   "tune_stages": args.tune_stages, "est_reuse_loc": bool(args.est_reuse_loc),
                   "fixed_k": bool(args.fixed_k),
                   "path": ("one CUDA graph per step (atsfft_batch_launch), a branch per signal"
                            if use_graph else
                            "plain per-signal path (one exec per transform)" if nstreams == 1 else
                            f"per-signal execs on {nstreams} concurrent streams"),
                   "cufft_c2c_ms": cufft_ms,
                   "cufft_c2c_transforms_per_s": (1e3 / cufft_ms) if cufft_ms else None,
                   "vs_cufft": (value * cufft_ms / 1e3) if cufft_ms else None,
                   "plain_vs_cufft": (plain_value * cufft_ms / 1e3) if cufft_ms else None,
                   "accuracy": acc,
                   "bin_pass_ms": bin_ms, "tune_stage2_ms": tune_stage2, "wall_s": wall},
        "e2e": {"value": ntrans / (e2e_total / 1e3), "unit": "transforms/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "roofline": roof,
        "phase_rooflines": phase_rooflines,
        "cpu_baseline": cpu,
        "cpu_baseline_all_cores": cpu_all,
        "image4096": image,
        "clocks": clocks,
    }
    print(json.dumps(line))


if __name__ == "__main__":
    main()
