"""The batched workload against the oracle: a mixed-size batch of independent noisy
signals in one CUDA graph, with parameters from the autotuner, each branch compared with
the FP64 oracle run on the same parameters under the parity rule of tests/_parity.py
(exact, or every difference traced to a decision the oracle logged within 2e-4 of its
boundary).  Needs a GPU.

The batch is a reduced form of the 512-signal workload: n over {2^16, 2^18, 2^20} five
times each and one 2^22, k log-uniform in [10, 1000], 40 dB noise, one plan clone per
signal, all 16 transforms as branches of one graph (the coop_* launch parameters are
still passed; they no longer change anything).  Half the branches take the autotuner's
choice for their n, the other half a fixed non-default set (5 + 5 loops, window tolerance 1e-5, alpha 1, tuning from
B = 32), so that parameters other than the defaults are compared whatever the autotuner
picks.
"""

import numpy as np
import pytest

from _parity import BAND, check

pytestmark = pytest.mark.gpu

LOGNS = [16] * 5 + [18] * 5 + [20] * 5 + [22]
SEED = 11
CAPACITY = 1 << 13
NONDEFAULT = dict(loops_loc=5, loops_est=5, filter_tol=1e-5, filter_alpha=1.0, b_min_log2=5)


@pytest.fixture(scope="module")
def A():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1908_02461_gb300 as A

    A.build()
    return A


def test_mixed_batch_with_autotuned_parameters_matches_oracle(A):
    import torch

    import oracle as O
    from paper_1908_02461_gb300.autotune import autotune
    from synth import sparse_signal_1d

    O.build()
    rng = np.random.default_rng(SEED)
    ks = [int(round(np.exp(rng.uniform(np.log(10), np.log(1000))))) for _ in LOGNS]
    sigs = [sparse_signal_1d(1 << b, k, 500 + i, snr_db=40.0)
            for i, (b, k) in enumerate(zip(LOGNS, ks))]
    tuned = {b: autotune(1 << b, k_range=(10, 1000), snr_db=40.0, probes=2, reps=1,
                         seed=SEED).params for b in sorted(set(LOGNS))}
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    launch = dict(coop_blocks_per_sm=1, coop_sms=nsm // 4)
    templates, plans, overs = {}, [], []
    for i, b in enumerate(LOGNS):
        over = dict(tuned[b]) if i % 2 == 0 else dict(NONDEFAULT)
        key = (b, tuple(sorted(over.items())))
        if key not in templates:
            templates[key] = A.Plan((1 << b,), params=A.params(**launch, **over), seed=SEED)
        plans.append(templates[key].clone())
        overs.append(over)
    xs = [torch.from_numpy(s.x).cuda() for s in sigs]
    outs = [dict(loc=torch.empty(CAPACITY, dtype=torch.int64, device="cuda"),
                 val=torch.empty(CAPACITY, dtype=torch.complex64, device="cuda"),
                 count=torch.zeros(1, dtype=torch.int64, device="cuda"),
                 k=torch.zeros(1, dtype=torch.int64, device="cuda"),
                 status=torch.zeros(1, dtype=torch.int32, device="cuda")) for _ in sigs]
    batch = A.Batch([(p, x, o["loc"], o["val"], o["count"], o["k"], o["status"])
                     for p, x, o in zip(plans, xs, outs)])
    assert batch.kernels() > 0
    for _ in range(2):   # a relaunch gives the same outputs
        batch.launch()
    torch.cuda.synchronize()
    non_default = 0
    for i, (b, k, s, p, o, over) in enumerate(zip(LOGNS, ks, sigs, plans, outs, overs)):
        count, kk, st = int(o["count"].item()), int(o["k"].item()), int(o["status"].item())
        m = min(count, CAPACITY)
        gpu = dict(trace=p.last_trace(), k=kk, status=st, count=count,
                   loc=o["loc"][:m].cpu().numpy(), val=o["val"][:m].cpu().numpy())
        ocfg = {key: v for key, v in over.items() if key != "tune_stages"}
        ref, dec = O.atsfft_log(s.x, params=O.default_params(**ocfg), seed=SEED,
                                capacity=CAPACITY, band=BAND)
        info = check(gpu, ref, dec, (1 << b,), SEED, loops_loc=over.get("loops_loc", 7),
                     capacity=CAPACITY)
        non_default += any(over.get(key, dv) != dv for key, dv in
                           (("loops_loc", 7), ("filter_tol", 1e-6), ("filter_alpha", 0.5),
                            ("b_min_log2", 0), ("b_max_log2", 0)))
        print(f"[config4] n=2^{b} k={k} {ocfg} {info}")
    assert non_default >= len(LOGNS) // 2
    batch.close()
    for p in plans + list(templates.values()):
        p.close()
