"""Writes oracle_1d_n2p28_k100.json: the oracle's result for the largest 1D size, an
exactly 100-sparse signal of n = 2^28 samples (unit magnitudes, uniform phases; Section
IV's recipe), which the oracle needs a few minutes for.  The GPU test of that size
compares its result with this file.

Inputs come from the seeded generator `synth.sparse_signal_1d`; every stored value is
the oracle's (Algorithm 2 for the trials, k* and B*; Section III-B location by voting;
Eq. (11) estimation is checked against the exact spectrum instead, so no value is
stored).  Run from the repository root:

    python tests/golden/make_oracle_large.py
"""

import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle as O  # noqa: E402
from synth import sparse_signal_1d  # noqa: E402

LOGN, K, SIGNAL_SEED, PLAN_SEED, CAPACITY = 28, 100, 28, 3, 1 << 14
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_1d_n2p28_k100.json")


def main():
    O.build()
    sig = sparse_signal_1d(1 << LOGN, K, SIGNAL_SEED)
    t0 = time.time()
    ref = O.atsfft_1d(sig.x, seed=PLAN_SEED, capacity=CAPACITY)
    secs = time.time() - t0
    on = np.isin(ref.loc, sig.support)
    doc = {
        "source": "oracle/ (FP64 C) on synth.sparse_signal_1d(2^28, 100, seed 28), written by "
                  "tests/golden/make_oracle_large.py",
        "logn": LOGN, "k": K, "signal_seed": SIGNAL_SEED, "plan_seed": PLAN_SEED,
        "capacity": CAPACITY,
        "status": int(ref.status), "B_star": int(ref.B_star), "k_star": int(ref.k_star),
        "count": int(ref.count), "min_margin": float(ref.min_margin),
        "outside_support": int((~on).sum()),
        "max_abs_outside": float(np.abs(ref.val[~on]).max()) if (~on).any() else 0.0,
        "oracle_seconds": round(secs, 1),
    }
    # scalars one per line, then the trial trace and the locations (ascending) one line each
    lists = {"trials_B_k": [[int(b), int(k)] for b, k, _ in ref.trials],
             "loc": [int(v) for v in ref.loc]}
    text = json.dumps(doc, indent=1)[:-2]
    for key, v in lists.items():
        text += f',\n "{key}": ' + json.dumps(v, separators=(",", ":"))
    with open(OUT, "w") as f:
        f.write(text + "\n}\n")
    print(f"wrote {OUT}: status {ref.status} B* {ref.B_star} k* {ref.k_star} "
          f"count {ref.count} margin {ref.min_margin:.3g} ({secs:.0f} s)")


if __name__ == "__main__":
    main()
