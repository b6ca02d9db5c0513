"""Train the library's cost network on GB300 timings and save it.

    python -m paper_2502_03000_gb300.train_costnet --out costnet.json \\
        [--records records.json[.gz]] [--dags 5000] [--budget-s 900]

Without --records, the candidates of --dags random expression DAGs (the
planner benchmark's generator: depth <= 5, dims log-uniform 16..8192,
FP32/BF16, literal work <= 2e11 FLOP) are timed on the GPU first (and saved
next to --out).  The network is trained by the library's own GPU kernels on
the first 80% of the DAGs, with targets centred per DAG; the held-out 20% give
the regrets of its picks and of the FLOP/byte estimate's.  The saved JSON
(weights, feature scaling) loads with ``costmodel.CostNet.load`` or
``costmodel.load_default``.
"""
from __future__ import annotations

import argparse
import gzip
import json
import math
import os
import sys
import time


def main(argv=None):
    from . import costmodel as cm
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", required=True)
    ap.add_argument("--records", default="")
    ap.add_argument("--dags", type=int, default=5000)
    ap.add_argument("--budget-s", type=float, default=900.0)
    ap.add_argument("--seed", type=int, default=20250203 + 5)
    ap.add_argument("--steps", type=int, default=1500)
    a = ap.parse_args(argv)
    if a.records:
        opener = gzip.open if a.records.endswith(".gz") else open
        with opener(a.records, "rt") as f:
            recs = json.load(f)
    else:
        dags = cm.make_dags(a.seed, a.dags, lo=16, hi=8192, cap_flops=2e11)
        recs, t0 = [], time.perf_counter()
        for i in range(0, len(dags), 100):
            part = cm.collect(dags[i:i + 100], target_s=5e-4)
            for r in part:
                r["dag"] += i
            recs += part
            if time.perf_counter() - t0 > a.budget_s:
                break
        cm.save_records(recs, os.path.splitext(a.out)[0] + "_records.json")
    train, test = cm.split_train_test(recs, 0.8)
    net = cm.CostNet(seed=0)
    losses = net.fit([r["features"] for r in train], [math.log(r["time"]) for r in train], steps=a.steps,
                     groups=[r["dag"] for r in train])
    net.save(a.out)
    res = cm.evaluate(test, net, guard=4.0)
    print(json.dumps({"records": len(recs), "train_dags": len({r["dag"] for r in train}),
                      "loss_first_last": [losses[0], losses[-1]], "held_out": res}), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
