"""The learned cost model end to end on a small scale: random seeded DAGs,
candidate plans timed on the GPU, the network trained by the library's own
kernels, and its held-out picks compared with the FLOP/byte heuristic, the
literal plan and the best candidate; picked plans are checked against the
oracle."""
import math

import numpy as np
import pytest

import oracle
from tests.gpu_util import need_gpu, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return need_gpu()


def test_learned_ranking_against_heuristic(torch, capsys):
    from paper_2502_03000_gb300 import costmodel as cm
    dags = cm.make_dags(20250203 + 5, 160, lo=16, hi=1024, cap_flops=2e10)
    recs = cm.collect(dags, reps=3)
    train, test = cm.split_train_test(recs, 0.75)
    net = cm.CostNet(seed=0)
    losses = net.fit([r["features"] for r in train], [math.log(r["time"]) for r in train], steps=1500)
    assert losses[-1] < losses[0]
    res = cm.evaluate(test, net)
    with capsys.disabled():
        print("\nheld-out:", {k: round(v, 4) if isinstance(v, float) else v for k, v in res.items()})
    # the optimised candidates beat the literal plan, and the learned pick
    # stays close to the best candidate
    assert res["best_geomean_s"] <= res["literal_geomean_s"]
    assert res["mlp_regret"] <= 1.25
    assert res["mlp_regret"] <= res["heuristic_regret"] * 1.10


def test_picked_plans_match_oracle(torch):
    from paper_2502_03000_gb300 import costmodel as cm
    from synth.dags import input_shapes
    import synth
    dags = [d for d in cm.make_dags(20250203 + 6, 40, lo=16, hi=96, cap_flops=1e8) if d[2] == "f32"][:12]
    for i, (nodes, outs, dt) in enumerate(dags):
        host = [synth.matrix(77 + i, s + 1, r, c, dt) for s, (r, c) in enumerate(input_shapes(nodes))]
        ref = oracle.evaluate(nodes, outs, host)
        for name, p in cm.candidate_plans(nodes, outs):
            got = p(*[to_dev(h, dt) for h in host])
            torch.cuda.synchronize()
            err = oracle.rel_err(to_host(got[0]), ref[0])
            assert err <= 1e-4, (i, name, err)
