"""The learned cost model end to end: random seeded DAGs, the library's
candidate plans timed on the GPU, the network trained by the library's own
kernels and loaded into the library, whose planner then picks among the
candidates itself (ARMA_PLAN_COST_MLP).  On fresh DAGs the shipped network's
picks must beat the FLOP/byte estimate's; the library's in-plan choice must
equal the rule computed here; every candidate must match the oracle."""
import math

import numpy as np
import pytest

import oracle
import paper_2502_03000_gb300 as ag
from tests.gpu_util import need_gpu, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return need_gpu()


@pytest.fixture(scope="module")
def trained(torch):
    from paper_2502_03000_gb300 import costmodel as cm
    dags = cm.make_dags(20250203 + 5, 320, lo=16, hi=1024, cap_flops=2e10)
    recs = cm.collect(dags)
    train, test = cm.split_train_test(recs, 0.75)
    net = cm.CostNet(seed=0)
    losses = net.fit([r["features"] for r in train], [math.log(r["time"]) for r in train], steps=3000)
    yield dags, recs, train, test, net, losses
    ag.clear_cost_model()


def test_learned_ranking_trains_and_ranks(trained, capsys):
    """A network trained here on 240 small DAGs (launch-bound, so the
    timings are noisy at the 1% level) learns: its loss drops and its picks
    on 80 held-out DAGs beat the literal plan by far.  Whether it also beats
    the FLOP/byte estimate is a 1% question that 80 DAGs cannot settle: that
    is asserted on the shipped network, trained on 4,000 DAGs, over 500
    fresh ones (below), and measured at 5,000 DAGs by the planner bench."""
    from paper_2502_03000_gb300 import costmodel as cm
    dags, recs, train, test, net, losses = trained
    assert losses[-1] < losses[0]
    res = cm.evaluate(test, net, guard=4.0)
    with capsys.disabled():
        print("\nheld-out:", {k: round(v, 4) if isinstance(v, float) else v for k, v in res.items()})
    assert res["best_geomean_s"] <= res["literal_geomean_s"]
    assert res["mlp_regret"] < res["literal_regret"] - 0.03, res


def test_library_choice_follows_the_network(trained):
    """The trained network, loaded into the library, makes arma_gpu_plan pick
    exactly the candidate the rule picks from the recorded features; with no
    model loaded the estimate decides."""
    from paper_2502_03000_gb300 import costmodel as cm
    dags, recs, train, test, net, _ = trained
    net.to_library(guard=4.0)
    _, mlp, _ = cm.picks(test, net, guard=4.0)
    heur, _, _ = cm.picks(test, None)
    checked = 0
    for d, r in sorted(mlp.items())[:40]:
        nodes, outs, _ = dags[d]
        picked, scorer = cm.library_pick(nodes, outs)
        assert scorer == "mlp"
        assert picked == r["cand"], (d, picked, r["cand"])
        checked += 1
    assert checked > 0
    ag.clear_cost_model()
    for d, r in sorted(heur.items())[:20]:
        nodes, outs, _ = dags[d]
        picked, scorer = cm.library_pick(nodes, outs)
        assert scorer == "heuristic" and picked == r["cand"], (d, picked, r["cand"])


def test_weights_persist(trained, tmp_path):
    from paper_2502_03000_gb300 import costmodel as cm
    _, recs, _, test, net, _ = trained
    path = str(tmp_path / "costnet.json")
    net.save(path)
    back = cm.CostNet.load(path)
    X = [r["features"] for r in test[:50]]
    assert np.array_equal(net.correction(X), back.correction(X))
    rp = str(tmp_path / "records.json")
    cm.save_records(recs[:20], rp)
    assert cm.load_records(rp) == recs[:20]


def test_host_inference_matches_gpu_kernel(torch):
    """The planner's host forward pass and arma_gpu_mlp_forward compute the
    same network output for the same standardised features."""
    import ctypes
    from paper_2502_03000_gb300 import costmodel as cm
    from synth.dags import random_dag
    rng = np.random.default_rng(5)
    F, H = ag.N_FEATURES, cm.HIDDEN
    P = int(ag.lib().arma_gpu_mlp_param_count(F, H))
    params = rng.normal(0, 0.2, P).astype(np.float32)
    plans = []
    for i in range(30):
        nodes, outs, _ = random_dag(99, i, 16, 512, dtype="f32")
        try:
            plans.append(ag.Plan(nodes, outs))
        except ag.ArmaError:
            continue
    feats = np.asarray([p.features() for p in plans], dtype=np.float32)
    mean = feats.mean(axis=0).astype(np.float32)
    scale = (feats.std(axis=0) + 1.0).astype(np.float32)
    ag.load_cost_model(params, mean, scale, H)
    try:
        z = ((feats - mean) / scale).astype(np.float32)
        x = torch.tensor(z, device="cuda").contiguous()
        pd = torch.tensor(params, device="cuda")
        y = torch.empty(len(plans), dtype=torch.float32, device="cuda")
        st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        assert ag.lib().arma_gpu_mlp_forward(ctypes.c_void_p(pd.data_ptr()), F, H, ctypes.c_void_p(x.data_ptr()),
                                             len(plans), ctypes.c_void_p(y.data_ptr()), st) == 0
        yg = y.cpu().numpy().astype(np.float64)
        for p, yk in zip(plans, yg):
            got = math.log(p.predicted_cost() / p.heuristic_cost())
            assert abs(got - yk) <= 1e-6 * max(1.0, abs(yk)), (got, yk)
    finally:
        ag.clear_cost_model()


def test_heuristic_choice_and_guard(torch):
    """ARMA_PLAN_COST_HEURISTIC keeps the candidate with the smallest
    estimate; a network whose pick the estimate rates more than `guard` times
    slower is overruled."""
    from paper_2502_03000_gb300 import costmodel as cm
    from synth.dags import random_dag
    F, H = ag.N_FEATURES, cm.HIDDEN
    P = int(ag.lib().arma_gpu_mlp_param_count(F, H))
    # a network that prefers the candidate with the LARGEST estimate:
    # output = -2 * z_16 (ln estimate), through one hidden unit
    params = np.zeros(P, dtype=np.float32)
    W1, b1 = 0, H * F
    W2, b2 = b1 + H, b1 + H + H * H
    W3 = b2 + H
    params[W1 + 0 * F + cm.HEURISTIC_FEATURE] = 1.0       # h1_0 = relu(z)
    params[W1 + 1 * F + cm.HEURISTIC_FEATURE] = -1.0      # h1_1 = relu(-z)
    params[W2 + 0 * H + 0] = 1.0
    params[W2 + 1 * H + 1] = 1.0
    params[W3 + 0] = -2.0
    params[W3 + 1] = 2.0
    mean = np.zeros(F, dtype=np.float32)
    scale = np.ones(F, dtype=np.float32)
    seen_guard = 0
    for i in range(40):
        nodes, outs, _ = random_dag(123, i, 16, 2048, dtype="f32")
        try:
            cands = ag.candidates(nodes, outs, flags=ag.PLAN_TIER_CHOICE)
        except ag.ArmaError:
            continue
        h = [c.heuristic_cost() for c in cands]
        p = ag.Plan(nodes, outs, flags=ag.PLAN_TIER_CHOICE | ag.PLAN_COST_HEURISTIC)
        assert p.info["choice"]["picked"] == int(np.argmin(h))
        ag.load_cost_model(params, mean, scale, H, guard=1.5)
        try:
            ch = ag.Plan(nodes, outs, flags=ag.PLAN_TIER_CHOICE | ag.PLAN_COST_MLP).info["choice"]
        finally:
            ag.clear_cost_model()
        worst = int(np.argmax(h))
        if h[worst] > 1.5 * min(h):
            assert ch["guarded"] and ch["picked"] == int(np.argmin(h))
            seen_guard += 1
        else:
            assert not ch["guarded"]
    assert seen_guard > 0


def test_candidates_match_oracle(torch):
    """Every candidate the library considers (chain orders, fusion, split-K,
    precision tiers at least as accurate as asked) gives the oracle's result."""
    from paper_2502_03000_gb300 import costmodel as cm
    from synth.dags import input_shapes
    import synth
    dags = [d for d in cm.make_dags(20250203 + 6, 40, lo=16, hi=96, cap_flops=1e8) if d[2] == "f32"][:12]
    for i, (nodes, outs, dt) in enumerate(dags):
        host = [synth.matrix(77 + i, s + 1, r, c, dt) for s, (r, c) in enumerate(input_shapes(nodes))]
        ref = oracle.evaluate(nodes, outs, host)
        for ci, p in cm.candidate_plans(nodes, outs):
            got = p(*[to_dev(h, dt) for h in host])
            torch.cuda.synchronize()
            err = oracle.rel_err(to_host(got[0]), ref[0])
            assert err <= 1e-4, (i, ci, p.info["tier"], err)


def test_shipped_cost_model_beats_heuristic_on_fresh_dags(torch, capsys):
    """The cost network shipped with the library (trained by its own kernels
    on GB300 timings of 4,000 DAGs of the benchmark's generator, seed
    20250203 + 5) ranks the candidates of 500 DAGs drawn with another seed
    better than the FLOP/byte estimate: lower geometric-mean regret against
    the fastest candidate (each candidate timed over at least 1 ms)."""
    from paper_2502_03000_gb300 import costmodel as cm
    import os
    assert os.path.exists(cm.DEFAULT_MODEL), "the shipped cost network is missing"
    net = cm.CostNet.load(cm.DEFAULT_MODEL)
    dags = cm.make_dags(20250203 + 7, 500, lo=16, hi=8192, cap_flops=2e11)
    recs = cm.collect(dags, target_s=1e-3)
    res = cm.evaluate(recs, net, guard=4.0)
    with capsys.disabled():
        print("\nshipped model, fresh DAGs:", {k: round(v, 4) if isinstance(v, float) else v for k, v in res.items()})
    assert res["mlp_regret"] < res["heuristic_regret"], res
    # and the library, given the network, picks what the rule picks
    net.to_library(guard=4.0)
    try:
        _, mlp, _ = cm.picks(recs, net, guard=4.0)
        for d, r in sorted(mlp.items())[:30]:
            assert cm.library_pick(dags[d][0], dags[d][1])[0] == r["cand"]
    finally:
        ag.clear_cost_model()
