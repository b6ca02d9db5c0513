"""Host-side plan choice (no GPU): arma_gpu_plan enumerates candidate plans
(chain order, fusion, split-K, precision tiers) and keeps the one its scorer
ranks fastest; the learned scorer's host forward pass agrees with the FP64
oracle of the network."""
import math

import numpy as np
import pytest

import paper_2502_03000_gb300 as ag
from oracle import mlp as M
from paper_2502_03000_gb300 import expr as E


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2502_03000_gb300 import build
    build.build()
    ag.lib.cache_clear()
    yield
    ag.clear_cost_model()


def chain_expr(dims, dtype="f32"):
    g = E.Graph()
    mats = [g.input(i, dims[i], dims[i + 1], dtype) for i in range(len(dims) - 1)]
    prod = mats[0]
    for m in mats[1:]:
        prod = prod * m
    return g.build(2 * prod)


def test_candidates_distinct_and_cover_variants():
    nodes, outs = chain_expr((64, 2048, 32, 512, 8))
    cands = ag.candidates(nodes, outs)
    infos = [c.info for c in cands]
    steps = [str([(s["kernel"], s["note"]) for s in i["steps"]]) for i in infos]
    assert len(set(steps)) == len(steps), "duplicate candidates"
    chains = {i["chain"] for i in infos}
    assert {"dp", "paper_greedy", "left_to_right"} <= chains
    assert any("nosplit" in s for s in steps)
    tiers = {i["tier"] for i in ag.candidates(nodes, outs, flags=ag.PLAN_TIER_CHOICE) for i in [i.info]}
    assert tiers == {"native", "f64"}


def test_tier_choice_only_more_accurate():
    g = E.Graph()
    A, B = g.input(0, 300, 200, "bf16"), g.input(1, 200, 100, "bf16")
    nodes, outs = g.build(A * B)
    tiers = {c.info["tier"] for c in ag.candidates(nodes, outs, tier="bf16", flags=ag.PLAN_TIER_CHOICE)}
    assert tiers == {"bf16", "split_bf16", "f64"}
    tiers = {c.info["tier"] for c in ag.candidates(nodes, outs, tier="split_bf16", flags=ag.PLAN_TIER_CHOICE)}
    assert tiers == {"split_bf16", "f64"}
    tiers = {c.info["tier"] for c in ag.candidates(nodes, outs, tier="f64", flags=ag.PLAN_TIER_CHOICE)}
    assert tiers == {"f64"}


def test_heuristic_choice_is_the_smallest_estimate():
    for dims in [(64, 2048, 32, 512, 8), (1000, 10, 1000, 10), (4096, 8192, 512, 4096, 1)]:
        nodes, outs = chain_expr(dims)
        h = [c.heuristic_cost() for c in ag.candidates(nodes, outs, flags=ag.PLAN_TIER_CHOICE)]
        p = ag.Plan(nodes, outs, flags=ag.PLAN_TIER_CHOICE | ag.PLAN_COST_HEURISTIC)
        ch = p.info["choice"]
        assert ch["scorer"] == "heuristic" and ch["picked"] == int(np.argmin(h))
        assert len(ch["candidates"]) == len(h)
        assert math.isclose(p.heuristic_cost(), min(h), rel_tol=1e-12)


def test_mlp_flag_without_model_uses_estimate():
    ag.clear_cost_model()
    nodes, outs = chain_expr((64, 2048, 32, 512, 8))
    ch = ag.Plan(nodes, outs, flags=ag.PLAN_COST_MLP).info["choice"]
    assert ch["scorer"] == "heuristic" and ch["picked"] == ch["heuristic_pick"]
    with pytest.raises(ag.ArmaError) as ei:
        ag.Plan(nodes, outs).predicted_cost()
    assert ei.value.status == "unsupported"


def test_host_forward_matches_network_oracle():
    """predicted seconds = estimate * exp(network(z)), z the standardised
    features; the network output against the FP64 oracle's forward pass."""
    F, H = ag.N_FEATURES, 64
    rng = np.random.default_rng(11)
    params = rng.normal(0, 0.15, M.param_count(F, H)).astype(np.float32)
    plans = []
    for dims in [(64, 2048, 32, 512, 8), (1000, 10, 1000, 10), (300, 300, 300), (17, 4096, 9)]:
        nodes, outs = chain_expr(dims)
        plans += ag.candidates(nodes, outs, flags=ag.PLAN_TIER_CHOICE)
    feats = np.asarray([p.features() for p in plans], dtype=np.float32)
    mean = feats.mean(axis=0).astype(np.float32)
    scale = (feats.std(axis=0) + 0.5).astype(np.float32)
    ag.load_cost_model(params, mean, scale, H)
    try:
        z = (feats.astype(np.float64) - mean) / scale
        y_ref, _ = M.forward(params.astype(np.float64), z, F, H)
        for p, yr in zip(plans, y_ref):
            got = math.log(p.predicted_cost() / p.heuristic_cost())
            assert abs(got - yr) <= 1e-4 * max(1.0, abs(yr)), (got, yr)
    finally:
        ag.clear_cost_model()


def test_cost_model_load_validates():
    F, H = ag.N_FEATURES, 8
    P = M.param_count(F, H)
    ok = dict(params=np.zeros(P), mean=np.zeros(F), scale=np.ones(F), hidden=H)
    ag.load_cost_model(**ok)
    ag.clear_cost_model()
    with pytest.raises(ag.ArmaError):
        ag.load_cost_model(np.zeros(P), np.zeros(F), np.zeros(F), H)          # zero scale
    with pytest.raises(ag.ArmaError):
        ag.load_cost_model(np.zeros(P), np.zeros(F - 1), np.ones(F - 1), H)   # wrong feature count
    with pytest.raises(ag.ArmaError):
        ag.load_cost_model(np.zeros(P), np.zeros(F), np.ones(F), H, guard=-1.0)
    p = np.zeros(P)
    p[0] = np.nan
    with pytest.raises(ag.ArmaError):
        ag.load_cost_model(p, np.zeros(F), np.ones(F), H)


def test_refinement_limit_flag_encoding():
    assert ag.PLAN_REFINE_STEPS(1) == 1 << 16 and ag.PLAN_REFINE_STEPS(15) == 15 << 16
    assert ag.PLAN_REFINE_STEPS(3) & ag.PLAN_REFINE_MASK == ag.PLAN_REFINE_STEPS(3)
    nodes, outs = E.config_solve(64, 2)
    ag.Plan(nodes, outs, tier="lu32_ir64", flags=ag.PLAN_REFINE_STEPS(2))


def test_wait_limit_roundtrip():
    old = ag.set_wait_limit_ns(12345)
    assert ag.set_wait_limit_ns(old) == 12345
    assert ag.lib().arma_gpu_status_string(10) == b"a bounded device-side wait ran out"


def test_split_count_flag():
    """ARMA_PLAN_SPLITS(k): the plan's products report the split count they
    will use, k or fewer (K blocks), and NO_SPLITK is one split"""
    assert ag.PLAN_SPLITS(3) == 3 << 20
    with pytest.raises(ValueError):
        ag.PLAN_SPLITS(16)
    nodes, outs = E.config_products(1024, "f64")
    for tier in ("bf16", "split_bf16", "f64"):
        for k in (1, 2, 4, 8, 15):
            p = ag.Plan(nodes, outs, tier=tier, flags=ag.PLAN_SPLITS(k))
            sp = [s["splits"] for s in p.info["steps"] if s["kernel"] == "gemm"]
            assert sp and all(1 <= x <= k for x in sp), (tier, k, sp)
        p = ag.Plan(nodes, outs, tier=tier, flags=ag.PLAN_NO_SPLITK | ag.PLAN_SPLITS(8))
        assert [s["splits"] for s in p.info["steps"] if s["kernel"] == "gemm"] == [1]


def test_autotune_table_keeps_split_choices(tmp_path):
    from paper_2502_03000_gb300 import autotune
    nodes, outs = E.config_products(256, "f32")
    sig = autotune.plan_signature(nodes, outs, "split_bf16", 0)
    autotune._cache[sig] = "splits4"
    path = str(tmp_path / "t.json")
    autotune.save(path)
    del autotune._cache[sig]
    assert autotune.load(path) >= 1 and autotune._cache[sig] == "splits4"


def test_planner_workload_dags_all_plan():
    """The cost-model workload keeps only DAGs the library plans: BF16 DAGs
    that do not conform are drawn again in FP32, and every kept DAG plans
    both literally and optimised."""
    from paper_2502_03000_gb300 import costmodel as cm
    dags = cm.make_dags(20250203 + 5, 150)
    assert len(dags) == 150
    kinds = {dt for _, _, dt in dags}
    assert kinds == {"f32", "bf16"}
    for nodes, outs, dt in dags:
        lit = ag.Plan(nodes, outs, flags=ag.PLAN_LITERAL)
        opt = ag.Plan(nodes, outs)
        assert lit.info["flops"] <= 2e11
        # fusion and folding only remove launches
        assert len(opt.info["steps"]) <= len(lit.info["steps"])


def test_concurrent_planning_matches_sequential():
    """arma_gpu_plan from 8 host threads at once (ctypes drops the GIL
    around each call) gives the same decision logs as one thread, with and
    without the cost-model choice."""
    import json
    from concurrent.futures import ThreadPoolExecutor
    from paper_2502_03000_gb300 import costmodel as cm
    dags = cm.make_dags(20250203 + 9, 64)
    flag_sets = [0, ag.PLAN_LITERAL, ag.PLAN_TIER_CHOICE | ag.PLAN_COST_HEURISTIC]

    def plan_all(order):
        out = {}
        for i in order:
            nodes, outs, _ = dags[i % len(dags)]
            f = flag_sets[i % len(flag_sets)]
            out[i] = json.dumps(ag.Plan(nodes, outs, flags=f).info, sort_keys=True)
        return out

    work = list(range(3 * len(dags)))
    ref = plan_all(work)
    with ThreadPoolExecutor(8) as ex:
        parts = list(ex.map(plan_all, [work[t::8][::-1] for t in range(8)]))
    got = {}
    for p in parts:
        got.update(p)
    assert got == ref


def test_model_swaps_during_concurrent_planning():
    """While host threads plan with ARMA_PLAN_COST_MLP, another thread loads
    and clears the shipped network over and over.  Every plan sees one
    consistent state: its pick is the network's pick when its log says the
    network scored it, and the estimate's otherwise."""
    import json
    import threading
    from concurrent.futures import ThreadPoolExecutor
    from paper_2502_03000_gb300 import costmodel as cm
    with open(cm.DEFAULT_MODEL) as f:
        d = json.load(f)
    model = dict(params=d["params"], mean=d["mean"], scale=d["scale"], hidden=d["hidden"], guard=4.0)
    dags = cm.make_dags(20250203 + 10, 48)
    flags = ag.PLAN_TIER_CHOICE | ag.PLAN_COST_MLP

    def picks():
        return [ag.Plan(n, o, flags=flags).info["choice"] for n, o, _ in dags]

    ag.clear_cost_model()
    heur = [c["picked"] for c in picks()]
    ag.load_cost_model(**model)
    try:
        first = picks()
        assert all(c["scorer"] == "mlp" for c in first)
        mlp = [c["picked"] for c in first]
        stop = threading.Event()

        def swap():
            while not stop.is_set():
                ag.clear_cost_model()
                ag.load_cost_model(**model)

        t = threading.Thread(target=swap)
        t.start()
        try:
            with ThreadPoolExecutor(6) as ex:
                runs = list(ex.map(lambda _: picks(), range(12)))
        finally:
            stop.set()
            t.join()
        seen = set()
        for run in runs:
            for i, c in enumerate(run):
                seen.add(c["scorer"])
                assert c["picked"] == (mlp[i] if c["scorer"] == "mlp" else heur[i]), (i, c)
        assert seen <= {"mlp", "heuristic"}
    finally:
        ag.clear_cost_model()
