"""Tensor-core products (tcgen05, BF16 and split-BF16 tiers) against the FP64
oracle: folded transposes, alpha / beta*C, diagonal scalings, ragged tiles,
split-K, every input element type, and the benchmark size on sampled
entries.  Smallest cases first."""
import numpy as np
import pytest

import oracle
import paper_2502_03000_gb300 as ag
import synth
from paper_2502_03000_gb300 import expr as E
from tests.gpu_util import TOL, check, need_gpu, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return need_gpu()


def product_case(m, n, k, ta, tb, dtype, extra=False):
    g = E.Graph()
    A = g.input(0, k, m, dtype) if ta else g.input(0, m, k, dtype)
    B = g.input(1, n, k, dtype) if tb else g.input(1, k, n, dtype)
    opA = A.t() if ta else A
    opB = B.t() if tb else B
    outs = [opA * opB]
    shapes = [(k, m) if ta else (m, k), (n, k) if tb else (k, n)]
    if extra:
        cdt = "f32" if dtype == "bf16" else dtype
        C = g.input(2, m, n, cdt)
        r, c = g.input(3, m, 1, cdt), g.input(4, n, 1, cdt)
        outs += [2 * opA * opB + C, E.diagmat(r) * (opA * opB) * E.diagmat(c)]
        shapes += [(m, n), (m, 1), (n, 1)]
    nodes, o = g.build(*outs)
    return nodes, o, shapes


def run_case(torch, nodes, outs, shapes, dtype, tier, seed=1, cdt=None):
    host = [synth.matrix(seed, s + 1, r, c, dtype if s < 2 else (cdt or dtype)) for s, (r, c) in enumerate(shapes)]
    plan = ag.Plan(nodes, outs, tier=tier)
    assert any(st["kernel"] == "gemm" for st in plan.info["steps"])
    ins = [to_dev(h, dtype if s < 2 else (cdt or dtype)) for s, h in enumerate(host)]
    got = plan(*ins)
    torch.cuda.synchronize()
    st, info = plan.status()
    assert st == "ok", (st, info)
    return got, oracle.evaluate(nodes, outs, host)


@pytest.mark.parametrize("tier", ["bf16", "split_bf16"])
def test_gemm_tile_exact(torch, tier):
    nodes, outs, shapes = product_case(128, 256, 64, 1, 0, "f64")
    got, ref = run_case(torch, nodes, outs, shapes, "f64", tier)
    check(got, ref, TOL[tier], f"128x256x64 {tier}")


@pytest.mark.parametrize("tier", ["bf16", "split_bf16"])
@pytest.mark.parametrize("ta,tb", [(1, 0), (0, 0), (0, 1), (1, 1)])
@pytest.mark.parametrize("mnk", [(129, 300, 77), (257, 513, 200), (64, 1000, 2000), (300, 2, 129)])
def test_gemm_folded(torch, tier, ta, tb, mnk):
    m, n, k = mnk
    nodes, outs, shapes = product_case(m, n, k, ta, tb, "f64", extra=True)
    got, ref = run_case(torch, nodes, outs, shapes, "f64", tier, seed=m + n + k)
    check(got, ref, TOL[tier], f"{mnk} {ta}{tb} {tier}")


@pytest.mark.parametrize("dtype,tier,tol", [("f32", "native", TOL["split_bf16"]), ("f32", "bf16", TOL["bf16"]),
                                            ("bf16", "native", TOL["bf16"]), ("bf16", "split_bf16", 1e-6)])
def test_gemm_input_types(torch, dtype, tier, tol):
    nodes, outs, shapes = product_case(200, 330, 520, 1, 0, dtype, extra=True)
    got, ref = run_case(torch, nodes, outs, shapes, dtype, tier, cdt="f32" if dtype == "bf16" else dtype)
    check(got, ref, tol, f"{dtype} {tier}")


@pytest.mark.parametrize("mnk", [(129, 300, 77), (256, 512, 1000), (1000, 64, 4096), (300, 2, 129)])
def test_gemm_bf16_operands_in_place(torch, mnk):
    """BF16 operands that are already K-major (op(A) = A^T, op(B) = B) are
    read by TMA in place.  The result equals, bit for bit, the one through the
    preparation pass (forced by a leading dimension that is not a multiple of
    8), and the oracle within the BF16 tolerance."""
    m, n, k = mnk
    nodes, outs, shapes = product_case(m, n, k, 1, 0, "bf16", extra=True)
    host = [synth.matrix(m + k, s + 1, r, c, "bf16" if s < 2 else "f32") for s, (r, c) in enumerate(shapes)]
    plan = ag.Plan(nodes, outs, tier="bf16")
    direct = plan(*[to_dev(h, "bf16" if s < 2 else "f32") for s, h in enumerate(host)])
    torch.cuda.synchronize()
    g = E.Graph()
    A = g.input(0, k, m, "bf16", ld=k + 1)
    B = g.input(1, k, n, "bf16", ld=k + 1)
    C = g.input(2, m, n, "f32")
    r, c = g.input(3, m, 1, "f32"), g.input(4, n, 1, "f32")
    nodes2, outs2 = g.build(A.t() * B, 2 * A.t() * B + C, E.diagmat(r) * (A.t() * B) * E.diagmat(c))
    plan2 = ag.Plan(nodes2, outs2, tier="bf16")
    ins2 = [to_dev(host[0], "bf16", pad=1), to_dev(host[1], "bf16", pad=1)] + \
        [to_dev(h, "f32") for h in host[2:]]
    prepared = plan2(*ins2)
    torch.cuda.synchronize()
    for x, y in zip(direct, prepared):
        assert torch.equal(x, y)
    check(direct, oracle.evaluate(nodes, outs, host), TOL["bf16"], f"{mnk} in place")


@pytest.mark.parametrize("k", [1, 8, 4096, 9000])
def test_gemm_split_k(torch, k):
    nodes, outs, shapes = product_case(256, 256, k, 1, 0, "f64")
    got, ref = run_case(torch, nodes, outs, shapes, "f64", "split_bf16", seed=k)
    check(got, ref, TOL["split_bf16"], f"k={k}")


def test_gemm_repeatable(torch):
    nodes, outs, shapes = product_case(384, 512, 1024, 1, 0, "f32")
    a, _ = run_case(torch, nodes, outs, shapes, "f32", "split_bf16")
    b, _ = run_case(torch, nodes, outs, shapes, "f32", "split_bf16")
    assert torch.equal(a[0], b[0])


@pytest.mark.parametrize("tier", ["split_bf16", "bf16", "f64"])
def test_gemm_benchmark_size_sampled(torch, tier):
    """2*trans(A)*B + C at 8192^3 with FP64 inputs, in the launch
    configuration the benchmark times (the FP64 tier is the DFMA product);
    sampled entries against the oracle's own increasing-l sums."""
    n = 8192
    nodes, outs = E.config_products(n, "f64")
    host = [synth.matrix(20250203 + 3, s + 1, n, n, "f64") for s in range(3)]
    plan = ag.Plan(nodes, outs, tier=tier)
    ins = [to_dev(h) for h in host]
    (D,) = plan(*ins)
    torch.cuda.synchronize()
    rng = np.random.default_rng(3)
    ii = rng.integers(0, n, 256)
    jj = rng.integers(0, n, 256)
    At = np.asfortranarray(host[0].T)   # trans(A) as stored values
    ref = 2.0 * oracle.matmul_entries(At, host[1], ii, jj) + host[2][ii, jj]
    got = D[torch.as_tensor(ii), torch.as_tensor(jj)].double().cpu().numpy()
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err <= TOL[tier], err


# ---- FP64 products from exact BF16 slices (tier f64_sliced) ----

@pytest.mark.parametrize("ta,tb", [(1, 0), (0, 0), (0, 1), (1, 1)])
@pytest.mark.parametrize("mnk", [(129, 300, 77), (257, 513, 2100), (64, 1000, 1024), (300, 2, 129), (2, 2, 1)])
def test_sliced_f64_folded(torch, ta, tb, mnk):
    """every transpose combination, ragged tiles, K across several 1024-chunks
    and split-K, alpha / beta*C / diagonal scalings: FP64 accuracy"""
    m, n, k = mnk
    nodes, outs, shapes = product_case(m, n, k, ta, tb, "f64", extra=True)
    got, ref = run_case(torch, nodes, outs, shapes, "f64", "f64_sliced", seed=m + n + 3 * k)
    check(got, ref, TOL["f64"], f"{mnk} {ta}{tb} f64_sliced")


def test_sliced_f64_exact_on_integers(torch):
    """integer operands (|x| < 2^20): every slice product and every FP64 sum
    is exact, so the result equals the integer product bit for bit"""
    rng = np.random.default_rng(5)
    m, n, k = 300, 200, 3000
    A = rng.integers(-(1 << 20) + 1, 1 << 20, size=(k, m)).astype(np.float64)
    B = rng.integers(-(1 << 20) + 1, 1 << 20, size=(k, n)).astype(np.float64)
    g = E.Graph()
    a, b = g.input(0, k, m), g.input(1, k, n)
    nodes, outs = g.build(a.t() * b)
    (D,) = ag.Plan(nodes, outs, tier="f64_sliced")(to_dev(A), to_dev(B))
    torch.cuda.synchronize()
    ref = A.T.astype(object) @ B.astype(object)       # exact integers
    got = to_host(D)
    assert np.array_equal(got, np.asarray(ref, dtype=np.float64))


def test_sliced_f64_scaling_and_specials(torch):
    """rows and columns scaled over 2^+-300 (each scaled by its own maximum),
    a zero row, a zero column; a NaN in a row of A makes that output row NaN
    and nothing else"""
    m, n, k = 150, 140, 700
    A = synth.matrix(91, 1, k, m, "f64") * (2.0 ** np.linspace(-300, 300, m))[None, :]
    B = synth.matrix(91, 2, k, n, "f64") * (2.0 ** np.linspace(200, -200, n))[None, :]
    A[:, 7] = 0.0
    B[:, 11] = 0.0
    g = E.Graph()
    a, b = g.input(0, k, m), g.input(1, k, n)
    nodes, outs = g.build(a.t() * b)
    plan = ag.Plan(nodes, outs, tier="f64_sliced")
    (D,) = plan(to_dev(A), to_dev(B))
    torch.cuda.synchronize()
    ref = oracle.matmul(np.asfortranarray(A.T), B)
    got = to_host(D)
    # relative to each entry's own scale 2^(e_i + f_j): row-column scaled error
    scale = np.abs(A).max(axis=0)[:, None] * np.abs(B).max(axis=0)[None, :] * k
    scale[scale == 0] = 1.0
    assert np.max(np.abs(got - ref) / scale) <= 1e-14
    assert np.all(got[7, :] == 0.0) and np.all(got[:, 11] == 0.0)
    A2 = A.copy()
    A2[3, 20] = np.nan
    (D2,) = plan(to_dev(A2), to_dev(B))
    torch.cuda.synchronize()
    got2 = to_host(D2)
    assert np.all(np.isnan(got2[20, :]))
    mask = np.ones(m, bool)
    mask[20] = False
    assert np.array_equal(got2[mask], got[mask])


def test_sliced_f64_benchmark_size_sampled(torch):
    """2*trans(A)*B + C at 8192^3 with tier f64_sliced, in the benchmark's
    launch configuration; sampled entries against the oracle's sums"""
    n = 8192
    nodes, outs = E.config_products(n, "f64")
    host = [synth.matrix(20250203 + 3, s + 1, n, n, "f64") for s in range(3)]
    plan = ag.Plan(nodes, outs, tier="f64_sliced")
    (D,) = plan(*[to_dev(h) for h in host])
    torch.cuda.synchronize()
    assert plan.status()[0] == "ok"
    rng = np.random.default_rng(3)
    ii = rng.integers(0, n, 256)
    jj = rng.integers(0, n, 256)
    At = np.asfortranarray(host[0].T)
    ref = 2.0 * oracle.matmul_entries(At, host[1], ii, jj) + host[2][ii, jj]
    got = D[torch.as_tensor(ii), torch.as_tensor(jj)].double().cpu().numpy()
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err <= TOL["f64"], err


@pytest.mark.parametrize("tier", ["split_bf16", "bf16", "f64"])
def test_requested_split_counts(torch, tier):
    """every K split count a plan may ask for (ARMA_PLAN_SPLITS) gives the
    oracle's product at the tier's tolerance, tensor-core and DFMA kernels"""
    m, n, k = 300, 200, 2500
    nodes, outs, shapes = product_case(m, n, k, 1, 0, "f64", extra=True)
    host = [synth.matrix(31, s + 1, r, c, "f64") for s, (r, c) in enumerate(shapes)]
    ref = oracle.evaluate(nodes, outs, host)
    ins = [to_dev(h, "f64") for h in host]
    seen = set()
    for kreq in (1, 2, 3, 4, 8, 15):
        plan = ag.Plan(nodes, outs, tier=tier, flags=ag.PLAN_SPLITS(kreq))
        sp = [st["splits"] for st in plan.info["steps"] if st["kernel"] == "gemm"]
        assert all(1 <= x <= kreq for x in sp)
        seen.add(tuple(sp))
        got = plan(*ins)
        torch.cuda.synchronize()
        assert plan.status()[0] == "ok"
        check(got, ref, TOL[tier if tier != "f64" else "f64"], f"{tier} splits={kreq}")
    assert len(seen) >= 4


def test_autotuner_times_split_counts(torch, tmp_path, monkeypatch):
    """the autotuner times the distinct split counts of a product on the
    caller's operands, keeps the fastest, persists the choice, and reuses it"""
    from paper_2502_03000_gb300 import autotune
    m, n, k = 512, 384, 6000
    nodes, outs, shapes = product_case(m, n, k, 1, 0, "f32", extra=True)
    host = [synth.matrix(32, s + 1, r, c, "f32") for s, (r, c) in enumerate(shapes)]
    ins = [to_dev(h, "f32") for h in host]
    cache = str(tmp_path / "tune.json")
    monkeypatch.setenv("ARMA_AUTOTUNE_CACHE", cache)
    best, times = autotune.tune_plan(nodes, outs, ins, tier="split_bf16", reps=2)
    assert len(times) >= 3 and all(t > 0 for t in times.values())
    got = best(*ins)
    torch.cuda.synchronize()
    check(got, oracle.evaluate(nodes, outs, host), TOL["split_bf16"], "tuned")
    import os
    assert os.path.exists(cache)
    best2, times2 = autotune.tune_plan(nodes, outs, ins, tier="split_bf16", reps=2)
    assert list(times2) == [min(times, key=times.get)]
