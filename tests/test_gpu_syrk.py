"""Symmetric products X*X^T and X^T*X (Sec. III (8); the run-time analysis of
Sec. II that maps them to xSYRK): only the lower-triangle tiles are
computed and the upper triangle is mirrored.  Checked against the FP64
oracle, for exact symmetry of the result, against the general product of
the same plan without the rewrite, and for the pointer comparison that
finds two input slots bound to the same matrix."""
import numpy as np
import pytest

import oracle
import paper_2502_03000_gb300 as ag
from paper_2502_03000_gb300 import expr as E
from tests.gpu_util import TOL, check, inputs, need_gpu, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return need_gpu()


def evaluate(nodes, outs, ins, flags=0, tier="native"):
    import torch as T
    plan = ag.Plan(nodes, outs, tier=tier, flags=flags)
    got = plan(*ins)
    T.cuda.synchronize()
    return plan, got


def symmetric_exactly(d):
    d = to_host(d)
    return d.shape[0] == d.shape[1] and np.array_equal(d, d.T)


SHAPES = [(2, 3), (64, 64), (65, 17), (130, 300), (257, 1), (1000, 1000)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("form", ["AAt", "AtA"])
def test_symmetric_product(torch, dtype, shape, form):
    m, k = shape if form == "AAt" else shape[::-1]
    g = E.Graph()
    A = g.input(0, m, k, dtype)
    e = 0.5 * (A * A.t()) if form == "AAt" else A.t() * A
    nodes, outs = g.build(e)
    host = inputs(1100 + m + k, [(m, k)], dtype)
    ins = [to_dev(host[0], dtype)]
    plan, got = evaluate(nodes, outs, ins)
    assert plan.info["steps"][-1]["kernel"] == "syrk"
    tol = TOL[dtype] if dtype != "f32" else TOL["split_bf16"] * 10
    check(got, oracle.evaluate(nodes, outs, host), tol, f"{form} {dtype} {shape}")
    assert symmetric_exactly(got[0])
    _, gen = evaluate(nodes, outs, ins, flags=ag.PLAN_NO_SYRK)
    if dtype == "f64":
        # FP64 SIMT tiles: the same sum in the same order for every element
        assert np.array_equal(to_host(got[0]), to_host(gen[0]))
    else:
        check(got, [to_host(gen[0])], tol, "syrk vs gemm")


@pytest.mark.parametrize("tier", ["f64", "split_bf16", "bf16"])
@pytest.mark.parametrize("n,k", [(300, 4096), (2000, 96), (1537, 700)])
def test_symmetric_product_tiers(torch, tier, n, k):
    """FP64 data under each product tier: split-K partials (few tiles, long
    K), many tiles, and a ragged edge on both tile heights"""
    g = E.Graph()
    A = g.input(0, n, k)
    nodes, outs = g.build(A * A.t())
    host = inputs(1200 + n, [(n, k)], "f64")
    plan, got = evaluate(nodes, outs, [to_dev(host[0])], tier=tier)
    assert plan.info["steps"][-1]["kernel"] == "syrk"
    check(got, oracle.evaluate(nodes, outs, host), TOL[tier], f"{tier} {n}x{k}")
    assert symmetric_exactly(got[0])


@pytest.mark.parametrize("layout", [dict(pad=5), dict(pad=3, offset=1)])
def test_symmetric_product_padded(torch, layout):
    m, k = 203, 77
    g = E.Graph()
    A = g.input(0, m, k, "f64", ld=m + layout["pad"])
    nodes, outs = g.build(A * A.t(), E.trace(A * A.t()))
    host = inputs(1300, [(m, k)], "f64")
    plan, got = evaluate(nodes, outs, [to_dev(host[0], "f64", **layout)])
    check(got, oracle.evaluate(nodes, outs, host), TOL["f64"], str(layout))
    assert symmetric_exactly(got[0])


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_same_matrix_in_two_slots(torch, dtype):
    """A*B^T with both slots bound to one matrix takes the symmetric path
    (exactly symmetric result); bound to two matrices it is the general
    product"""
    n, k = 333, 129
    g = E.Graph()
    A, B = g.input(0, n, k, dtype), g.input(1, n, k, dtype)
    nodes, outs = g.build(A * B.t())
    host = inputs(1400, [(n, k), (n, k)], dtype)
    tol = TOL[dtype] if dtype != "f32" else TOL["split_bf16"] * 10
    a = to_dev(host[0], dtype)
    plan, got = evaluate(nodes, outs, [a, a])
    assert plan.info["steps"][-1]["kernel"] == "gemm"
    check(got, oracle.evaluate(nodes, outs, [host[0], host[0]]), tol, "same")
    assert symmetric_exactly(got[0])
    _, got2 = evaluate(nodes, outs, [a, to_dev(host[1], dtype)])
    check(got2, oracle.evaluate(nodes, outs, host), tol, "different")
    assert not symmetric_exactly(got2[0])


def test_symmetric_product_of_expression(torch):
    """X*X^T where X = A + B is computed once and multiplied symmetrically;
    and 2*X^T*X inside a larger sum"""
    m, k = 150, 90
    g = E.Graph()
    A, B = g.input(0, m, k), g.input(1, m, k)
    C = g.input(2, k, k)
    X = A + 2.0 * B
    host = inputs(1500, [(m, k), (m, k), (k, k)], "f64")
    for e in (X * X.t(), 2.0 * (X.t() * X) - C):
        nodes, outs = g.build(e, E.accu(e))
        _, got = evaluate(nodes, outs, [to_dev(h) for h in host])
        check(got, oracle.evaluate(nodes, outs, host), TOL["f64"], "expr")
