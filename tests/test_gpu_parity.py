"""Parity of the CUDA path with the CPU FP64 oracle, element by element, on
seeded inputs: the paper's expressions (Sec. III), the fused benchmark
expression, folded transposes / scalars / diagonals, chains, and the edge
cases (empty, 1 x 1, ragged, padded leading dimensions, misaligned
pointers).  Every call goes through the C ABI."""
import numpy as np
import pytest

import oracle
import paper_2502_03000_gb300 as ag
import synth
from paper_2502_03000_gb300 import expr as E
from tests.gpu_util import TOL, check, inputs, need_gpu, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return need_gpu()


def run(nodes, outs, host, dtype, flags=0, tier="native", **kw):
    plan = ag.Plan(nodes, outs, tier=tier, flags=flags)
    ins = [to_dev(h, dtype, **kw) for h in host]
    got = plan(*ins)
    import torch as T
    T.cuda.synchronize()
    return got


def plain_inputs(seed, n, dtype):
    return inputs(seed, [(n, n)] * 4 + [(n, 1)], dtype)


@pytest.mark.parametrize("n", [1, 2, 37, 130, 256])
@pytest.mark.parametrize("flags", [0, ag.PLAN_LITERAL, ag.PLAN_NO_FUSE])
def test_plain_expressions_f64(torch, n, flags):
    host = plain_inputs(11 + n, n, "f64")
    for name, (nodes, outs) in E.config_plain(n, "f64").items():
        got = run(nodes, outs, host, "f64", flags)
        check(got, oracle.evaluate(nodes, outs, host), TOL["f64"], f"{name} n={n} flags={flags}")


@pytest.mark.parametrize("n", [33, 256])
def test_plain_expressions_f32(torch, n):
    host = plain_inputs(21, n, "f32")
    for name, (nodes, outs) in E.config_plain(n, "f32").items():
        for flags in (0, ag.PLAN_LITERAL):
            got = run(nodes, outs, host, "f32", flags)
            check(got, oracle.evaluate(nodes, outs, host), TOL["f32"], f"{name} f32 flags={flags}")


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("shape", [(257, 263), (1, 1), (8, 8), (1000, 3), (3, 1000)])
@pytest.mark.parametrize("flags", [0, ag.PLAN_LITERAL])
def test_fused_expression(torch, dtype, shape, flags):
    m, n = shape
    g = E.Graph()
    A, B, C, D = (g.input(s, m, n, dtype) for s in range(4))
    out = A % B + 3 * C - D / 2
    nodes, outs = g.build(out, E.accu(out), E.norm_fro(out))
    host = inputs(31, [shape] * 4, dtype)
    got = run(nodes, outs, host, dtype, flags)
    ref = oracle.evaluate(nodes, outs, host)
    tol = TOL[dtype]
    check(got[:1], ref[:1], tol, f"out {dtype} {shape}")
    # the reductions of a BF16-stored result are computed from the
    # unrounded values when fused; BF16-rounded temporaries in the literal plan
    tol_red = TOL["f32"] if (dtype == "bf16" and flags == 0) else tol
    check(got[1:], ref[1:], tol_red, f"reductions {dtype} {shape}")


@pytest.mark.parametrize("layout", [dict(pad=3), dict(offset=1), dict(pad=5, offset=3)])
def test_fused_padded_and_misaligned(torch, layout):
    m, n = 129, 67
    g = E.Graph()
    ld = m + layout.get("pad", 0)
    A, B, C, D = (g.input(s, m, n, "f64", ld=ld) for s in range(4))
    out = A % B + 3 * C - D / 2
    nodes, outs = g.build(out, E.accu(out))
    host = inputs(41, [(m, n)] * 4, "f64")
    got = run(nodes, outs, host, "f64", **layout)
    check(got, oracle.evaluate(nodes, outs, host), TOL["f64"], str(layout))


def test_empty_inputs(torch):
    g = E.Graph()
    A, B = g.input(0, 0, 5), g.input(1, 0, 5)
    out = A + B
    nodes, outs = g.build(out, E.accu(out), E.norm_fro(out))
    host = [np.zeros((0, 5)), np.zeros((0, 5))]
    plan = ag.Plan(nodes, outs)
    import torch as T
    ins = [T.zeros((5, 1), dtype=T.float64, device="cuda").t()[:0, :] for _ in range(2)]
    got = plan(*ins)
    T.cuda.synchronize()
    assert got[0].shape == (0, 5)
    assert to_host(got[1]) == 0.0 and to_host(got[2]) == 0.0


def test_elementwise_views(torch):
    """transposed operands, diagonal masks, broadcasts and trace of an
    elementwise expression (the strided and diagonal modes of the fused pass)"""
    m = 45
    g = E.Graph()
    A, B = g.input(0, m, m), g.input(1, m, m)
    v = g.input(2, m, 1)
    e1 = A + B.t()
    e2 = E.diagmat(A) + 2 * B
    e3 = E.trace(A % B - 3 * A)
    e4 = E.diagmat(v) - A
    nodes, outs = g.build(e1, e2, e3, e4)
    host = inputs(51, [(m, m), (m, m), (m, 1)], "f64")
    for flags in (0, ag.PLAN_LITERAL):
        got = run(nodes, outs, host, "f64", flags)
        check(got, oracle.evaluate(nodes, outs, host), TOL["f64"], f"views flags={flags}")


@pytest.mark.parametrize("ta,tb", [(0, 0), (1, 0), (0, 1), (1, 1)])
@pytest.mark.parametrize("mnk", [(64, 64, 64), (70, 33, 129), (1, 40, 17), (40, 1, 17), (3, 5, 1)])
def test_products_folded(torch, ta, tb, mnk):
    m, n, k = mnk
    g = E.Graph()
    A = g.input(0, k, m) if ta else g.input(0, m, k)
    B = g.input(1, n, k) if tb else g.input(1, k, n)
    C = g.input(2, m, n)
    r, c = g.input(3, m, 1), g.input(4, n, 1)
    opA = A.t() if ta else A
    opB = B.t() if tb else B
    e1 = 2 * opA * opB + C
    e2 = E.diagmat(r) * (opA * opB) * E.diagmat(c)
    e3 = -(opA * opB) / 4 - C
    e4 = E.trace(opA * opB * E.trans(C))
    nodes, outs = g.build(e1, e2, e3, e4)
    shapes = [(k, m) if ta else (m, k), (n, k) if tb else (k, n), (m, n), (m, 1), (n, 1)]
    host = inputs(61 + m + n + k, shapes, "f64")
    for flags in (0, ag.PLAN_LITERAL):
        got = run(nodes, outs, host, "f64", flags)
        check(got, oracle.evaluate(nodes, outs, host), TOL["f64"], f"products {ta}{tb} {mnk} {flags}")


@pytest.mark.parametrize("ta,tb", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_trace_of_product(torch, ta, tb):
    for (m, k, n) in [(50, 70, 50), (33, 7, 40), (1, 9, 1), (129, 257, 100)]:
        g = E.Graph()
        A = g.input(0, k, m) if ta else g.input(0, m, k)
        B = g.input(1, n, k) if tb else g.input(1, k, n)
        e = E.trace(0.5 * (A.t() if ta else A) * (B.t() if tb else B))
        nodes, outs = g.build(e)
        shapes = [(k, m) if ta else (m, k), (n, k) if tb else (k, n)]
        host = inputs(71 + m, shapes, "f64")
        got = run(nodes, outs, host, "f64")
        check(got, oracle.evaluate(nodes, outs, host), TOL["f64"], f"trace {ta}{tb} {(m, k, n)}")


@pytest.mark.parametrize("dims", [(40, 80, 5, 40, 1), (12, 12, 6, 4, 3), (7, 1, 9, 2)])
@pytest.mark.parametrize("flags", [0, ag.PLAN_CHAIN_LEFT, ag.PLAN_CHAIN_GREEDY, ag.PLAN_LITERAL])
def test_chains(torch, dims, flags):
    nodes, outs = E.config_chain(dims, "f64")
    host = inputs(81, [(dims[i], dims[i + 1]) for i in range(len(dims) - 1)], "f64")
    got = run(nodes, outs, host, "f64", flags)
    check(got, oracle.evaluate(nodes, outs, host), TOL["f64"], f"chain {dims} {flags}")


def test_deterministic(torch):
    nodes, outs = E.config_fused(1031, "f32")
    host = inputs(91, [(1031, 1031)] * 4, "f32")
    a = run(nodes, outs, host, "f32")
    b = run(nodes, outs, host, "f32")
    for x, y in zip(a, b):
        assert torch.equal(x, y)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_fused_full_size(torch, dtype):
    """The benchmark workload at its full size (8192 x 8192), in the launch
    configuration the benchmark times, against the oracle's literal
    evaluation of the same inputs."""
    n = 8192
    nodes, outs = E.config_fused(n, dtype)
    host = inputs(20250203 + 2, [(n, n)] * 4, dtype)
    got = run(nodes, outs, host, dtype)
    ref = oracle.evaluate(nodes, outs, host)
    check(got, ref, TOL[dtype], f"full size {dtype}")


@pytest.mark.parametrize("scale", [1e-30, 1e-20, 1.0, 1e20, 1e36])
def test_fused_f64_reductions_any_magnitude(torch, scale):
    """FP64 sums and sums of squares are carried as float pairs when the
    values fit a float's exponent range and in FP64 otherwise; both routes
    (and a mix of them in one pass) must meet the FP64 tolerance."""
    m, n = 300, 211
    g = E.Graph()
    A, B, C, D = (g.input(s, m, n, "f64") for s in range(4))
    out = A % B + 3 * C - D / 2
    nodes, outs = g.build(out, E.accu(out), E.norm_fro(out))
    host = inputs(97, [(m, n)] * 4, "f64")
    host = [h * scale for h in host]
    host[2][:, : n // 2] *= 1e-12          # a spread of magnitudes inside one pass
    got = run(nodes, outs, host, "f64")
    check(got, oracle.evaluate(nodes, outs, host), TOL["f64"], f"scale {scale}")


@pytest.mark.parametrize("s", [1e-50, 3e-13, 1e13, 1e60])
def test_fused_f64_extreme_scalars(torch, s):
    """scalars outside the float-pair range send the pass to native FP64"""
    m, n = 131, 97
    g = E.Graph()
    A, B = g.input(0, m, n), g.input(1, m, n)
    out = s * A + B % A
    nodes, outs = g.build(out, E.accu(out), E.norm_fro(out))
    host = inputs(98, [(m, n)] * 2, "f64")
    got = run(nodes, outs, host, "f64")
    check(got, oracle.evaluate(nodes, outs, host), TOL["f64"], f"scalar {s}")


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_fused_power_of_two_load_edges(torch, dtype):
    """s*D with s = +-2^e is loaded by exponent arithmetic in FP64 passes;
    zeros, subnormals, values that overflow or underflow, infinities and NaNs
    take the FP64 multiply.  With B = 0 the products add only zeros, so the
    result equals s*D exactly."""
    m, n = 67, 33
    rng = np.random.default_rng(5)
    D = rng.uniform(-1, 1, (m, n)) * np.exp2(rng.integers(-60, 60, (m, n)))
    big, tiny = (1.5e308, 5e-324) if dtype == "f64" else (3e38, 1.4e-45)
    special = [0.0, -0.0, tiny, -tiny, 1e-310 if dtype == "f64" else 1e-40, big, -big, np.inf, -np.inf, np.nan]
    D.flat[: len(special)] = special
    A = rng.uniform(-1, 1, (m, n))
    B = np.zeros((m, n))
    host = [synth.cast(x, dtype) for x in (A, B, D)]
    for s in (4.0, -0.25, 2.0 ** -1000, -(2.0 ** 900), 1.0, -1.0):
        if dtype == "f32" and abs(np.log2(abs(s))) > 100:
            continue
        g = E.Graph()
        a, b, d = (g.input(k, m, n, dtype) for k in range(3))
        out = s * d + a % b
        nodes, outs = g.build(out)
        plan = ag.Plan(nodes, outs)
        assert "ldp2" in plan.info["steps"][0]["note"], plan.info["steps"][0]["note"]
        (got,) = plan(*[to_dev(h, dtype) for h in host])
        torch.cuda.synchronize()
        want = (synth.cast(s * host[2].astype(np.float64), dtype) if dtype == "f32"
                else s * host[2])
        np.testing.assert_array_equal(to_host(got), want, err_msg=f"s = {s}")


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_fused_contracted_sums(torch, dtype):
    """sums with elementwise products become fused multiply-adds in a new
    order; every mix of signs, scalars and one general subtree must still
    match the literal oracle within the dtype's tolerance"""
    m, n = 190, 77
    host = inputs(321, [(m, n)] * 5, dtype)
    g = E.Graph()
    A, B, C, D, F = (g.input(k, m, n, dtype) for k in range(5))
    exprs = [A % B + 3 * C - D / 2, C - A % B, -(A % B) - D % F + 0.125 * C,
             A % B + (C + D) % F - 2 * D, D / 4 - A % B + C % C, (A + B) / (C % C + 2) - A % D,
             -(D % F) - (A % B)]
    for k, e in enumerate(exprs):
        nodes, outs = g.build(e, E.accu(e))
        got = run(nodes, outs, host, dtype)
        check(got, oracle.evaluate(nodes, outs, host), TOL[dtype], f"expression {k}")


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("mkn", [(1, 1, 1), (37, 53, 29), (100, 100, 100), (257, 130, 64), (64, 513, 300)])
def test_diagmat_of_product(torch, dtype, mkn):
    """diagmat(op(A)*op(B)) from the diagonal alone (Sec. III (4)), every
    transpose combination and scalar factors, rectangular results included"""
    m, k, n = mkn
    for ta in (0, 1):
        for tb in (0, 1):
            g = E.Graph()
            A = g.input(0, k if ta else m, m if ta else k, dtype)
            B = g.input(1, n if tb else k, k if tb else n, dtype)
            opA = A.t() if ta else A
            opB = B.t() if tb else B
            nodes, outs = g.build(E.diagmat(-0.5 * (opA * opB)))
            plan = ag.Plan(nodes, outs)
            if m > 1 and n > 1:   # a 1 x n or m x 1 product is a vector: diagmat builds from it
                assert [s["kernel"] for s in plan.info["steps"]] == ["diagdot", "diagbuild"]
            host = inputs(600 + m + n + k + 2 * ta + tb, [(k if ta else m, m if ta else k),
                                                         (n if tb else k, k if tb else n)], dtype)
            got = run(nodes, outs, host, dtype)
            check(got, oracle.evaluate(nodes, outs, host), TOL[dtype], f"{mkn} {ta}{tb}")


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("n", [1, 7, 256, 1000, 4099])
def test_vector_diagmat_vector(torch, dtype, n):
    """v'*diagmat(B)*w and v'*diagmat(u)*w as one diagonal reduction pass
    (Sec. III (7)); vectors given as columns or as transposed rows"""
    for diag_of in ("matrix", "vector"):
        for vt in (0, 1):
            g = E.Graph()
            v = g.input(0, 1, n, dtype) if vt else g.input(0, n, 1, dtype)
            X = g.input(1, n, n, dtype) if diag_of == "matrix" else g.input(1, n, 1, dtype)
            w = g.input(2, n, 1, dtype)
            left = v if vt else v.t()
            nodes, outs = g.build(3.0 * (left * E.diagmat(X) * w))
            plan = ag.Plan(nodes, outs)
            assert plan.info["steps"][0]["kernel"] == "ew"
            host = inputs(700 + n + vt, [(1, n) if vt else (n, 1), (n, n) if diag_of == "matrix" else (n, 1),
                                         (n, 1)], dtype)
            got = run(nodes, outs, host, dtype)
            ref = oracle.evaluate(nodes, outs, host)
            # a scalar from n terms: its error is relative to the size of the terms
            terms = np.abs(np.asarray(host[0], dtype=np.float64).reshape(-1)
                           * (np.diag(np.asarray(host[1], dtype=np.float64)) if diag_of == "matrix"
                              else np.asarray(host[1], dtype=np.float64).reshape(-1))
                           * np.asarray(host[2], dtype=np.float64).reshape(-1)).sum() * 3.0
            assert abs(float(to_host(got[0]).reshape(-1)[0]) - float(np.asarray(ref[0]).reshape(-1)[0])) <= \
                TOL[dtype] * max(terms, 1e-300), (diag_of, vt)


def test_golden_fixtures_on_gpu(torch):
    """every hand-computed fixture of the paper's expressions, through the
    CUDA path in FP64, equals its stored value within the fixture's
    tolerance (small integers: exactly)"""
    import glob
    import json
    import os
    for path in sorted(glob.glob(os.path.join(os.path.dirname(__file__), "golden", "*.json"))):
        fx = json.load(open(path))
        if "nodes" not in fx:
            continue
        nodes = [dict(nd) for nd in fx["nodes"]]
        for nd in nodes:
            if nd["op"] == "input":
                nd.setdefault("dtype", "f64")
                nd.setdefault("ld", max(1, nd["rows"]))
        host = [np.array(fx["inputs"][s_], dtype=np.float64) for s_ in fx["slots"]]
        got = run(nodes, fx["outputs"], host, "f64")
        for g_, e_ in zip(got, fx["expected"]):
            e = np.array(e_, dtype=np.float64)
            v = np.asarray(to_host(g_), dtype=np.float64).reshape(e.shape)
            tol = max(fx["tol"], 1e-14) * max(1.0, float(np.max(np.abs(e))))
            assert np.max(np.abs(v - e)) <= tol, (os.path.basename(path), v, e)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_diagmat_of_matrix_expressions(torch, dtype):
    """diagmat of a matrix that is not a bare product: the matrix, then its
    off-diagonal zeroed (square and rectangular)"""
    for (m, n) in [(40, 40), (33, 70), (90, 17)]:
        g = E.Graph()
        A, C, D = g.input(0, m, n, dtype), g.input(1, m, n, dtype), g.input(2, m, n, dtype)
        B = g.input(3, n, n, dtype)
        host = inputs(800 + m + n, [(m, n), (m, n), (m, n), (n, n)], dtype)
        for e in (E.diagmat(A), E.diagmat(A + C % D), E.diagmat(A * B + C), E.diagmat(2.0 * (A * B) - C)):
            nodes, outs = g.build(e)
            got = run(nodes, outs, host, dtype)
            check(got, oracle.evaluate(nodes, outs, host), TOL[dtype], f"{m}x{n}")


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("n", [1, 100, 250, 1000])
def test_column_plus_transposed_row(torch, dtype, n):
    """C = A(:,1) + B(2,:)^T (Sec. III (2)) read in place, one pass"""
    g = E.Graph()
    A, B = g.input(0, n, max(n, 2), dtype), g.input(1, max(n, 3), n, dtype)
    nodes, outs = g.build(A.col(1) + B.row(2).t())
    host = inputs(900 + n, [(n, max(n, 2)), (max(n, 3), n)], dtype)
    ref = oracle.evaluate(nodes, outs, host)
    for flags in (0, ag.PLAN_LITERAL):
        check(run(nodes, outs, host, dtype, flags), ref, TOL[dtype], f"n={n} flags={flags}")


@pytest.mark.parametrize("layout", [dict(), dict(pad=5, offset=3)])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_submatrix_views(torch, dtype, layout):
    """ragged blocks at odd offsets, transposed views, views of views and
    of transposes, reductions over views, views in products; inputs with a
    padded leading dimension and a misaligned start"""
    m, n = 203, 171
    ld = m + layout.get("pad", 0)
    g = E.Graph()
    A, B, C = (g.input(s, m, n, dtype, ld=ld) for s in range(3))
    Q = g.input(3, n, m, dtype, ld=n + layout.get("pad", 0))
    host = inputs(950, [(m, n), (m, n), (m, n), (n, m)], dtype)
    va, vb = A.sub(3, 7, 150, 101), B.sub(50, 70, 150, 101)
    cases = {
        "block": 2.0 * va - vb,
        "fused": va % vb + 3.0 * C.sub(1, 1, 150, 101),
        "transposed": A.sub(5, 9, 60, 140).t() + Q.sub(9, 5, 140, 60),
        "view_of_view": A.sub(10, 10, 120, 120).sub(7, 3, 80, 90) * 0.5,
        "view_of_transpose": A.t().sub(11, 17, 100, 150) - Q.sub(0, 1, 100, 150),
        "column_row": A.col(n - 1).sub(0, 0, n, 1) + C.row(m - 1).t(),
        "product": A.sub(0, 0, 100, 171) * Q.sub(0, 3, 171, 90),
        "product_transposed": va.t() * vb,
    }
    for name, e in cases.items():
        nodes, outs = g.build(e, E.accu(e), E.norm_fro(e))
        ref = oracle.evaluate(nodes, outs, host)
        for flags in (0, ag.PLAN_LITERAL):
            got = run(nodes, outs, host, dtype, flags, **layout)
            check(got, ref, TOL[dtype] * (10 if name.startswith("product") else 1), f"{name} flags={flags}")


def test_empty_and_whole_views(torch):
    """a 0-column view gives an empty result and zero reductions; a view of
    the whole matrix is the matrix"""
    g = E.Graph()
    A = g.input(0, 40, 30)
    host = inputs(990, [(40, 30)], "f64")
    nodes, outs = g.build(A.sub(0, 0, 40, 30) * 3.0, E.accu(A.sub(0, 0, 40, 30)))
    check(run(nodes, outs, host, "f64"), oracle.evaluate(nodes, outs, host), TOL["f64"], "whole")
    g = E.Graph()
    A = g.input(0, 40, 30)
    v = A.sub(5, 30, 10, 0)
    nodes, outs = g.build(v * 2.0, E.accu(v))
    got = run(nodes, outs, host, "f64")
    assert got[0].shape == (10, 0) and to_host(got[1]) == 0.0


@pytest.mark.parametrize("layout", [dict(), dict(pad=5, offset=3)])
def test_views_read_in_place_by_other_kernels(torch, layout):
    """views passed to the product, trace, symmetric-product and solve
    kernels as offsets into their matrices (odd offsets, padded and
    misaligned inputs)"""
    m, n = 203, 171
    ld = m + layout.get("pad", 0)
    g = E.Graph()
    A, B = g.input(0, m, n, "f64", ld=ld), g.input(1, m, n, "f64", ld=ld)
    host = inputs(960, [(m, n), (m, n)], "f64")
    host[0] = host[0] + np.eye(m, n) * 8.0        # the square view below is well conditioned
    va, vb = A.sub(3, 7, 150, 101), B.sub(50, 70, 150, 101)
    cases = {
        "product": va.t() * vb,
        "trace": E.trace(va.t() * vb),
        "syrk": 0.5 * (va * va.t()),
        "view_of_view": A.sub(10, 10, 120, 120).sub(7, 3, 80, 90).t() * B.sub(1, 2, 80, 5),
        "solve": E.solve(A.sub(0, 0, 150, 150), B.sub(3, 1, 150, 4)),
    }
    for name, e in cases.items():
        nodes, outs = g.build(e)
        ref = oracle.evaluate(nodes, outs, host)
        for flags in (0, ag.PLAN_LITERAL):
            got = run(nodes, outs, host, "f64", flags, **layout)
            check(got, ref, TOL["f64"] * (100 if name == "solve" else 10), f"{name} flags={flags}")


def test_concurrent_evaluations_from_threads(torch):
    """plans evaluated from several host threads at once, each on its own
    stream with its own workspace, give the same bits as one at a time
    (the library's host-side caches are shared)"""
    import threading
    import torch as T
    n = 300
    g = E.Graph()
    A, B, C, D = (g.input(s, n, n) for s in range(4))
    exprs = [A % B + 3 * C - D / 2, 2 * A.t() * B + C, A * A.t(), E.trace(A * B), E.accu(A % B)]
    host = inputs(970, [(n, n)] * 4, "f64")
    dev_in = [to_dev(h) for h in host]
    plans = [ag.Plan(*g.build(e)) for e in exprs]
    ref = []
    for p in plans:
        out = p(*dev_in)
        T.cuda.synchronize()
        ref.append([to_host(o) for o in out])
    results, errors = {}, []

    def work(i):
        try:
            s = T.cuda.Stream()
            p = plans[i % len(plans)]
            ws = T.empty(max(256, p.workspace_bytes), dtype=T.uint8, device="cuda")
            outs = p.alloc_outputs(T.device("cuda"))
            for _ in range(5):
                p(*dev_in, outputs=outs, workspace=ws, stream=s.cuda_stream)
            s.synchronize()
            results[i] = [to_host(o) for o in outs]
        except Exception as e:          # reported below
            errors.append(repr(e))

    threads = [threading.Thread(target=work, args=(i,)) for i in range(10)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    for i, got in results.items():
        for x, y in zip(got, ref[i % len(plans)]):
            assert np.array_equal(np.asarray(x), np.asarray(y)), i
