"""Host-side tests of the C-ABI library (no GPU): it loads, exports every
symbol the header declares, validates descriptors (the paper's conformance
checks, Sec. II), orders matrix chains exactly like exhaustive search, and
plans the paper's rewrites onto the expected kernels."""
import os
import random
import re

import pytest

import paper_2502_03000_gb300 as ag
from paper_2502_03000_gb300 import expr as E

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2502_03000_gb300 import build
    build.build()
    ag.lib.cache_clear()


def test_exports_every_declared_symbol():
    hdr = open(os.path.join(ROOT, "include", "arma_gpu.h")).read()
    declared = set(re.findall(r"\b(arma_gpu_\w+)\s*\(", hdr))
    assert declared, "no declarations found"
    L = ag.lib()
    for name in sorted(declared):
        assert hasattr(L, name), name
    assert set(ag.EXPORTS) <= declared


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """No fallback: without the compiled library, loading it and planning
    through it raise instead of computing anything elsewhere."""
    monkeypatch.setattr(ag, "LIB_PATH", str(tmp_path / "libarma_gpu.so"))
    ag.lib.cache_clear()
    try:
        with pytest.raises(ImportError):
            ag.lib()
        nodes, outs = E.config_fused(8, "f64")
        with pytest.raises(ImportError):
            ag.Plan(nodes, outs)
    finally:
        monkeypatch.undo()
        ag.lib.cache_clear()
    assert ag.lib() is not None


def test_status_strings():
    L = ag.lib()
    for code in range(11):
        assert L.arma_gpu_status_string(code)


def _plan_err(nodes, outputs, **kw):
    with pytest.raises(ag.ArmaError) as ei:
        ag.Plan(nodes, outputs, **kw)
    return ei.value.status


def test_conformance_errors():
    g = E.Graph()
    A = g.input(0, 4, 5); B = g.input(1, 5, 4)
    assert _plan_err(*g.build(A + B)) == "shape"
    g = E.Graph()
    A = g.input(0, 4, 5); B = g.input(1, 4, 5)
    assert _plan_err(*g.build(A * B)) == "shape"
    g = E.Graph()
    A = g.input(0, 4, 4, "f64"); B = g.input(1, 4, 4, "f32")
    assert _plan_err(*g.build(A % B)) == "dtype"
    g = E.Graph()
    A = g.input(0, 3, 4)
    assert _plan_err(*g.build(E.inv(A))) == "shape"
    # operand indices must point backwards
    assert _plan_err([{"op": "add", "a": 0, "b": 1}], [0]) == "invalid"
    assert _plan_err([{"op": "input", "slot": 0, "rows": 4, "cols": 4, "ld": 2}], [0]) == "shape"
    # a scalar cannot feed another operation
    g = E.Graph()
    A = g.input(0, 3, 3)
    t = E.trace(A)
    nodes, _ = g.build(t)
    nodes.append({"op": "neg", "a": len(nodes) - 1})
    assert _plan_err(nodes, [len(nodes) - 1]) == "unsupported"


def test_workspace_and_outputs():
    nodes, outs = E.config_fused(64, "f32")
    p = ag.Plan(nodes, outs)
    assert p.workspace_bytes >= 4096 and p.workspace_bytes % 256 == 0
    assert p.out_info[0][:3] == (64, 64, ag.F32)
    assert p.out_info[1][3] and p.out_info[2][3]


# ---------------------------------------------------------------- chains

def _splits_to_tree(splits, n):
    return ag.tree_from_splits(splits, 0, n - 1)


@pytest.mark.parametrize("seed", range(40))
def test_chain_dp_equals_exhaustive(orc, seed):
    rnd = random.Random(seed)
    n = rnd.randint(1, 9)
    dims = [rnd.choice([1, 2, 3, 5, 8, 13, 64, 100, 512, 4096]) for _ in range(n + 1)]
    splits, cost = ag.chain_order(dims, 0)
    if n == 1:
        assert cost == 0
        return
    best_cost, best_tree = orc.chain_exhaustive(dims)
    assert cost == best_cost
    assert _splits_to_tree(splits, n) == best_tree


@pytest.mark.parametrize("seed", range(20))
def test_chain_greedy_and_left_match_oracle(orc, seed):
    rnd = random.Random(100 + seed)
    n = rnd.randint(2, 8)
    dims = [rnd.randint(1, 300) for _ in range(n + 1)]
    s1, c1 = ag.chain_order(dims, 1)
    t1 = orc.chain_paper_greedy(dims)
    assert _splits_to_tree(s1, n) == t1 and c1 == orc.tree_cost(t1, dims)
    s2, c2 = ag.chain_order(dims, 2)
    t2 = orc.chain_left_to_right(n)
    assert _splits_to_tree(s2, n) == t2 and c2 == orc.tree_cost(t2, dims)


def test_chain_benchmark_dims():
    splits, cost = ag.chain_order([4096, 8192, 512, 4096, 1], 0)
    assert cost == 39845888 and _splits_to_tree(splits, 4) == (0, 0, (1, 1, (2, 2, 3)))
    _, left = ag.chain_order([4096, 8192, 512, 4096, 1], 2)
    assert left == 25786580992


# ---------------------------------------------------------------- rewrites

def kernels(p):
    return [s["kernel"] for s in p.info["steps"]]


def test_rewrites_config_plain():
    ex = E.config_plain(256)
    k = {name: kernels(ag.Plan(*ex[name])) for name in ex}
    assert k["ew"] == ["ew"]                       # one fused pass, no temporaries
    assert k["transAB"] == ["gemm"]                # transpose folded into the product
    assert k["2AB+C"] == ["gemm"]                  # alpha and beta*C in the epilogue
    assert k["traceAB"] == ["diagdot"]             # diagonal-only product
    assert k["diagvB"] == ["ew"]                   # row scaling, no dense diagonal
    assert k["accuAoB"] == ["ew"]                  # product and sum in one pass, no store
    lit = {name: kernels(ag.Plan(*ex[name], flags=ag.PLAN_LITERAL)) for name in ex}
    assert lit["ew"] == ["ew"] * 5
    assert lit["transAB"] == ["transpose", "gemm"]
    assert lit["2AB+C"] == ["ew", "gemm", "ew"]
    assert lit["traceAB"] == ["gemm", "ew"]
    assert lit["diagvB"] == ["diagbuild", "gemm"]
    assert lit["accuAoB"] == ["ew", "ew"]


def test_reductions_look_through_transposes():
    """trace(X^T) = trace(X), and accu and the Frobenius norm sum every
    element: a transpose that only the reduction uses is not materialised,
    and the plan is step for step the plan of the reduction of X (the fused
    diagonal or reducing pass, the diagonal-only product, or a reduction of
    a materialised matrix)."""
    import re

    def N(op, **k):
        d = {"op": op}
        d.update(k)
        return d

    def steps(nodes, outs, **kw):
        p = ag.Plan(nodes, outs, **kw)
        return ([(s["kernel"], s["flops"], s["bytes"], re.sub(r"node \d+", "node", s["note"]))
                 for s in p.info["steps"]], p.info["workspace"])

    A = N("input", slot=0, rows=97, cols=97, dtype="f32", ld=97)
    R = N("input", slot=0, rows=40, cols=70, dtype="f64", ld=41)
    S = N("input", slot=1, rows=40, cols=70, dtype="f64", ld=40)
    B = N("input", slot=1, rows=97, cols=60, dtype="f32", ld=97)
    C = N("input", slot=2, rows=60, cols=97, dtype="f32", ld=60)
    cases = [
        ([A, N("scale", a=0, s=0.91), N("trans", a=1), N("trace", a=2)],
         [A, N("scale", a=0, s=0.91), N("trace", a=1)]),
        ([R, S, N("add", a=0, b=1), N("trans", a=2), N("trace", a=3)],          # non-square
         [R, S, N("add", a=0, b=1), N("trace", a=2)]),
        ([A, B, C, N("matmul", a=1, b=2), N("trans", a=3), N("trace", a=4)],
         [A, B, C, N("matmul", a=1, b=2), N("trace", a=3)]),
        ([A, N("trans", a=0), N("trace", a=1)], [A, N("trace", a=0)]),
        ([A, N("scale", a=0, s=2.0), N("trans", a=1), N("trans", a=2), N("trace", a=3)],
         [A, N("scale", a=0, s=2.0), N("trace", a=1)]),
    ]
    for with_t, without in cases:
        got, ref = steps(with_t, [len(with_t) - 1]), steps(without, [len(without) - 1])
        assert got == ref, (got, ref)
        assert "transpose" not in [k for k, *_ in got[0]]
    # accu and the Frobenius norm of a transpose: the plans of accu(X) and norm(X)
    for red in ("accu", "norm_fro"):
        got = steps([A, N("scale", a=0, s=0.91), N("trans", a=1), N(red, a=2)], [3])
        ref = steps([A, N("scale", a=0, s=0.91), N(red, a=1)], [2])
        assert got == ref, (red, got, ref)
        got = steps([R, N("trans", a=0), N(red, a=1)], [2])
        assert got == steps([R, N(red, a=0)], [1]) and "transpose" not in [k for k, *_ in got[0]]
    # a transpose that is also an output is materialised once; the trace reads it
    nodes = [A, N("scale", a=0, s=0.91), N("trans", a=1), N("trace", a=2)]
    k = kernels(ag.Plan(nodes, [2, 3]))
    assert k.count("transpose") == 1
    # the literal plan keeps the written order
    assert "transpose" in kernels(ag.Plan(cases[0][0], [3], flags=ag.PLAN_LITERAL))


def test_rewrites_fused_and_chain_and_solve():
    p = ag.Plan(*E.config_fused(128))
    assert kernels(p) == ["ew"]
    assert "+sum" in p.info["steps"][0]["note"] and "+sumsq" in p.info["steps"][0]["note"]
    assert kernels(ag.Plan(*E.config_fused(128), flags=ag.PLAN_LITERAL)) == ["ew"] * 7
    p = ag.Plan(*E.config_chain((40, 80, 5, 40, 1)))
    notes = [s["note"] for s in p.info["steps"]]
    assert kernels(p) == ["gemm"] * 3 and all(n.startswith("gemv") for n in notes)
    assert p.info["flops"] == 2 * (5 * 40 + 80 * 5 + 40 * 80)
    p = ag.Plan(*E.config_solve(64, 3))
    assert kernels(p) == ["solve"]
    assert kernels(ag.Plan(*E.config_solve(64, 3), flags=ag.PLAN_LITERAL)) == ["solve", "gemm"]


def test_rewrites_next_rows():
    """diagmat(A*B): only the product's diagonal (no GEMM); v'*diagmat(B)*w:
    one diagonal reduction pass (no dense diagonal, no product)"""
    plans = {k: kernels(ag.Plan(*v)) for k, v in E.config_next(64).items()}
    assert plans["diagmatAB"] == ["diagdot", "diagbuild"]
    assert plans["vdiagBw"] == ["ew"]
    assert plans["colrow"] == ["ew"]
    assert plans["AAt"] == ["syrk"]
    lit = {k: kernels(ag.Plan(*v, flags=ag.PLAN_LITERAL)) for k, v in E.config_next(64).items()}
    assert "gemm" in lit["diagmatAB"] and "gemm" in lit["vdiagBw"]


def test_symmetric_products_plan():
    """X*X^T and X^T*X (Sec. III (8)) plan as a symmetric product when the
    same value sits on both sides; a beta*C term, a different operand or
    the no-syrk flag give a general product; two input slots are marked for
    the pointer comparison at evaluation"""
    g = E.Graph()
    A, B = g.input(0, 50, 30), g.input(1, 50, 30)
    X = A + B
    for e in (A * A.t(), A.t() * A, 2.0 * (A * A.t()), X * X.t()):
        nodes, outs = g.build(e)
        assert kernels(ag.Plan(nodes, outs))[-1] == "syrk"
        assert kernels(ag.Plan(nodes, outs, flags=ag.PLAN_NO_SYRK))[-1] == "gemm"
        assert "syrk" not in kernels(ag.Plan(nodes, outs, flags=ag.PLAN_LITERAL))
    nodes, outs = g.build(A * A.t() + g.input(2, 50, 50))
    assert kernels(ag.Plan(nodes, outs)) == ["gemm"]
    nodes, outs = g.build(A * B.t())
    p = ag.Plan(nodes, outs)
    assert kernels(p) == ["gemm"] and "symmetric if both slots" in p.info["steps"][0]["note"]
    nodes, outs = g.build(A * A.t())
    p = ag.Plan(nodes, outs)
    assert p.info["steps"][0]["flops"] == 50 * 51 * 30


def test_solve_plans():
    """solve(A, B) and inv(A)*B plan an analysed solve; the literal plan and
    the no-analysis flag plan a dense LU; shapes and dtypes are checked"""
    g = E.Graph()
    A, B = g.input(0, 40, 40), g.input(1, 40, 3)
    for e in (E.solve(A, B), E.inv(A) * B):
        nodes, outs = g.build(e)
        assert "analysed solve" in ag.Plan(nodes, outs).info["steps"][0]["note"]
        for f in (ag.PLAN_LITERAL, ag.PLAN_NO_SOLVE_ANALYSIS):
            assert "analysed" not in " ".join(s["note"] for s in ag.Plan(nodes, outs, flags=f).info["steps"])
    for bad in (((40, 30), (40, 3)), ((40, 40), (39, 3))):
        g = E.Graph()
        nodes, outs = g.build(E.solve(g.input(0, *bad[0]), g.input(1, *bad[1])))
        with pytest.raises(ag.ArmaError) as ei:
            ag.Plan(nodes, outs)
        assert ei.value.status == "shape"
    g = E.Graph()
    nodes, outs = g.build(E.solve(g.input(0, 8, 8, "f32"), g.input(1, 8, 1, "f64")))
    with pytest.raises(ag.ArmaError) as ei:
        ag.Plan(nodes, outs)
    assert ei.value.status == "dtype"


def test_submatrix_views_in_place():
    """A(:,1) + B(2,:)^T (Sec. III (2)) is one strided pass reading both
    views in place; the literal plan copies both and transposes; views
    outside the matrix are shape errors"""
    g = E.Graph()
    A, B = g.input(0, 50, 50), g.input(1, 50, 50)
    nodes, outs = g.build(A.col(1) + B.row(2).t())
    p = ag.Plan(nodes, outs)
    assert kernels(p) == ["ew"] and "strided" in p.info["steps"][0]["note"]
    assert kernels(ag.Plan(nodes, outs, flags=ag.PLAN_LITERAL)) == ["ew", "ew", "transpose", "ew"]
    g = E.Graph()
    A = g.input(0, 10, 10)
    for bad in ((5, 0, 6, 1), (0, 9, 1, 2), (-1, 0, 1, 1)):
        nodes, outs = g.build(A.sub(*bad) * 2.0)
        with pytest.raises(ag.ArmaError) as ei:
            ag.Plan(nodes, outs)
        assert ei.value.status == "shape"


def test_views_feed_kernels_in_place():
    """a submatrix view (no transpose on the way) is an offset into its
    matrix: products, trace, solve and the symmetric product read it with no
    copy; the literal plan copies every view"""
    g = E.Graph()
    A, B, Q = g.input(0, 203, 171), g.input(1, 203, 171), g.input(3, 171, 203)
    va, vb = A.sub(3, 7, 150, 101), B.sub(50, 70, 150, 101)
    for e, want in ((A.sub(0, 0, 100, 171) * Q.sub(0, 3, 171, 90), ["gemm"]), (va.t() * vb, ["gemm"]),
                    (E.trace(va.t() * vb), ["diagdot"]), (va * va.t(), ["syrk"]),
                    (E.solve(A.sub(0, 0, 150, 150), B.sub(0, 0, 150, 3)), ["solve"])):
        nodes, outs = g.build(e)
        assert kernels(ag.Plan(nodes, outs)) == want
        assert "ew" in kernels(ag.Plan(nodes, outs, flags=ag.PLAN_LITERAL))


def test_symmetric_product_of_views():
    """the same view on both sides is a symmetric product; two different
    views of one matrix (different offsets) are not"""
    g = E.Graph()
    A = g.input(0, 100, 80)
    v, w = A.sub(0, 0, 60, 80), A.sub(1, 0, 60, 80)
    nodes, outs = g.build(v * v.t())
    assert kernels(ag.Plan(nodes, outs)) == ["syrk"]
    nodes, outs = g.build(v * w.t())
    assert kernels(ag.Plan(nodes, outs)) == ["gemm"]


def test_fused_program_contracts_products():
    """A%B + 3*C - D/2: the sum is reordered so that the product becomes one
    fused multiply-add and the power-of-two term an exact exponent load:
    two FMAs per element instead of a multiply and two FMAs."""
    for dt in ("f64", "f32"):
        note = ag.Plan(*E.config_fused(128, dt)).info["steps"][0]["note"]
        prog = [ins.split()[0] for ins in note.split("program:")[1].split(";")]
        assert prog == ["ldp2", "axpy", "fma"], note
    # no product in the sum: the plain left-to-right program
    g = E.Graph()
    A, C, D = (g.input(k, 8, 8) for k in range(3))
    note = ag.Plan(*g.build(C + A - 2 * D)).info["steps"][0]["note"]
    assert [i.split()[0] for i in note.split("program:")[1].split(";")] == ["ld", "add", "axpy"], note


def test_plan_info_is_json():
    p = ag.Plan(*E.config_products(256))
    info = p.info
    assert info["mode"] == "optimised" and info["steps"][0]["flops"] == 2 * 256 ** 3


def test_status_before_any_evaluation_is_an_error():
    g = E.Graph()
    nodes, outs = g.build(E.solve(g.input(0, 8, 8), g.input(1, 8, 1)))
    p = ag.Plan(nodes, outs)
    with pytest.raises(ValueError):
        p.status()
    with pytest.raises(ValueError):
        p.solve_path()


def test_view_planning_edges():
    """a view of a transpose feeding a product is copied once (one strided
    pass); a view that is itself an output gets its own copy; views of views
    compose without copies"""
    g = E.Graph()
    A, Q = g.input(0, 120, 90), g.input(1, 60, 4)
    nodes, outs = g.build(A.t().sub(5, 7, 60, 60) * Q)
    assert kernels(ag.Plan(nodes, outs)) == ["ew", "gemm"]
    nodes, outs = g.build(A.sub(1, 2, 30, 40))
    assert kernels(ag.Plan(nodes, outs)) == ["ew"]
    nodes, outs = g.build(A.sub(10, 10, 100, 60).sub(5, 5, 60, 50).t() * A.sub(0, 0, 60, 3))
    assert kernels(ag.Plan(nodes, outs)) == ["gemm"]


def test_analysed_solve_workspace():
    """the analysed solve reserves the structured solvers' scratch on top of
    the general solver's"""
    g = E.Graph()
    nodes, outs = g.build(E.solve(g.input(0, 500, 500), g.input(1, 500, 8)))
    full = ag.Plan(nodes, outs).workspace_bytes
    plain = ag.Plan(nodes, outs, flags=ag.PLAN_NO_SOLVE_ANALYSIS).workspace_bytes
    assert full > plain > 0


def test_c_program_uses_the_abi(tmp_path):
    """A plain C99 program compiled against include/arma_gpu.h and linked to
    the library plans the fused benchmark expression, reads the decision
    log, meets the conformance check and orders the benchmark chain through
    the C ABI alone (host calls, no GPU)."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler")
    libdir = os.path.dirname(ag.LIB_PATH)
    exe = str(tmp_path / "plan_from_c")
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                        "-I", os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "c", "plan_from_c.c"),
                        "-o", exe, "-L", libdir, "-larma_gpu", "-Wl,-rpath," + libdir],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0 and r.stdout.strip().endswith("OK"), r.stdout + r.stderr


def test_builder_operators_follow_armadillo():
    """The Python expression builder writes Armadillo's operators as nodes:
    '*' between matrices is the product ('@' too), '%' the Schur product,
    scalars scale, shift and divide, and s - X is -X + s.  The literal
    oracle evaluates what was built as numpy does, and every elementwise
    result plans into one fused pass."""
    import numpy as np
    import oracle
    import synth
    g = E.Graph()
    A, B = g.input(0, 6, 5), g.input(1, 6, 5)
    C = g.input(2, 5, 3)
    outs = [1 - A, A + 1, -A, A / 4, 0.5 * A % B, A - B, A * C, A @ C, E.trans(A)]
    nodes, o = g.build(*outs)
    a, b, c = synth.matrix(2, 1, 6, 5), synth.matrix(2, 2, 6, 5), synth.matrix(2, 3, 5, 3)
    got = oracle.evaluate(nodes, o, [a, b, c])
    want = [1 - a, a + 1, -a, a / 4, 0.5 * a * b, a - b, a @ c, a @ c, a.T]
    for x, y in zip(got, want):
        np.testing.assert_allclose(x, y, rtol=0, atol=1e-15)
    for out in outs[:6]:
        nodes, o = g.build(out)
        assert kernels(ag.Plan(nodes, o)) == ["ew"]


def test_plan_log_environment_variable():
    """ARMA_PLAN_LOG=1 makes every arma_gpu_plan call write its decision log
    (or the status it failed with) to stderr; unset, planning is silent."""
    import json
    import subprocess
    import sys
    script = ("import paper_2502_03000_gb300 as ag\n"
              "from paper_2502_03000_gb300 import expr as E\n"
              "ag.Plan(*E.config_fused(64, 'f64'))\n"
              "g = E.Graph(); A = g.input(0, 4, 5); B = g.input(1, 4, 6)\n"
              "try:\n    ag.Plan(*g.build(A + B))\nexcept ag.ArmaError:\n    pass\n")
    for value, lines in (("1", 2), ("0", 0), (None, 0)):
        env = dict(os.environ, PYTHONPATH=ROOT)
        env.pop("ARMA_PLAN_LOG", None)
        if value is not None:
            env["ARMA_PLAN_LOG"] = value
        r = subprocess.run([sys.executable, "-c", script], env=env, cwd=ROOT, capture_output=True, text=True,
                           timeout=120)
        assert r.returncode == 0, r.stderr
        logged = [ln for ln in r.stderr.splitlines() if ln.startswith("arma_gpu_plan: ")]
        assert len(logged) == lines, r.stderr
        if lines:
            assert json.loads(logged[0][len("arma_gpu_plan: "):])["steps"][0]["kernel"] == "ew"
            assert logged[1] == "arma_gpu_plan: failed: non-conforming operand sizes"
