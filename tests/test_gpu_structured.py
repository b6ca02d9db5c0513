"""Solves dispatched on the structure of the matrix (Sec. III (10); the band,
triangular and symmetry checks of the solve trace in Fig. 3).  The analysis
the GPU records (solver taken, bandwidths, symmetry) must equal the
oracle's, and the solution must match the oracle's tailored solver for that
structure within the stated tolerance (1e-12 FP64, 1e-5 FP32); where the
matrix's condition number makes that unreachable for any backward-stable
solve, within kappa_F(A) times the two solutions' backward errors.  The
backward error itself must be at the working precision."""
import numpy as np
import pytest

import oracle
import paper_2502_03000_gb300 as ag
import synth
from paper_2502_03000_gb300 import expr as E
from tests.gpu_util import need_gpu, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return need_gpu()


def solve_plan(n, k, dtype="f64", flags=0, ld=None, inverse=False):
    g = E.Graph()
    A = g.input(0, n, n, dtype, ld=ld or n)
    B = g.input(1, n, k, dtype)
    nodes, outs = g.build(E.inv(A) * B if inverse else E.solve(A, B))
    return ag.Plan(nodes, outs, flags=flags)


def run(plan, a, b, dtype="f64", **layout):
    import torch as T
    ins = [to_dev(a, dtype, **layout), to_dev(b, dtype)]
    got = plan(*ins)
    T.cuda.synchronize()
    return to_host(got[0])


def expect(a, b):
    """the oracle's solver for the structure its analysis finds"""
    path = oracle.solve_path(a)
    kl, ku = oracle.band_widths(a)
    if path in ("diagonal", "band"):
        return path, oracle.solve_band(a, b, kl, ku)
    if path in ("upper", "lower"):
        return path, oracle.solve_triangular(a, b, path == "lower")
    return path, oracle.matmul(oracle.inv(a), b)      # "cholesky" and "general": the definition


TOL = {"f64": 1e-12, "f32": 1e-5}
# normwise backward error of a backward-stable solve in the data's precision
BWD = {"f64": 1e-14, "f32": 1e-7}
U64 = 2.0 ** -53


def kappa_f(a) -> float:
    """Frobenius-norm condition number, ||A||_F ||inv(A)||_F, with the
    oracle's Gauss-Jordan inverse."""
    a = np.asarray(a, dtype=np.float64)
    return oracle.norm_fro(a) * oracle.norm_fro(oracle.inv(a))


def check_solve(plan, a, b, dtype, what, **layout):
    x = run(plan, a, b, dtype, **layout)
    path, ref = expect(a, b)
    got_path, kl, ku, sym = plan.solve_path()
    assert got_path == path, (what, got_path, path)
    assert (kl, ku) == oracle.band_widths(a), what
    assert sym == oracle.is_symmetric(a), what
    assert plan.status()[0] == "ok", what
    eta = oracle.backward_error(a, x, b)
    assert eta <= BWD[dtype], f"{what}: backward error {eta:.2e}"
    err = oracle.rel_err(x, ref)
    if err > TOL[dtype]:
        # Both solutions are exact for the system with residual r: x - x* =
        # inv(A) r, so ||x - x*||_F <= ||inv(A)||_F ||r||_F, i.e. the forward
        # error is at most kappa_F(A) times the backward error (times
        # ||x||/||x*|| + 1).  The difference of two solutions is bounded by the
        # sum of their bounds; the residuals are formed in FP64 (n u64).
        n = a.shape[0]
        eta_ref = oracle.backward_error(a, ref, b)
        ratio = np.linalg.norm(x) / max(np.linalg.norm(ref), 1e-300) + 1.0
        tol = kappa_f(a) * (eta + eta_ref + 2 * n * U64) * ratio
        assert err <= tol, f"{what}: rel err {err:.2e} > kappa-scaled bound {tol:.1e}"
    return path


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("n", [100, 250, 500, 1000, 7000])
@pytest.mark.parametrize("k", [1, 3, 64])
def test_tridiagonal(torch, dtype, n, k):
    """E10: solve(A, b) with A tridiagonal, at the paper's sizes and beyond
    (n = 7000 with 64 right-hand sides keeps the band in the workspace)"""
    a = synth.band_matrix(2000 + n, 1, n, 1, 1, dtype, diag_shift=3.0)
    b = synth.matrix(2000 + n, 2, n, k, dtype)
    assert check_solve(solve_plan(n, k, dtype), a, b, dtype, f"n={n} k={k}") == "band"


@pytest.mark.parametrize("kl,ku,k,dtype", [(1, 1, 5, "f64"), (2, 0, 5, "f64"), (0, 3, 5, "f64"), (3, 5, 5, "f64"),
                                            (31, 32, 5, "f64"), (7, 2, 5, "f64"), (3, 5, 40, "f64"),
                                            (3, 5, 5, "f32"), (2, 2, 33, "f32")])
def test_band_with_row_exchanges(torch, kl, ku, k, dtype):
    """no diagonal dominance and zeros on the diagonal: partial pivoting
    must exchange rows (elimination without it breaks down); more than 32
    right-hand sides take the lanes' second pass"""
    n = 4 * (2 * kl + ku + 1) + 37
    both = kl > 0 and ku > 0
    a = synth.band_matrix(2100 + kl, 1, n, kl, ku, "f64", zero_diag_every=5 if both else 0)
    if not both:
        a += 4.0 * np.eye(n)          # a triangular band with a zero diagonal element is singular
    a = synth.cast(a, dtype)
    b = synth.matrix(2100 + kl, 2, n, k, dtype)
    assert check_solve(solve_plan(n, k, dtype), a, b, dtype, f"kl={kl} ku={ku} k={k}") == "band"


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("shape", [(64, 1), (130, 7), (1000, 64), (333, 100)])
@pytest.mark.parametrize("side", ["upper", "lower"])
def test_triangular(torch, dtype, shape, side):
    n, k = shape
    m = synth.matrix(2200 + n, 1, n, n, dtype).astype(np.float64) + 4.0 * np.eye(n)
    a = synth.cast(np.triu(m) if side == "upper" else np.tril(m), dtype)
    b = synth.matrix(2200 + n, 2, n, k, dtype)
    assert check_solve(solve_plan(n, k, dtype), a, b, dtype, f"{side} {shape}") == side


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_diagonal(torch, dtype):
    n, k = 513, 9
    a = synth.band_matrix(2300, 1, n, 0, 0, dtype, diag_shift=2.0)
    b = synth.matrix(2300, 2, n, k, dtype)
    assert check_solve(solve_plan(n, k, dtype), a, b, dtype, "diagonal") == "diagonal"


def test_general_and_symmetric(torch):
    """dense matrices keep the general solver; the analysis still reports
    symmetry"""
    n = 300
    m = synth.matrix(2400, 1, n, n, "f64") + 8.0 * np.eye(n)
    b = synth.matrix(2400, 2, n, 4, "f64")
    for a, sym in ((m, False), (m + m.T, True)):
        plan = solve_plan(n, 4)
        check_solve(plan, a, b, "f64", f"sym={sym}")
        assert plan.solve_path()[3] == sym


def test_padded_and_inverse_form(torch):
    """a padded, misaligned matrix; inv(A)*B takes the same analysis"""
    n = 400
    a = synth.band_matrix(2500, 1, n, 2, 1, "f64", diag_shift=2.0)
    b = synth.matrix(2500, 2, n, 3, "f64")
    check_solve(solve_plan(n, 3, ld=n + 3), a, b, "f64", "padded", pad=3, offset=1)
    check_solve(solve_plan(n, 3, inverse=True), a, b, "f64", "inverse form")


def test_literal_and_unanalysed(torch):
    """the literal plan and the no-analysis flag factor densely (record
    'none'); results agree with the structured solver"""
    n = 256
    a = synth.band_matrix(2600, 1, n, 1, 1, "f64", diag_shift=3.0)
    b = synth.matrix(2600, 2, n, 2, "f64")
    ref = oracle.solve_band(a, b, 1, 1)
    for flags in (ag.PLAN_LITERAL, ag.PLAN_NO_SOLVE_ANALYSIS):
        plan = solve_plan(n, 2, flags=flags)
        x = run(plan, a, b)
        assert plan.solve_path()[0] == "none"
        assert oracle.rel_err(x, ref) <= 1e-10


@pytest.mark.parametrize("kind", ["diagonal", "upper", "lower", "band"])
def test_singular_structured(torch, kind):
    """an exactly singular structured matrix reports ARMA_ERR_SINGULAR with
    the first zero pivot (1-based), as the oracle's solver raises"""
    n = 200
    if kind == "band":
        a = synth.band_matrix(2700, 1, n, 1, 1, "f64", diag_shift=3.0)
        a[:, 50] = 0.0                      # a zero column: no pivot in column 50
    else:
        m = synth.matrix(2700, 1, n, n, "f64") + 4.0 * np.eye(n)
        a = np.diag(np.diag(m)) if kind == "diagonal" else np.triu(m) if kind == "upper" else np.tril(m)
        a[77, 77] = 0.0
    b = synth.matrix(2700, 2, n, 2, "f64")
    plan = solve_plan(n, 2)
    run(plan, a, b)
    status, info = plan.status()
    assert plan.solve_path()[0] == kind
    assert status == "singular"
    assert info == (51 if kind == "band" else 78)
    with pytest.raises(oracle.SingularMatrix):
        expect(a, b)


def test_tridiagonal_tiers_and_fallback(torch):
    """FP64 data: FP32 factors refined in FP64 (info = refinement steps), the
    FP64 tier factoring directly, and a matrix whose entries vanish in FP32
    (the refined solve gives up and the direct FP64 band solve runs)"""
    n, k = 1000, 2
    a = synth.band_matrix(2800, 1, n, 1, 1, "f64", diag_shift=3.0)
    b = synth.matrix(2800, 2, n, k, "f64")
    ref = oracle.solve_band(a, b, 1, 1)
    plan = solve_plan(n, k)
    x = run(plan, a, b)
    status, steps = plan.status()
    assert status == "ok" and 1 <= steps <= 4, (status, steps)
    assert oracle.rel_err(x, ref) <= 1e-13
    g = E.Graph()
    A, B = g.input(0, n, n), g.input(1, n, k)
    nodes, outs = g.build(E.solve(A, B))
    p64 = ag.Plan(nodes, outs, tier="f64")
    assert oracle.rel_err(run(p64, a, b), ref) <= 1e-13 and p64.solve_path()[0] == "band"
    tiny = a * 1e-50
    x = run(plan, tiny, b)
    assert plan.status()[0] == "ok" and plan.solve_path()[0] == "band"
    assert oracle.rel_err(x, oracle.solve_band(tiny, b, 1, 1)) <= 1e-13


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("n,k", [(2, 1), (64, 1), (130, 7), (1000, 64), (777, 3)])
def test_cholesky(torch, dtype, n, k):
    """a symmetric positive definite matrix takes the Cholesky path (panels
    of 64, ragged last panel); FP64 data is refined in FP64"""
    m = synth.matrix(2900 + n, 1, n, n, "f64")
    a = synth.cast(m @ m.T / n + np.eye(n), dtype)
    b = synth.matrix(2900 + n, 2, n, k, dtype)
    assert check_solve(solve_plan(n, k, dtype), a, b, dtype, f"n={n} k={k}") == "cholesky"


@pytest.mark.parametrize("tier", ["native", "f64"])
def test_cholesky_ill_conditioned(torch, tier):
    """A = Q diag(s) Q^T with condition number 1e6 (the symmetric variant of
    the solve benchmark's matrix): refined to the general solve's stopping rule
    (native tier), or factored in FP64 (f64 tier)"""
    n, k = 1024, 16
    a = synth.conditioned_matrix(3000, n, 1e6, symmetric=True)
    b = synth.matrix(3000, 2, n, k, "f64")
    g = E.Graph()
    nodes, outs = g.build(E.solve(g.input(0, n, n), g.input(1, n, k)))
    plan = ag.Plan(nodes, outs, tier=tier)
    x = run(plan, a, b)
    assert plan.solve_path()[0] == "cholesky" and plan.status()[0] == "ok"
    assert oracle.backward_error(a, x, b) <= 1e-14
    ref = oracle.matmul(oracle.inv(a), b)
    assert oracle.rel_err(x, ref) <= 1e-16 * 1e6 * 100


def test_symmetric_not_positive_definite(torch):
    """symmetric with a positive diagonal but indefinite: the Cholesky attempt
    fails and the general LU solves it; a negative diagonal element skips the
    attempt"""
    n, k = 300, 2
    m = synth.matrix(3100, 1, n, n, "f64")
    spd = m @ m.T / n + np.eye(n)
    ind = spd.copy()
    ind[10, 20] = ind[20, 10] = 50.0
    neg = spd.copy()
    neg[5, 5] = -2.0
    b = synth.matrix(3100, 2, n, k, "f64")
    for a in (ind, neg):
        plan = solve_plan(n, k)
        assert check_solve(plan, a, b, "f64", "indefinite") == "general"
        assert plan.solve_path()[3] is True


def test_analysed_solve_under_graph_capture(torch):
    """while the stream is captured into a CUDA graph no analysis (and no host
    wait) runs: the graph holds the general solve, and its replays solve the
    system"""
    import torch as T
    n, k = 300, 2
    a = synth.band_matrix(3200, 1, n, 1, 1, "f64", diag_shift=3.0)
    b = synth.matrix(3200, 2, n, k, "f64")
    plan = solve_plan(n, k)
    ins = [to_dev(a), to_dev(b)]
    out = plan.alloc_outputs(ins[0].device)
    ws = plan.workspace(ins[0].device)
    s = T.cuda.Stream()
    s.wait_stream(T.cuda.current_stream())
    g = T.cuda.CUDAGraph()
    with T.cuda.stream(s):
        plan(*ins, outputs=out, workspace=ws, stream=s.cuda_stream)   # warm-up outside capture
        s.synchronize()
        with T.cuda.graph(g, stream=s):
            plan(*ins, outputs=out, workspace=ws, stream=s.cuda_stream)
    out[0].zero_()
    g.replay()
    T.cuda.synchronize()
    assert plan.solve_path(workspace=ws)[0] == "none"
    assert oracle.rel_err(to_host(out[0]), oracle.solve_band(a, b, 1, 1)) <= 1e-12


@pytest.mark.parametrize("side", ["upper", "lower"])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_triangular_many_right_hand_sides(torch, side, dtype):
    """20000 right-hand sides: more (block row, 16-column slice) CTAs than the
    GPU holds at once, so the triangular substitution takes its per-block
    launches (forward only for lower, backward only for upper, non-unit
    diagonal blocks)"""
    n, k = 256, 20000
    m = synth.matrix(3300, 1, n, n, "f64") + 4.0 * np.eye(n)
    a = synth.cast(np.triu(m) if side == "upper" else np.tril(m), dtype)
    b = synth.matrix(3300, 2, n, k, dtype)
    plan = solve_plan(n, k, dtype)
    x = run(plan, a, b, dtype)
    assert plan.solve_path()[0] == side and plan.status()[0] == "ok"
    ref = oracle.solve_triangular(a, b, side == "lower")
    assert oracle.rel_err(x, ref) <= (1e-13 if dtype == "f64" else 1e-5)
