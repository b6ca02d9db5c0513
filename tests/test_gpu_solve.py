"""inv(A)*B as a solve (Sec. I; Sec. III (9)): blocked LU with partial
pivoting and, for the mixed-precision tiers, FP64 iterative refinement.
Checked against the oracle's literal Gauss-Jordan inverse times B, against
the normwise backward error, and for the reported device status."""
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


def solve(torch, A, B, tier="native", flags=0, dtype="f64"):
    n, nrhs = B.shape
    nodes, outs = E.config_solve(n, nrhs, dtype)
    plan = ag.Plan(nodes, outs, tier=tier, flags=flags)
    (X,) = plan(to_dev(A, dtype), to_dev(B, dtype))
    torch.cuda.synchronize()
    return to_host(X), plan.status()


def well_conditioned(seed, n):
    return synth.matrix(seed, 1, n, n, "f64") + n * np.eye(n) * 0.1 + np.eye(n)


@pytest.mark.parametrize("n,nrhs", [(1, 1), (5, 3), (64, 1), (65, 7), (200, 64), (257, 33), (300, 130),
                                    (1000, 5)])
@pytest.mark.parametrize("tier", ["f64", "lu32_ir64", "split_bf16"])
def test_solve_small(torch, n, nrhs, tier):
    A = well_conditioned(n, n)
    B = synth.matrix(n + 1, 2, n, nrhs, "f64")
    X, (st, info) = solve(torch, A, B, tier)
    assert st == "ok", (st, info)
    ref = oracle.solve_literal(A, B)
    tol = {"f64": 1e-12, "lu32_ir64": 1e-12, "split_bf16": 1e-5}[tier]
    assert oracle.rel_err(X, ref) <= tol
    if tier != "split_bf16":
        assert oracle.backward_error(A, X, B) <= 1e-14


def test_solve_needs_pivoting(torch):
    """a permutation-like matrix whose leading entries are zero"""
    n = 97
    P = np.eye(n)[np.random.default_rng(0).permutation(n)]
    A = P + 1e-3 * synth.matrix(3, 1, n, n, "f64")
    B = synth.matrix(3, 2, n, 4, "f64")
    for tier in ("f64", "lu32_ir64"):
        X, (st, _) = solve(torch, A, B, tier)
        assert st == "ok"
        assert oracle.rel_err(X, oracle.solve_literal(A, B)) <= 1e-11


def test_singular_reported(torch):
    n = 40
    A = synth.matrix(4, 1, n, n, "f64")
    A[:, 17] = 0.0
    B = synth.matrix(4, 2, n, 2, "f64")
    X, (st, info) = solve(torch, A, B, "f64")
    assert st == "singular" and info >= 1


@pytest.mark.parametrize("flags", [0, ag.PLAN_LITERAL])
def test_explicit_inverse_and_literal(torch, flags):
    n = 130
    A = well_conditioned(7, n)
    g = E.Graph()
    Ai = g.input(0, n, n)
    Bi = g.input(1, n, 5)
    nodes, outs = g.build(E.inv(Ai), E.inv(Ai) * Bi)
    B = synth.matrix(7, 2, n, 5, "f64")
    plan = ag.Plan(nodes, outs, flags=flags)
    got = plan(to_dev(A), to_dev(B))
    torch.cuda.synchronize()
    check(got, oracle.evaluate(nodes, outs, [A, B]), 1e-11, f"inverse flags={flags}")


def test_solve_f32_inputs(torch):
    n = 300
    A = synth.cast(well_conditioned(9, n), "f32")
    B = synth.matrix(9, 2, n, 8, "f32")
    X, (st, _) = solve(torch, A, B, "native", dtype="f32")
    assert st == "ok"
    assert oracle.rel_err(X, oracle.solve_literal(A, B)) <= TOL["f32"]


_COND = {}


def conditioned(symmetric):
    """The benchmark matrix A = Q1 diag(s) Q2^T (n = 4096, kappa = 1e6) and
    the oracle's literal Gauss-Jordan inverse of it, computed once."""
    if symmetric not in _COND:
        A = synth.conditioned_matrix(20250203 + 3, 4096, 1e6, symmetric=symmetric)
        _COND[symmetric] = (A, oracle.inv(A))
    return _COND[symmetric]


@pytest.mark.parametrize("symmetric", [True, False])
def test_solve_conditioned_benchmark_size(torch, symmetric):
    """A = Q1 diag(s) Q2^T, n = 4096, kappa = 1e6, B 4096 x 64 (the benchmark
    configuration): backward error <= 1e-12, and forward error <= 1e-12 *
    kappa against the oracle's literal inv(A) * B (Gauss-Jordan inverse, then
    the triple-loop product)."""
    n, nrhs = 4096, 64
    A, Ainv = conditioned(symmetric)
    B = synth.matrix(20250203 + 3, 2, n, nrhs, "f64")
    X, (st, info) = solve(torch, A, B, "lu32_ir64")
    assert st == "ok", (st, info)
    assert oracle.backward_error(A, X, B) <= 1e-12
    assert oracle.rel_err(X, oracle.matmul(Ainv, B)) <= 1e-12 * 1e6


def test_refinement_step_cap(torch):
    """ARMA_PLAN_REFINE_STEPS(k) stops the FP64 refinement after k steps: with
    the number of steps the solve needs it converges (info = that number), one
    step fewer reports ARMA_ERR_NOCONVERGE with info = the cap."""
    n, nrhs = 4096, 64
    A, _ = conditioned(False)
    B = synth.matrix(20250203 + 3, 2, n, nrhs, "f64")
    _, (st, need) = solve(torch, A, B, "lu32_ir64")
    assert st == "ok" and 2 <= need <= 10, (st, need)
    X, (st, info) = solve(torch, A, B, "lu32_ir64", flags=ag.PLAN_REFINE_STEPS(need))
    assert (st, info) == ("ok", need)
    assert oracle.backward_error(A, X, B) <= 1e-12
    X1, (st, info) = solve(torch, A, B, "lu32_ir64", flags=ag.PLAN_REFINE_STEPS(need - 1))
    assert (st, info) == ("noconverge", need - 1)
    _, (st, info) = solve(torch, A, B, "lu32_ir64", flags=ag.PLAN_REFINE_STEPS(1))
    assert (st, info) == ("noconverge", 1)


@pytest.mark.parametrize("flags", [0, ag.PLAN_DFMA_RESIDUAL])
def test_residual_sliced_or_dfma(torch, flags):
    """The FP64 refinement residual by the sliced tensor-core product
    (default at this size) or by DFMA: both reach the backward error bound and
    agree with the oracle's literal inverse times B."""
    n, nrhs = 4096, 64
    A, Ainv = conditioned(False)
    B = synth.matrix(20250203 + 3, 2, n, nrhs, "f64")
    X, (st, info) = solve(torch, A, B, "lu32_ir64", flags=flags)
    assert st == "ok", (st, info)
    assert oracle.backward_error(A, X, B) <= 1e-12
    assert oracle.rel_err(X, oracle.matmul(Ainv, B)) <= 1e-12 * 1e6


@pytest.mark.parametrize("n,nrhs", [(4096, 64), (1000, 5), (257, 3), (2100, 17)])
def test_lookahead_equals_one_stream(torch, n, nrhs):
    """The look-ahead factorisation (next panel beside the trailing update,
    two streams) gives the one-stream factorisation's result bit for bit."""
    A = synth.conditioned_matrix(20250203 + 3, n, 1e6, symmetric=False) if n == 4096 else well_conditioned(n + 7, n)
    B = synth.matrix(n + 8, 2, n, nrhs, "f64")
    X1, (st1, i1) = solve(torch, A, B, "lu32_ir64")
    X2, (st2, i2) = solve(torch, A, B, "lu32_ir64", flags=ag.PLAN_NO_LOOKAHEAD)
    assert (st1, i1) == (st2, i2) and st1 == "ok"
    assert np.array_equal(X1, X2)
    assert oracle.backward_error(A, X1, B) <= 1e-14


def test_bf16_tier(torch):
    """The BF16 tier factors in BF16 (one tensor-core product per trailing
    update) and refines in FP64.  At kappa = 1e6, kappa * u_bf16 >> 1: the
    refinement cannot converge and the solve reports ARMA_ERR_NOCONVERGE after
    its 10 steps.  On a well-conditioned matrix it converges to the FP64
    backward error."""
    n, nrhs = 4096, 64
    A, Ainv = conditioned(False)
    B = synth.matrix(20250203 + 3, 2, n, nrhs, "f64")
    X, (st, info) = solve(torch, A, B, "bf16")
    assert (st, info) == ("noconverge", 10)
    err = oracle.rel_err(X, oracle.matmul(Ainv, B))
    print(f"\nbf16 tier, kappa 1e6: forward error {err:.3e}, status {st}")
    A2 = well_conditioned(31, 1000)
    B2 = synth.matrix(32, 2, 1000, 16, "f64")
    X2, (st, info) = solve(torch, A2, B2, "bf16")
    assert st == "ok" and 1 <= info <= 10, (st, info)
    assert oracle.backward_error(A2, X2, B2) <= 1e-14
    assert oracle.rel_err(X2, oracle.solve_literal(A2, B2)) <= 1e-12


def test_bounded_wait_runs_out(torch):
    """Failure detection without a hung GPU: with the wait limit at 0 the
    cooperative substitution gives up at the first flag it finds unset; the
    kernels return, the status reads ARMA_ERR_TIMEOUT, and the next
    evaluation with the default limit, on the same plan and workspace,
    succeeds."""
    n, nrhs = 4096, 64
    A = well_conditioned(41, n)
    B = synth.matrix(42, 2, n, nrhs, "f64")
    nodes, outs = E.config_solve(n, nrhs)
    plan = ag.Plan(nodes, outs, tier="lu32_ir64", flags=ag.PLAN_NO_SOLVE_ANALYSIS)
    dA, dB = to_dev(A), to_dev(B)
    old = ag.set_wait_limit_ns(0)
    try:
        plan(dA, dB)
        torch.cuda.synchronize()
        st, _ = plan.status()
    finally:
        ag.set_wait_limit_ns(old)
    assert st == "timeout"
    (X,) = plan(dA, dB)
    torch.cuda.synchronize()
    assert plan.status()[0] == "ok"
    assert oracle.backward_error(A, to_host(X), B) <= 1e-14


def test_solve_panel_beyond_cluster_memory(torch):
    """n = 5200 in FP64: the first panels hold more rows than one cluster's
    shared memory and take the grid-barrier panel kernel, the later ones the
    cluster kernel; both must give the same partial-pivoting factorisation."""
    n, nrhs = 5200, 3
    A = well_conditioned(11, n)
    B = synth.matrix(12, 2, n, nrhs, "f64")
    X, (st, info) = solve(torch, A, B, "f64")
    assert st == "ok", (st, info)
    assert oracle.backward_error(A, X, B) <= 1e-14
    assert oracle.rel_err(X, np.linalg.solve(A, B)) <= 1e-12


def test_refinement_steps_reported(torch):
    """lu32_ir64 reports the refinement steps it took (info) on success."""
    n = 4096
    A, _ = conditioned(False)
    B = synth.matrix(20250203 + 3, 2, n, 4, "f64")
    X, (st, info) = solve(torch, A, B, "lu32_ir64")
    assert st == "ok" and 1 <= info <= 10, (st, info)
    _, (st64, info64) = solve(torch, A, B, "f64")
    assert st64 == "ok" and info64 == 0


@pytest.mark.parametrize("tier", ["f64", "lu32_ir64"])
def test_solve_many_right_hand_sides(torch, tier):
    """20000 right-hand sides: more (block row, 16-column slice) CTAs than the
    GPU holds at once, so the substitution takes its per-block launches."""
    n, nrhs = 256, 20000
    A = well_conditioned(13, n)
    B = synth.matrix(14, 2, n, nrhs, "f64")
    X, (st, info) = solve(torch, A, B, tier)
    assert st == "ok", (st, info)
    assert oracle.rel_err(X, oracle.solve_literal(A, B)) <= 1e-12
    assert oracle.backward_error(A, X, B) <= 1e-14
