"""Pins for the CPU FP64 oracle: each check compares the oracle with
something other than itself -- hand-computed fixtures from the paper's
expressions, closed forms, algebraic invariants, library routines (numpy,
math.fsum) and exact brute force over small integers."""
import glob
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _tree(t):
    return t if isinstance(t, int) else (t[0], _tree(t[1]), _tree(t[2]))


# ---------------------------------------------------------------- fixtures

@pytest.mark.parametrize("path", sorted(p for p in glob.glob(os.path.join(GOLDEN, "*.json"))
                                        if not p.endswith("chain_e6.json")))
def test_golden_expression(orc, path):
    g = json.load(open(path))
    ins = [np.array(g["inputs"][s], dtype=np.float64) for s in g["slots"]]
    got = orc.evaluate(g["nodes"], g["outputs"], ins)
    for v, e in zip(got, g["expected"]):
        e = np.array(e, dtype=np.float64)
        tol = g["tol"] * max(1.0, float(np.max(np.abs(e))))
        assert np.max(np.abs(np.asarray(v) - e)) <= tol, (path, v, e)


def test_golden_chain_closed_forms(orc):
    g = json.load(open(os.path.join(GOLDEN, "chain_e6.json")))
    for case in g["cases"]:
        dims = case["dims"]
        cost, tree = orc.chain_exhaustive(dims)
        assert cost == case["optimal_cost"]
        assert tree == _tree(case["optimal_tree"])
        assert orc.tree_cost(orc.chain_left_to_right(len(dims) - 1), dims) == case["left_to_right_cost"]
        # the paper's own greedy rule reaches the right-to-left order here
        assert orc.chain_paper_greedy(dims) == _tree(case["optimal_tree"])


# ---------------------------------------------------------------- elementwise

def _rand(seed, stream, m, n):
    return synth.matrix(seed, stream, m, n, "f64")


@pytest.mark.parametrize("m,n", [(1, 1), (37, 53), (128, 3)])
def test_elementwise_vs_numpy(orc, m, n):
    A, B = _rand(1, 1, m, n), _rand(1, 2, m, n)
    B = np.where(np.abs(B) < 1e-3, 0.5, B)
    np.testing.assert_array_equal(orc.add(A, B), A + B)
    np.testing.assert_array_equal(orc.sub(A, B), A - B)
    np.testing.assert_array_equal(orc.schur(A, B), A * B)
    np.testing.assert_array_equal(orc.div(A, B), A / B)
    np.testing.assert_array_equal(orc.scale(A, -2.5), -2.5 * A)
    np.testing.assert_array_equal(orc.div_scalar(A, 3.0), A / 3.0)
    np.testing.assert_array_equal(orc.add_scalar(A, 0.25), A + 0.25)
    np.testing.assert_array_equal(orc.neg(A), -A)
    np.testing.assert_array_equal(orc.trans(A), A.T)


def test_small_integer_brute_force(orc):
    """Every shape 1x1 .. 4x4 with small integers: FP64 is exact here, so the
    oracle must equal exact integer arithmetic bit for bit."""
    for m in range(1, 5):
        for k in range(1, 5):
            for n in range(1, 5):
                A = synth.small_ints(m * 100 + k * 10 + n, 1, m, k)
                B = synth.small_ints(m * 100 + k * 10 + n, 2, k, n)
                C = synth.small_ints(m * 100 + k * 10 + n, 3, m, n)
                Ai = [[int(A[i, l]) for l in range(k)] for i in range(m)]
                Bi = [[int(B[l, j]) for j in range(n)] for l in range(k)]
                exact = [[sum(Ai[i][l] * Bi[l][j] for l in range(k)) for j in range(n)]
                         for i in range(m)]
                assert orc.matmul(A, B).tolist() == [[float(x) for x in r] for r in exact]
                D = synth.small_ints(7 * m + n, 4, m, n)
                ew = [[int(C[i, j]) + 3 * int(D[i, j]) * int(C[i, j]) - 2 * int(D[i, j])
                       for j in range(n)] for i in range(m)]
                # C + 3*(D%C) - 2*D
                got = orc.sub(orc.add(C, orc.scale(orc.schur(D, C), 3.0)), orc.scale(D, 2.0))
                assert got.tolist() == [[float(x) for x in r] for r in ew]
                assert orc.accu(C) == float(sum(sum(int(x) for x in r) for r in C.tolist()))
                assert orc.trace(C) == float(sum(int(C[i, i]) for i in range(min(m, n))))


# ---------------------------------------------------------------- reductions

def test_accu_vs_fsum_and_dot(orc):
    A, B = _rand(2, 1, 300, 257), _rand(2, 2, 300, 257)
    exact = math.fsum(A.ravel(order="F"))
    bound = A.size * 2.0 ** -53 * float(np.sum(np.abs(A)))
    assert abs(orc.accu(A) - exact) <= bound
    # accu(A%B) is the dot product of the vectorised operands
    dot = math.fsum((A * B).ravel())
    assert abs(orc.accu(orc.schur(A, B)) - dot) <= 2 * A.size * 2.0 ** -53 * float(np.sum(np.abs(A * B)))
    # linearity: accu(2A - 3B) = 2 accu(A) - 3 accu(B)
    lhs = orc.accu(orc.sub(orc.scale(A, 2.0), orc.scale(B, 3.0)))
    rhs = 2 * orc.accu(A) - 3 * orc.accu(B)
    assert abs(lhs - rhs) <= 1e-11 * float(np.sum(np.abs(A)) + np.sum(np.abs(B)))


def test_norm_fro(orc):
    A = _rand(3, 1, 129, 65)
    assert orc.norm_fro(A) == pytest.approx(float(np.linalg.norm(A, "fro")), rel=1e-14)
    assert orc.norm_fro(A) ** 2 == pytest.approx(orc.accu(orc.schur(A, A)), rel=1e-14)
    I = np.eye(9)
    assert orc.norm_fro(I) == 3.0


# ---------------------------------------------------------------- products

def test_matmul_vs_numpy_and_transpose_identity(orc):
    A, B = _rand(4, 1, 33, 17), _rand(4, 2, 17, 29)
    C = orc.matmul(A, B)
    np.testing.assert_allclose(C, A @ B, rtol=0, atol=1e-13)
    # (AB)^T = B^T A^T
    np.testing.assert_allclose(orc.trans(C), orc.matmul(orc.trans(B), orc.trans(A)), rtol=0, atol=1e-13)
    # identity and permutation special cases are exact
    np.testing.assert_array_equal(orc.matmul(A, np.eye(17)), A)
    P = np.eye(33)[::-1]
    np.testing.assert_array_equal(orc.matmul(P, A), A[::-1, :])


def test_transpose_moves_entries(orc):
    # element (i, j) of trans(X) is element (j, i) of X, square or not
    for m, n in ((1, 1), (5, 5), (16, 16), (3, 7), (7, 3)):
        X = np.arange(m * n, dtype=np.float64).reshape(m, n, order="F") + 1.0
        T = orc.trans(X)
        assert T.shape == (n, m)
        for i in range(n):
            for j in range(m):
                assert T[i, j] == X[j, i]
    # (S R)^T = R^T S^T for square factors too
    S, R = _rand(4, 3, 12, 12), _rand(4, 4, 12, 12)
    np.testing.assert_allclose(orc.trans(orc.matmul(S, R)), orc.matmul(orc.trans(R), orc.trans(S)),
                               rtol=0, atol=1e-13)
    assert not np.array_equal(orc.trans(S), S)


def test_matmul_entries_match_full_product(orc):
    A, B = _rand(5, 1, 40, 31), _rand(5, 2, 31, 23)
    C = orc.matmul(A, B)
    ii = np.array([0, 39, 7, 21]); jj = np.array([0, 22, 13, 5])
    np.testing.assert_array_equal(orc.matmul_entries(A, B, ii, jj), C[ii, jj])


def test_trace_invariants(orc):
    A, B = _rand(6, 1, 23, 41), _rand(6, 2, 41, 23)
    assert orc.trace(orc.matmul(A, B)) == pytest.approx(orc.trace(orc.matmul(B, A)), rel=1e-13)
    S = _rand(6, 3, 31, 31)
    assert orc.trace(orc.matmul(S, np.eye(31))) == float(sum(S[i, i] for i in range(31)))
    assert orc.trace(S) == pytest.approx(float(np.trace(S)), rel=1e-14)
    R = _rand(6, 4, 5, 9)           # non-square: first min(m, n) diagonal entries
    assert orc.trace(R) == pytest.approx(float(np.trace(R)), rel=1e-14)


def test_diagmat(orc):
    v = _rand(7, 5, 19, 1)
    B = _rand(7, 2, 19, 11)
    D = orc.diagmat(v)
    np.testing.assert_array_equal(D, np.diag(v[:, 0]))
    np.testing.assert_array_equal(orc.matmul(D, B), v * B)      # row scaling, exact
    M = _rand(7, 1, 6, 8)
    np.testing.assert_array_equal(orc.diagmat(M), np.eye(6, 8) * M)
    np.testing.assert_array_equal(orc.diagmat(v.T), np.diag(v[:, 0]))


# ---------------------------------------------------------------- chains

def test_chain_all_orders_agree(orc):
    dims = [7, 13, 5, 11, 3, 9]
    mats = [_rand(8, t + 1, dims[t], dims[t + 1]) for t in range(5)]
    assert len(orc.all_trees(5)) == orc.catalan(4) == 14
    assert orc.all_permutations_agree(mats) < 1e-14


def test_chain_exhaustive_brute_costs(orc):
    # by hand: 10x100, 100x5, 5x50 -> (AB)C = 5000 + 2500 = 7500, A(BC) = 25000 + 50000
    cost, tree = orc.chain_exhaustive([10, 100, 5, 50])
    assert (cost, tree) == (7500, (1, (0, 0, 1), 2))
    # ties go to the left-most split: all-square chain, every tree costs the same
    cost, tree = orc.chain_exhaustive([4, 4, 4, 4])
    assert cost == 128 and tree == (0, 0, (1, 1, 2))


# ---------------------------------------------------------------- inverse / solve

def test_inverse(orc):
    A = _rand(9, 1, 40, 40) + 40 * np.eye(40)
    X = orc.inv(A)
    np.testing.assert_allclose(orc.matmul(A, X), np.eye(40), rtol=0, atol=1e-13)
    np.testing.assert_allclose(X, np.linalg.inv(A), rtol=0, atol=1e-14)
    # a permutation matrix needs pivoting and its inverse is its transpose, exactly
    P = np.eye(6)[[3, 0, 5, 1, 4, 2]]
    np.testing.assert_array_equal(orc.inv(P), P.T)
    with pytest.raises(orc.SingularMatrix):
        orc.inv(np.array([[1.0, 2.0], [2.0, 4.0]]))


def test_solve_literal_and_backward_error(orc):
    A = synth.conditioned_matrix(11, 64, cond=1e6, symmetric=False)
    s = np.linalg.svd(A, compute_uv=False)
    assert s[0] / s[-1] == pytest.approx(1e6, rel=1e-6)
    B = _rand(11, 7, 64, 5)
    X = orc.solve_literal(A, B)
    assert orc.backward_error(A, X, B) < 1e-12
    Xn = np.linalg.solve(A, B)
    assert orc.rel_err(X, Xn) < 1e6 * 1e-13


def test_backward_error_closed_form(orc):
    # A = 2I, X = I, B = I (n = 4): B - AX = -I, so the error is
    # ||I||_F / (||2I||_F ||I||_F + ||I||_F) = 2 / (4 * 2 + 2) = 0.2
    I4 = np.eye(4)
    assert orc.backward_error(2 * I4, I4, I4) == 0.2
    # an exact solution has no backward error; X = 0 has the largest, 1
    A = np.array([[2.0, 1.0], [1.0, 3.0]])
    B = np.array([[3.0], [4.0]])
    assert orc.backward_error(A, np.array([[1.0], [1.0]]), B) == 0.0
    assert orc.backward_error(A, np.zeros((2, 1)), B) == 1.0


def test_rel_err_definition(orc):
    assert orc.rel_err(3.0, 4.0) == 0.25
    assert orc.rel_err(1e-310, 0.0) == 1e-310
    assert orc.rel_err(np.array([[3.0, 4.0]]), np.array([[0.0, 0.0]])) == 5.0
    assert orc.rel_err(np.array([[1.0, 1.0]]), np.array([[1.0, 0.0]])) == 1.0


def test_pivot_helpers(orc):
    assert orc.check_pivots([2, 1, 2], 3)
    assert not orc.check_pivots([0, 0, 2], 3)
    assert list(orc.permutation_from_pivots([2, 2, 2], 3)) == [2, 0, 1]


def test_exact_fraction_inverse(orc):
    """Gauss-Jordan on a 3x3 integer matrix against exact rational
    arithmetic (adjugate formula)."""
    M = [[2, -1, 0], [-1, 2, -1], [0, -1, 2]]
    A = np.array(M, dtype=np.float64)
    def det(m):
        return (m[0][0] * (m[1][1] * m[2][2] - m[1][2] * m[2][1])
                - m[0][1] * (m[1][0] * m[2][2] - m[1][2] * m[2][0])
                + m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]))
    d = det(M)
    def minor(i, j):
        r = [[M[a][b] for b in range(3) if b != j] for a in range(3) if a != i]
        return r[0][0] * r[1][1] - r[0][1] * r[1][0]
    exact = [[Fraction((-1) ** (i + j) * minor(j, i), d) for j in range(3)] for i in range(3)]
    np.testing.assert_allclose(orc.inv(A), np.array(exact, dtype=np.float64), rtol=0, atol=1e-15)


def test_submat_against_index_arithmetic(orc):
    """the oracle's submatrix equals element-by-element index arithmetic on
    the column-major storage (a different route from its own slicing)"""
    rng = np.random.default_rng(12)
    for (m, n, r0, c0, rows, cols) in [(5, 7, 1, 2, 3, 4), (4, 4, 0, 0, 4, 4), (6, 3, 5, 2, 1, 1), (3, 8, 0, 7, 3, 1)]:
        x = np.asfortranarray(rng.standard_normal((m, n)))
        flat = x.ravel(order="F")
        got = orc.submat(x, r0, c0, rows, cols)
        for j in range(cols):
            for i in range(rows):
                assert got[i, j] == flat[(r0 + i) + (c0 + j) * m]
    with pytest.raises(ValueError):
        orc.submat(np.zeros((3, 3)), 2, 0, 2, 1)


# ------------------------------------------------- structured solves (Sec. III (10))

def _band(rng, n, kl, ku):
    """a matrix whose non-zero diagonals are exactly -kl .. ku (no zeros on them)"""
    a = np.zeros((n, n))
    for d in range(-kl, ku + 1):
        v = rng.uniform(0.5, 1.5, n - abs(d)) * rng.choice([-1.0, 1.0], n - abs(d))
        a += np.diag(v, d)
    return a


def test_band_widths_and_symmetry(orc):
    rng = np.random.default_rng(30)
    for (n, kl, ku) in [(10, 1, 1), (40, 3, 7), (17, 0, 4), (17, 5, 0), (9, 0, 0), (6, 5, 5)]:
        assert orc.band_widths(_band(rng, n, kl, ku)) == (kl, ku)
    assert orc.band_widths(np.zeros((5, 5))) == (0, 0)
    a = np.zeros((8, 8))
    a[7, 0] = -0.0          # a negative zero is a zero
    a[0, 6] = 1e-300
    assert orc.band_widths(a) == (0, 6)
    s = rng.standard_normal((9, 9))
    s = s + s.T
    assert orc.is_symmetric(s)
    s[2, 5] += 1e-15
    assert not orc.is_symmetric(s)
    z = np.eye(4)
    z[1, 2], z[2, 1] = 0.0, -0.0
    assert orc.is_symmetric(z)


def test_solve_path_order(orc):
    """the order of the checks in the solve trace of Fig. 3: band first, then
    triangular, then general; a diagonal matrix is the narrowest band"""
    rng = np.random.default_rng(31)
    assert orc.solve_path(_band(rng, 100, 0, 0)) == "diagonal"
    assert orc.solve_path(_band(rng, 100, 1, 1)) == "band"
    assert orc.solve_path(_band(rng, 100, 0, 1)) == "band"        # bidiagonal: band before triangular
    assert orc.solve_path(_band(rng, 400, 31, 32)) == "band"
    assert orc.solve_path(_band(rng, 300, 31, 32)) == "general"     # 4 (2 kl + ku + 1) > n
    assert orc.solve_path(_band(rng, 200, 32, 0)) == "lower"        # 32 subdiagonals: not a band
    assert orc.solve_path(np.triu(rng.standard_normal((50, 50)))) == "upper"
    assert orc.solve_path(np.tril(rng.standard_normal((50, 50)))) == "lower"
    assert orc.solve_path(_band(rng, 12, 1, 1)) == "general"      # band storage would not pay
    assert orc.solve_path(rng.standard_normal((30, 30))) == "general"
    assert orc.solve_path(_band(rng, 300, 40, 2)) == "general"     # too many subdiagonals


def test_solve_band_against_dense_and_exact(orc):
    rng = np.random.default_rng(32)
    for (n, kl, ku, k) in [(50, 1, 1, 1), (64, 3, 5, 4), (40, 0, 2, 2), (33, 4, 0, 3)]:
        a = _band(rng, n, kl, ku)
        b = rng.standard_normal((n, k))
        x = orc.solve_band(a, b, kl, ku)
        ref = np.linalg.solve(a, b)
        assert np.max(np.abs(x - ref)) <= 1e-10 * max(1.0, np.max(np.abs(ref))) * np.linalg.cond(a)
    # a zero leading diagonal element: the pivot search must exchange rows
    a = np.array([[0, 2, 0, 0], [1, 1, 3, 0], [0, 4, 1, 1], [0, 0, 2, 5]], dtype=float)
    xs = np.array([[1.0], [-2.0], [3.0], [0.5]])
    x = orc.solve_band(a, a @ xs, 1, 1)
    assert np.max(np.abs(x - xs)) < 1e-14
    with pytest.raises(orc.SingularMatrix):
        orc.solve_band(np.array([[1.0, 2.0, 0.0], [2.0, 4.0, 0.0], [0.0, 1.0, 1.0]]), np.ones((3, 1)), 1, 1)


def test_solve_triangular_against_scipy(orc):
    sla = pytest.importorskip("scipy.linalg")
    rng = np.random.default_rng(33)
    for lower in (True, False):
        a = rng.standard_normal((40, 40)) + 8 * np.eye(40)
        a = np.tril(a) if lower else np.triu(a)
        b = rng.standard_normal((40, 3))
        x = orc.solve_triangular(a, b, lower)
        assert np.max(np.abs(x - sla.solve_triangular(a, b, lower=lower))) < 1e-13
    a = np.triu(np.ones((4, 4)))
    a[2, 2] = 0.0
    with pytest.raises(orc.SingularMatrix):
        orc.solve_triangular(a, np.ones((4, 1)), False)


def test_cholesky_against_numpy(orc):
    rng = np.random.default_rng(34)
    for n in (1, 5, 40):
        m = rng.standard_normal((n, n))
        a = m @ m.T + n * np.eye(n)
        L = orc.cholesky(a)
        assert np.allclose(L, np.tril(L)) and np.all(np.diag(L) > 0)
        assert np.max(np.abs(L - np.linalg.cholesky(a))) < 1e-12 * max(1.0, np.max(np.abs(L)))
    # symmetric with a positive diagonal, but indefinite
    with pytest.raises(orc.NotPositiveDefinite):
        orc.cholesky(np.array([[1.0, 2.0], [2.0, 1.0]]))
    spd = rng.standard_normal((30, 30))
    spd = spd @ spd.T + 30 * np.eye(30)
    assert orc.solve_path(spd) == "cholesky"
    ind = spd.copy()
    ind[0, 1] = ind[1, 0] = 1e3
    assert orc.solve_path(ind) == "general"
    neg = spd.copy()
    neg[3, 3] = -1.0
    assert orc.solve_path(neg) == "general"


def test_threads_do_not_change_results(tmp_path):
    """The oracle's OpenMP loops run over independent output columns and
    leave every summation order as written, so one thread and several give
    bit-identical results."""
    import subprocess
    import sys
    script = (
        "import sys, numpy as np, oracle, synth\n"
        "from paper_2502_03000_gb300 import expr as E\n"
        "nodes, outs = E.config_fused(300, 'f64')\n"
        "ins = [synth.matrix(3, s + 1, 300, 300, 'f64') for s in range(4)]\n"
        "r = oracle.evaluate(nodes, outs, ins)\n"
        "A, B = synth.matrix(4, 1, 120, 90, 'f64'), synth.matrix(4, 2, 90, 70, 'f64')\n"
        "M = synth.matrix(4, 3, 50, 50, 'f64') + 50 * np.eye(50)\n"
        "np.savez(sys.argv[1], out=r[0], accu=r[1], norm=r[2], prod=oracle.matmul(A, B),\n"
        "         inv=oracle.inv(M), t=oracle.trans(A), acc=oracle.accu(A), nf=oracle.norm_fro(A),\n"
        "         threads=oracle.num_threads())\n")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    res = {}
    for t in (1, 4):
        env = dict(os.environ, OMP_NUM_THREADS=str(t), PYTHONPATH=root)
        path = str(tmp_path / f"r{t}.npz")
        r = subprocess.run([sys.executable, "-c", script, path], env=env, cwd=root,
                           capture_output=True, text=True, timeout=300)
        assert r.returncode == 0, r.stderr[-2000:]
        res[t] = np.load(path)
    assert int(res[1]["threads"]) == 1 and int(res[4]["threads"]) == 4
    for k in ("out", "accu", "norm", "prod", "inv", "t", "acc", "nf"):
        np.testing.assert_array_equal(res[1][k], res[4][k], err_msg=k)
