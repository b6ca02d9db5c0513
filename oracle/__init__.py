"""CPU FP64 oracle -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The
product library (``paper_2502_03000_gb300``) never imports it and shares no
code with it; the two sides see the same inputs only through ``synth``.

What it computes
----------------
The literal, eager evaluation of an expression that the paper describes as
the naive baseline (Sec. II, before delayed evaluation; Sec. III, the naive
column of each expression): nodes are evaluated one at a time in written
order, each operator writes a fresh FP64 temporary, a transpose is an
explicit copy, ``diagmat`` builds a dense matrix, products are the textbook
triple loop, and ``inv`` is Gauss-Jordan elimination followed by the
product.  Every rewrite the paper describes (fusion, folded transposes and
scalars, diagonal-only products, chain reordering, solve instead of
inverse) reaches the same mathematical result, so this literal evaluation
is the definition the GPU path is checked against.

The arithmetic is in ``oracle.c`` (one plain loop per operator); this file
only walks the expression, allocates temporaries and calls those loops.
Matrix-chain parenthesisation (Sec. II, the paragraph on chains; Sec. III,
expression (6)) is checked by exhaustive enumeration of every binary tree
(``chain_exhaustive``), written here in plain Python.

Expression format (plain data, shared with the tests): a list of node
dicts in topological order, e.g. ``{"op": "input", "slot": 0, "rows": m,
"cols": n}``, ``{"op": "add", "a": 0, "b": 1}``, ``{"op": "scale", "a": 2,
"s": 2.0}``; the ops are input, add, sub, schur, div, scale, div_scalar,
add_scalar, neg, trans, matmul, diagmat, trace, accu, norm_fro, inv, submat,
solve.

Structured solves (Sec. III (10); the band, triangular and symmetry checks
of the solve trace in Fig. 3) have their own functions at the end: the
analysis of the matrix (``band_widths``, ``is_symmetric``), the choice it
leads to (``solve_path``) and the tailored solvers (``solve_band``: Gaussian
elimination with partial pivoting kept inside the band; ``solve_triangular``:
plain substitution), written in Python loops for the test sizes.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from functools import lru_cache

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

_d = ctypes.c_double
_i64 = ctypes.c_int64
_P = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (OpenMP over independent output columns)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", _LIB + ".tmp", _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


@lru_cache(maxsize=1)
def lib() -> ctypes.CDLL:
    L = ctypes.CDLL(build())
    two = [_i64, _i64, _P, _i64, _P, _i64, _P, _i64]
    for name in ("or_add", "or_sub", "or_schur", "or_div"):
        getattr(L, name).argtypes = two
        getattr(L, name).restype = None
    for name in ("or_scale", "or_div_scalar", "or_add_scalar"):
        getattr(L, name).argtypes = [_i64, _i64, _d, _P, _i64, _P, _i64]
        getattr(L, name).restype = None
    for name in ("or_neg", "or_trans", "or_diagmat_mat"):
        getattr(L, name).argtypes = [_i64, _i64, _P, _i64, _P, _i64]
        getattr(L, name).restype = None
    L.or_matmul.argtypes = [_i64, _i64, _i64, _P, _i64, _P, _i64, _P, _i64]
    L.or_matmul.restype = None
    L.or_matmul_entries.argtypes = [_i64, _P, _i64, _P, _i64, ctypes.POINTER(_i64),
                                    ctypes.POINTER(_i64), _i64, _P]
    L.or_matmul_entries.restype = None
    L.or_diagmat_vec.argtypes = [_i64, _P, _i64, _P, _i64]
    L.or_diagmat_vec.restype = None
    for name in ("or_trace", "or_accu", "or_norm_fro"):
        getattr(L, name).argtypes = [_i64, _i64, _P, _i64]
        getattr(L, name).restype = _d
    L.or_inv.argtypes = [_i64, _P, _i64, _P, _i64]
    L.or_inv.restype = ctypes.c_int
    L.or_diff_norms.argtypes = [_i64, _i64, _P, _i64, _P, _i64, _P]
    L.or_diff_norms.restype = None
    L.or_num_threads.argtypes = []
    L.or_num_threads.restype = ctypes.c_int
    return L


def num_threads() -> int:
    return int(lib().or_num_threads())


# ---------------------------------------------------------------------------
# array plumbing (no arithmetic)
# ---------------------------------------------------------------------------

def f64(x) -> np.ndarray:
    """Exact upcast to an FP64 Fortran-ordered 2-D array."""
    a = np.asarray(x)
    if a.ndim == 1:
        a = a.reshape((-1, 1))
    return np.asfortranarray(a, dtype=np.float64)


def _p(a: np.ndarray):
    return a.ctypes.data_as(_P)


def _ld(a: np.ndarray) -> int:
    return max(1, a.shape[0])


def _new(m: int, n: int) -> np.ndarray:
    return np.zeros((m, n), dtype=np.float64, order="F")


# ---------------------------------------------------------------------------
# one function per operator; each returns a fresh temporary
# ---------------------------------------------------------------------------

def _binary(name, a, b):
    if a.shape != b.shape:
        raise ValueError(f"{name}: non-conforming {a.shape} vs {b.shape}")
    c = _new(*a.shape)
    getattr(lib(), name)(a.shape[0], a.shape[1], _p(a), _ld(a), _p(b), _ld(b), _p(c), _ld(c))
    return c


def add(a, b): return _binary("or_add", f64(a), f64(b))
def sub(a, b): return _binary("or_sub", f64(a), f64(b))
def schur(a, b): return _binary("or_schur", f64(a), f64(b))
def div(a, b): return _binary("or_div", f64(a), f64(b))


def _scalar_op(name, a, s):
    a = f64(a)
    c = _new(*a.shape)
    getattr(lib(), name)(a.shape[0], a.shape[1], float(s), _p(a), _ld(a), _p(c), _ld(c))
    return c


def scale(a, s): return _scalar_op("or_scale", a, s)
def div_scalar(a, s): return _scalar_op("or_div_scalar", a, s)
def add_scalar(a, s): return _scalar_op("or_add_scalar", a, s)


def neg(a):
    a = f64(a)
    c = _new(*a.shape)
    lib().or_neg(a.shape[0], a.shape[1], _p(a), _ld(a), _p(c), _ld(c))
    return c


def trans(a):
    a = f64(a)
    c = _new(a.shape[1], a.shape[0])
    lib().or_trans(a.shape[0], a.shape[1], _p(a), _ld(a), _p(c), _ld(c))
    return c


def matmul(a, b):
    a, b = f64(a), f64(b)
    if a.shape[1] != b.shape[0]:
        raise ValueError(f"matmul: non-conforming {a.shape} * {b.shape}")
    m, k, n = a.shape[0], a.shape[1], b.shape[1]
    c = _new(m, n)
    lib().or_matmul(m, n, k, _p(a), _ld(a), _p(b), _ld(b), _p(c), _ld(c))
    return c


def matmul_entries(a, b, ii, jj) -> np.ndarray:
    """(A*B)[ii[t], jj[t]] for each t, by the same sum as ``matmul``."""
    a, b = f64(a), f64(b)
    ii = np.ascontiguousarray(ii, dtype=np.int64)
    jj = np.ascontiguousarray(jj, dtype=np.int64)
    out = np.zeros(len(ii))
    lib().or_matmul_entries(a.shape[1], _p(a), _ld(a), _p(b), _ld(b),
                            ii.ctypes.data_as(ctypes.POINTER(_i64)),
                            jj.ctypes.data_as(ctypes.POINTER(_i64)), len(ii),
                            out.ctypes.data_as(_P))
    return out


def diagmat(a):
    a = f64(a)
    m, n = a.shape
    if m == 1 or n == 1:
        v = np.ascontiguousarray(a.reshape(-1, order="F"))
        c = _new(v.size, v.size)
        lib().or_diagmat_vec(v.size, v.ctypes.data_as(_P), 1, _p(c), _ld(c))
        return c
    c = _new(m, n)
    lib().or_diagmat_mat(m, n, _p(a), _ld(a), _p(c), _ld(c))
    return c


def trace(a) -> float:
    a = f64(a)
    return float(lib().or_trace(a.shape[0], a.shape[1], _p(a), _ld(a)))


def accu(a) -> float:
    a = f64(a)
    return float(lib().or_accu(a.shape[0], a.shape[1], _p(a), _ld(a)))


def norm_fro(a) -> float:
    a = f64(a)
    return float(lib().or_norm_fro(a.shape[0], a.shape[1], _p(a), _ld(a)))


class SingularMatrix(ArithmeticError):
    pass


def inv(a):
    a = f64(a)
    if a.shape[0] != a.shape[1]:
        raise ValueError("inv: matrix is not square")
    c = _new(*a.shape)
    info = lib().or_inv(a.shape[0], _p(a), _ld(a), _p(c), _ld(c))
    if info != 0:
        raise SingularMatrix(f"inv: no non-zero pivot in column {info - 1}")
    return c


# ---------------------------------------------------------------------------
# literal walker
# ---------------------------------------------------------------------------

_BIN = {"add": add, "sub": sub, "schur": schur, "div": div}
_SCAL = {"scale": scale, "div_scalar": div_scalar, "add_scalar": add_scalar}
_RED = {"trace": trace, "accu": accu, "norm_fro": norm_fro}


def submat(x, r0: int, c0: int, rows: int, cols: int):
    """The block x(r0 : r0+rows-1, c0 : c0+cols-1) as a new FP64 matrix
    (Armadillo's submatrix view, Sec. III (2), materialised literally)."""
    x = f64(x)
    if r0 < 0 or c0 < 0 or r0 + rows > x.shape[0] or c0 + cols > x.shape[1]:
        raise ValueError("submatrix outside the matrix")
    out = np.zeros((rows, cols), order="F")
    for j in range(cols):
        out[:, j] = x[r0:r0 + rows, c0 + j]
    return out


def evaluate(nodes, outputs, inputs):
    """Evaluate ``nodes`` literally and return the values of ``outputs``.

    ``inputs[slot]`` are arrays of any float dtype; they are upcast exactly.
    Matrix results are FP64 Fortran arrays, scalar results Python floats."""
    vals = []
    for nd in nodes:
        op = nd["op"]
        if op == "input":
            x = f64(inputs[nd["slot"]])
            if x.shape != (nd["rows"], nd["cols"]):
                raise ValueError(f"input slot {nd['slot']}: shape {x.shape}")
            vals.append(x)
        elif op in _BIN:
            vals.append(_BIN[op](vals[nd["a"]], vals[nd["b"]]))
        elif op in _SCAL:
            vals.append(_SCAL[op](vals[nd["a"]], nd["s"]))
        elif op == "neg":
            vals.append(neg(vals[nd["a"]]))
        elif op == "trans":
            vals.append(trans(vals[nd["a"]]))
        elif op == "matmul":
            vals.append(matmul(vals[nd["a"]], vals[nd["b"]]))
        elif op == "diagmat":
            vals.append(diagmat(vals[nd["a"]]))
        elif op in _RED:
            vals.append(_RED[op](vals[nd["a"]]))
        elif op == "inv":
            vals.append(inv(vals[nd["a"]]))
        elif op == "submat":
            vals.append(submat(vals[nd["a"]], nd["slot"], nd["ld"], nd["rows"], nd["cols"]))
        elif op == "solve":
            # solve(A, B) means X = A^-1 B (Sec. III (9), (10)); taken literally
            vals.append(matmul(inv(vals[nd["a"]]), vals[nd["b"]]))
        else:
            raise ValueError(f"unknown op {op!r}")
    return [vals[o] for o in outputs]


# ---------------------------------------------------------------------------
# error measures
# ---------------------------------------------------------------------------

def rel_err(x, ref) -> float:
    """Relative Frobenius error ||x - ref||_F / ||ref||_F in FP64; for a
    scalar |x - ref| / |ref|, and the absolute error when |ref| < 1e-300."""
    if np.isscalar(ref) or np.ndim(ref) == 0:
        r = float(ref)
        d = abs(float(x) - r)
        return d if abs(r) < 1e-300 else d / abs(r)
    x, ref = f64(x), f64(ref)
    if x.shape != ref.shape:
        raise ValueError(f"shape {x.shape} vs {ref.shape}")
    out = np.zeros(2)
    lib().or_diff_norms(x.shape[0], x.shape[1], _p(x), _ld(x), _p(ref), _ld(ref),
                        out.ctypes.data_as(_P))
    return float(out[0]) if out[1] < 1e-300 else float(out[0] / out[1])


# ---------------------------------------------------------------------------
# matrix chains (Sec. II, chain paragraph; Sec. III expression (6))
# ---------------------------------------------------------------------------
# A chain M_0 ... M_{n-1} has dims p_0..p_n (M_t is p_t x p_{t+1}).  A tree
# is an int (leaf index) or a tuple (split, left, right) where ``split`` is
# the index of the last factor of the left part.  The cost of a tree is the
# number of scalar multiply-adds, sum over its products of rows*inner*cols.

def _trees(i, j):
    if i == j:
        yield i
        return
    for k in range(i, j):
        for left in _trees(i, k):
            for right in _trees(k + 1, j):
                yield (k, left, right)


def tree_cost(tree, dims, i=None, j=None) -> int:
    def rec(t):
        if isinstance(t, int):
            return t, t, 0
        k, l, r = t
        li, lj, lc = rec(l)
        ri, rj, rc = rec(r)
        return li, rj, lc + rc + dims[li] * dims[k + 1] * dims[rj + 1]
    return rec(tree)[2]


def tree_splits(tree):
    """Preorder sequence of split points (for the tie-break)."""
    if isinstance(tree, int):
        return ()
    k, l, r = tree
    return (k,) + tree_splits(l) + tree_splits(r)


def chain_exhaustive(dims):
    """Enumerate every binary tree (Catalan(n-1) of them).  Returns
    (min cost, tree) where, among trees of equal cost, the one whose
    preorder split sequence is lexicographically smallest wins."""
    n = len(dims) - 1
    best = None
    for t in _trees(0, n - 1):
        key = (tree_cost(t, dims), tree_splits(t))
        if best is None or key < best[0]:
            best = (key, t)
    return best[0][0], best[1]


def chain_left_to_right(n):
    t = 0
    for k in range(1, n):
        t = (k - 1, t, k)
    return t


def chain_paper_greedy(dims):
    """The paper's rule (Sec. II, chain paragraph): among adjacent pairs,
    multiply first the pair whose result has the fewest elements; repeat.
    Ties go to the left-most pair."""
    parts = [(t, t, t) for t in range(len(dims) - 1)]   # (first, last, tree)
    while len(parts) > 1:
        best = None
        for q in range(len(parts) - 1):
            a, b = parts[q], parts[q + 1]
            size = dims[a[0]] * dims[b[1] + 1]
            if best is None or size < best[0]:
                best = (size, q)
        q = best[1]
        a, b = parts[q], parts[q + 1]
        parts[q:q + 2] = [(a[0], b[1], (a[1], a[2], b[2]))]
    return parts[0][2]


def chain_eval(mats, tree):
    """Evaluate a chain of matrices in the order ``tree`` gives."""
    if isinstance(tree, int):
        return f64(mats[tree])
    _, l, r = tree
    return matmul(chain_eval(mats, l), chain_eval(mats, r))


def catalan(n: int) -> int:
    return math.comb(2 * n, n) // (n + 1)


# ---------------------------------------------------------------------------
# solve checks (Sec. I and Sec. III expression (9): inv(A)*b is a solve)
# ---------------------------------------------------------------------------

def solve_literal(a, b):
    """inv(A) * B exactly as written: Gauss-Jordan inverse, then the product."""
    return matmul(inv(a), b)


def backward_error(a, x, b) -> float:
    """Normwise relative backward error ||B - A X||_F / (||A||_F ||X||_F + ||B||_F),
    with the residual formed by the oracle's own FP64 product."""
    r = sub(f64(b), matmul(a, x))
    return norm_fro(r) / (norm_fro(a) * norm_fro(x) + norm_fro(b))


def check_pivots(piv, n) -> bool:
    """LAPACK-style pivots (row i swapped with piv[i], 0-based, applied in
    order) describe a valid permutation: each entry in [i, n)."""
    piv = np.asarray(piv)
    return bool(np.all(piv >= np.arange(len(piv))) and np.all(piv < n))


def permutation_from_pivots(piv, n) -> np.ndarray:
    perm = np.arange(n)
    for i, p in enumerate(np.asarray(piv)):
        perm[[i, p]] = perm[[p, i]]
    return perm


def all_permutations_agree(mats) -> float:
    """Max relative spread between all parenthesisations of a short chain."""
    vals = [chain_eval(mats, t) for t in _trees(0, len(mats) - 1)]
    ref = vals[0]
    return max(rel_err(v, ref) for v in vals)


def all_trees(n):
    """Every binary tree over n factors (for the tests)."""
    return list(_trees(0, n - 1))


# ---------------------------------------------------------------------------
# structured solves (Sec. III (10); Fig. 3: band check, triangular checks,
# symmetry check, then the tailored solver)
# ---------------------------------------------------------------------------

BAND_MAX_KL, BAND_MAX_KU = 31, 32


def band_widths(a):
    """(kl, ku): the largest i - j and the largest j - i over the non-zero
    elements of a (0 when there are none below / above the diagonal)."""
    a = f64(a)
    kl = ku = 0
    rows, cols = np.nonzero(a)
    for i, j in zip(rows.tolist(), cols.tolist()):
        if i > j:
            kl = max(kl, i - j)
        elif j > i:
            ku = max(ku, j - i)
    return kl, ku


def is_symmetric(a) -> bool:
    """a equals its transpose element by element (0.0 and -0.0 are equal)."""
    a = f64(a)
    if a.shape[0] != a.shape[1]:
        return False
    return bool(np.all(a == a.T))


def solve_path(a) -> str:
    """The solver the analysis selects, tried in the order of the solve trace
    of Fig. 3: a diagonal matrix; a band matrix (at most 31 sub- and 32
    superdiagonals, and band storage at most a quarter of the rows); an
    upper or lower triangular matrix; a symmetric matrix with a positive
    diagonal whose Cholesky factorisation succeeds; otherwise the general
    solver."""
    a = f64(a)
    n = a.shape[0]
    kl, ku = band_widths(a)
    if kl == 0 and ku == 0:
        return "diagonal"
    if kl <= BAND_MAX_KL and ku <= BAND_MAX_KU and 4 * (2 * kl + ku + 1) <= n:
        return "band"
    if kl == 0:
        return "upper"
    if ku == 0:
        return "lower"
    if n > 1 and is_symmetric(a) and bool(np.all(np.diag(a) > 0.0)):
        try:
            cholesky(a)
            return "cholesky"
        except NotPositiveDefinite:
            pass
    return "general"


class NotPositiveDefinite(ArithmeticError):
    pass


def cholesky(a):
    """Lower-triangular L with L L^T = A, column by column: l_jj is the square
    root of a_jj minus the squares already in row j, the entries below it are
    the remaining inner products divided by l_jj.  Raises NotPositiveDefinite
    when a pivot is not positive."""
    a = f64(a)
    n = a.shape[0]
    L = np.zeros((n, n), order="F")
    for j in range(n):
        d = a[j, j] - float(np.dot(L[j, :j], L[j, :j]))
        if not d > 0.0:
            raise NotPositiveDefinite(f"cholesky: pivot {d!r} in column {j}")
        L[j, j] = math.sqrt(d)
        for i in range(j + 1, n):
            L[i, j] = (a[i, j] - float(np.dot(L[i, :j], L[j, :j]))) / L[j, j]
    return L


def solve_band(a, b, kl: int, ku: int):
    """X with A X = B for A with kl sub- and ku superdiagonals: Gaussian
    elimination with partial pivoting in which every step touches only the
    rows j .. j + kl and the columns j .. j + kl + ku (the row interchanges
    can widen U by kl superdiagonals), the right-hand sides eliminated
    alongside, then back substitution with the banded U.  Raises
    SingularMatrix on an exactly zero pivot."""
    u = f64(a).copy()
    x = f64(b).copy()
    n = u.shape[0]
    for j in range(n):
        last = min(j + kl, n - 1)
        p = j
        for i in range(j + 1, last + 1):      # the first largest magnitude
            if abs(u[i, j]) > abs(u[p, j]):
                p = i
        if u[p, j] == 0.0:
            raise SingularMatrix(f"solve_band: zero pivot in column {j}")
        ju = min(j + kl + ku, n - 1)
        if p != j:
            u[[j, p], j:ju + 1] = u[[p, j], j:ju + 1]
            x[[j, p], :] = x[[p, j], :]
        for i in range(j + 1, last + 1):
            m = u[i, j] / u[j, j]
            u[i, j] = 0.0
            for c in range(j + 1, ju + 1):
                u[i, c] -= m * u[j, c]
            x[i, :] -= m * x[j, :]
    for j in range(n - 1, -1, -1):
        ju = min(j + kl + ku, n - 1)
        for c in range(j + 1, ju + 1):
            x[j, :] -= u[j, c] * x[c, :]
        x[j, :] /= u[j, j]
    return x


def solve_triangular(a, b, lower: bool):
    """X with A X = B for triangular A by plain substitution (forward for
    lower, backward for upper).  Raises SingularMatrix on a zero diagonal
    element."""
    a = f64(a)
    x = f64(b).copy()
    n = a.shape[0]
    order = range(n) if lower else range(n - 1, -1, -1)
    for j in order:
        if a[j, j] == 0.0:
            raise SingularMatrix(f"solve_triangular: zero diagonal element in row {j}")
        known = range(j) if lower else range(j + 1, n)
        for c in known:
            x[j, :] -= a[j, c] * x[c, :]
        x[j, :] /= a[j, j]
    return x
