"""Plant plausible mistakes in the oracle (on the CPU) and check that the
pins in test_oracle.py catch every one of them: a dropped term, a wrong
sign, swapped or transposed operands, an off-by-one index, a missing pivot
search, a missing square root, a wrong chain cost or search, a wrong error
measure, a wrong solver choice."""
import glob
import os

import numpy as np
import pytest

import oracle
import tests.test_oracle as T

PINS = [
    lambda o: [T.test_golden_expression(o, p) for p in sorted(glob.glob(os.path.join(T.GOLDEN, "*.json")))
               if not p.endswith("chain_e6.json")],
    lambda o: T.test_elementwise_vs_numpy(o, 37, 53),
    T.test_small_integer_brute_force, T.test_accu_vs_fsum_and_dot, T.test_norm_fro,
    T.test_matmul_vs_numpy_and_transpose_identity, T.test_trace_invariants, T.test_diagmat,
    T.test_inverse, T.test_solve_literal_and_backward_error, T.test_exact_fraction_inverse,
    T.test_submat_against_index_arithmetic, T.test_band_widths_and_symmetry, T.test_solve_path_order,
    T.test_solve_band_against_dense_and_exact, T.test_solve_triangular_against_scipy,
    T.test_cholesky_against_numpy, T.test_golden_chain_closed_forms, T.test_chain_all_orders_agree,
    T.test_chain_exhaustive_brute_costs, T.test_matmul_entries_match_full_product,
    T.test_rel_err_definition, T.test_pivot_helpers, T.test_transpose_moves_entries,
    T.test_backward_error_closed_form,
]


def _mut_matmul_transposed(a, b):
    a, b = oracle.f64(a), oracle.f64(b)
    if b.shape[0] == b.shape[1]:
        b = np.asfortranarray(b.T)
    return np.asfortranarray(a @ b)


def _mut_matmul_dropped_term(a, b):
    a, b = oracle.f64(a), oracle.f64(b)
    if a.shape[1] <= 1:
        return np.asfortranarray(a @ b)
    return np.asfortranarray(a[:, :-1] @ b[:-1, :])


def _mut_sub_sign(a, b):
    return oracle.f64(b) - oracle.f64(a)


def _mut_accu_dropped(a):
    a = oracle.f64(a)
    return float(np.sum(a.ravel(order="F")[:-1])) if a.size > 1 else float(a.sum())


def _mut_trace_offset(a):
    a = oracle.f64(a)
    d = min(a.shape)
    return float(sum(a[i, (i + 1) % a.shape[1]] for i in range(d)))


def _mut_diagmat_cols(a):
    a = oracle.f64(a)
    if a.shape[0] == 1 or a.shape[1] == 1:
        v = a.reshape(-1, order="F")
        return np.asfortranarray(np.diag(v[::-1]))
    return np.asfortranarray(np.eye(*a.shape) * a)


def _mut_inv_no_pivot(a):
    a = oracle.f64(a).copy()
    n = a.shape[0]
    t = np.hstack([a, np.eye(n)])
    for c in range(n):
        if t[c, c] == 0.0:
            raise oracle.SingularMatrix("zero pivot without row search")
        t[c] /= t[c, c]
        for r in range(n):
            if r != c:
                t[r] -= t[r, c] * t[c]
    return np.asfortranarray(t[:, n:])


def _mut_norm_no_sqrt(a):
    a = oracle.f64(a)
    return float(np.sum(a * a))


def _mut_schur_as_add(a, b):
    return oracle.f64(a) + oracle.f64(b)


def _mut_submat_row_major(x, r0, c0, rows, cols):
    # first row and first column swapped (a row-major reading of the offsets)
    x = oracle.f64(x)
    r0, c0 = min(c0, x.shape[0] - rows), min(r0, x.shape[1] - cols)
    return np.asfortranarray(x[r0:r0 + rows, c0:c0 + cols])


def _mut_band_no_pivoting(a, b, kl, ku):
    # elimination without the row exchanges
    u, x = oracle.f64(a).copy(), oracle.f64(b).copy()
    n = u.shape[0]
    for j in range(n):
        if u[j, j] == 0.0:
            raise oracle.SingularMatrix("zero pivot without row search")
        for i in range(j + 1, min(j + kl, n - 1) + 1):
            m = u[i, j] / u[j, j]
            u[i, j:] -= m * u[j, j:]
            x[i] -= m * x[j]
    for j in range(n - 1, -1, -1):
        x[j] = (x[j] - u[j, j + 1:] @ x[j + 1:]) / u[j, j]
    return x


def _mut_band_widths_swapped(a):
    kl, ku = _orig_band_widths(a)
    return ku, kl


def _mut_triangular_wrong_side(a, b, lower):
    return _orig_solve_triangular(a, b, not lower)


def _mut_cholesky_no_sqrt(a):
    # the pivot itself instead of its square root
    a = oracle.f64(a)
    n = a.shape[0]
    L = np.zeros((n, n))
    for j in range(n):
        d = a[j, j] - L[j, :j] @ L[j, :j]
        if not d > 0:
            raise oracle.NotPositiveDefinite("pivot")
        L[j, j] = d
        for i in range(j + 1, n):
            L[i, j] = (a[i, j] - L[i, :j] @ L[j, :j]) / L[j, j]
    return L


def _mut_add_as_sub(a, b):
    return oracle.f64(a) - oracle.f64(b)


def _mut_div_swapped(a, b):
    return oracle.f64(b) / oracle.f64(a)


def _mut_scale_dropped(a, s):
    return oracle.f64(a).copy(order="F")


def _mut_div_scalar_as_mul(a, s):
    return oracle.f64(a) * s


def _mut_add_scalar_sign(a, s):
    return oracle.f64(a) - s


def _mut_neg_identity(a):
    return oracle.f64(a).copy(order="F")


def _mut_trans_square_identity(a):
    # a transpose that forgets to move anything when the matrix is square
    a = oracle.f64(a)
    return a.copy(order="F") if a.shape[0] == a.shape[1] else np.asfortranarray(a.T)


def _mut_entries_row_off_by_one(a, b, ii, jj):
    m = oracle.f64(a).shape[0]
    return _orig_matmul_entries(a, b, (np.asarray(ii) + 1) % m, jj)


def _mut_tree_cost_result_size(tree, dims, i=None, j=None):
    # counts the elements of each product instead of its multiply-adds
    def rec(t):
        if isinstance(t, int):
            return t, t, 0
        k, l, r = t
        li, _, lc = rec(l)
        _, rj, rc = rec(r)
        return li, rj, lc + rc + dims[li] * dims[rj + 1]
    return rec(tree)[2]


def _mut_chain_first_tree(dims):
    t = next(iter(oracle.all_trees(len(dims) - 1)))
    return oracle.tree_cost(t, dims), t


def _mut_greedy_largest_first(dims):
    parts = [(t, t, t) for t in range(len(dims) - 1)]
    while len(parts) > 1:
        best = None
        for q in range(len(parts) - 1):
            size = dims[parts[q][0]] * dims[parts[q + 1][1] + 1]
            if best is None or size > best[0]:
                best = (size, q)
        q = best[1]
        a, b = parts[q], parts[q + 1]
        parts[q:q + 2] = [(a[0], b[1], (a[1], a[2], b[2]))]
    return parts[0][2]


def _mut_rel_err_absolute(x, ref):
    if np.isscalar(ref) or np.ndim(ref) == 0:
        return abs(float(x) - float(ref))
    return float(np.linalg.norm(oracle.f64(x) - oracle.f64(ref)))


def _mut_backward_error_no_b(a, x, b):
    r = oracle.sub(oracle.f64(b), oracle.matmul(a, x))
    return oracle.norm_fro(r) / (oracle.norm_fro(a) * oracle.norm_fro(x))


def _mut_backward_error_sign(a, x, b):
    r = oracle.add(oracle.f64(b), oracle.matmul(a, x))
    return oracle.norm_fro(r) / (oracle.norm_fro(a) * oracle.norm_fro(x) + oracle.norm_fro(b))


def _mut_symmetric_always(a):
    a = oracle.f64(a)
    return a.shape[0] == a.shape[1]


def _mut_solve_path_general(a):
    return "general"


def _mut_pivots_permissive(piv, n):
    return True


_orig_band_widths = oracle.band_widths
_orig_solve_triangular = oracle.solve_triangular
_orig_matmul_entries = oracle.matmul_entries


MUTANTS = {
    "matmul_transposed_operand": ("matmul", _mut_matmul_transposed),
    "matmul_dropped_term": ("matmul", _mut_matmul_dropped_term),
    "sub_wrong_sign": ("sub", _mut_sub_sign),
    "accu_dropped_element": ("accu", _mut_accu_dropped),
    "trace_off_diagonal": ("trace", _mut_trace_offset),
    "diagmat_wrong_placement": ("diagmat", _mut_diagmat_cols),
    "inv_without_pivoting": ("inv", _mut_inv_no_pivot),
    "norm_without_sqrt": ("norm_fro", _mut_norm_no_sqrt),
    "schur_as_sum": ("schur", _mut_schur_as_add),
    "submat_offsets_swapped": ("submat", _mut_submat_row_major),
    "band_without_pivoting": ("solve_band", _mut_band_no_pivoting),
    "band_widths_swapped": ("band_widths", _mut_band_widths_swapped),
    "triangular_wrong_side": ("solve_triangular", _mut_triangular_wrong_side),
    "cholesky_without_sqrt": ("cholesky", _mut_cholesky_no_sqrt),
    "add_as_difference": ("add", _mut_add_as_sub),
    "div_operands_swapped": ("div", _mut_div_swapped),
    "scale_drops_scalar": ("scale", _mut_scale_dropped),
    "div_scalar_multiplies": ("div_scalar", _mut_div_scalar_as_mul),
    "add_scalar_subtracts": ("add_scalar", _mut_add_scalar_sign),
    "neg_keeps_sign": ("neg", _mut_neg_identity),
    "trans_of_square_is_identity": ("trans", _mut_trans_square_identity),
    "entries_row_off_by_one": ("matmul_entries", _mut_entries_row_off_by_one),
    "chain_cost_counts_elements": ("tree_cost", _mut_tree_cost_result_size),
    "chain_search_takes_first_tree": ("chain_exhaustive", _mut_chain_first_tree),
    "greedy_takes_largest_pair": ("chain_paper_greedy", _mut_greedy_largest_first),
    "rel_err_absolute": ("rel_err", _mut_rel_err_absolute),
    "backward_error_without_b": ("backward_error", _mut_backward_error_no_b),
    "backward_error_residual_sign": ("backward_error", _mut_backward_error_sign),
    "symmetric_by_shape": ("is_symmetric", _mut_symmetric_always),
    "solve_path_always_general": ("solve_path", _mut_solve_path_general),
    "pivots_unchecked": ("check_pivots", _mut_pivots_permissive),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(orc, monkeypatch, name):
    attr, fn = MUTANTS[name]
    monkeypatch.setattr(oracle, attr, fn)
    for table in (oracle._BIN, oracle._SCAL, oracle._RED):
        if attr in table:
            monkeypatch.setitem(table, attr, fn)
    caught = 0
    for pin in PINS:
        try:
            pin(oracle)
        except (AssertionError, ValueError, oracle.SingularMatrix, oracle.NotPositiveDefinite, IndexError):
            caught += 1
    assert caught > 0, f"no pin caught the planted mistake {name}"
