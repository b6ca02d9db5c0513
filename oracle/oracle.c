/*
 * CPU FP64 oracle for the expression evaluator -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the smoke check and the CPU-baseline leg of the benchmark
 * use this file.  The product library never links, loads or calls it, and
 * it shares no code with the CUDA path.
 *
 * It is the literal, eager evaluation that the paper uses as its "naive"
 * reference (Sec. II, the discussion of Z = 0.4*X + 0.6*Y before delayed
 * evaluation is introduced): every operator runs on its own and writes a
 * fresh temporary.  The Python side (oracle/__init__.py) allocates those
 * temporaries and walks the expression in written order; this file holds
 * one plain loop per operator.
 *
 * Conventions: all matrices are FP64, column-major, element (i, j) at
 * p[i + j*ld].  Every sum runs in increasing index order in one FP64
 * accumulator.  Loops over independent output columns may run on several
 * OpenMP threads; that never changes any summation order, so the results
 * are the same for any thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define AT(p, ld, i, j) (p)[(int64_t)(i) + (int64_t)(j) * (int64_t)(ld)]

/* ---- elementwise operators (Sec. II: Z[i] = f(X[i], Y[i]) per element) ---- */

void or_add(int64_t m, int64_t n, const double* a, int64_t lda, const double* b,
            int64_t ldb, double* c, int64_t ldc) {
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < m; ++i) AT(c, ldc, i, j) = AT(a, lda, i, j) + AT(b, ldb, i, j);
}

void or_sub(int64_t m, int64_t n, const double* a, int64_t lda, const double* b,
            int64_t ldb, double* c, int64_t ldc) {
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < m; ++i) AT(c, ldc, i, j) = AT(a, lda, i, j) - AT(b, ldb, i, j);
}

/* Schur (elementwise) product, Armadillo's operator % */
void or_schur(int64_t m, int64_t n, const double* a, int64_t lda, const double* b,
              int64_t ldb, double* c, int64_t ldc) {
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < m; ++i) AT(c, ldc, i, j) = AT(a, lda, i, j) * AT(b, ldb, i, j);
}

/* elementwise division, Armadillo's operator / between matrices */
void or_div(int64_t m, int64_t n, const double* a, int64_t lda, const double* b,
            int64_t ldb, double* c, int64_t ldc) {
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < m; ++i) AT(c, ldc, i, j) = AT(a, lda, i, j) / AT(b, ldb, i, j);
}

/* s * X (the Op<Mat, op_mul> marker of Sec. II) */
void or_scale(int64_t m, int64_t n, double s, const double* a, int64_t lda, double* c,
              int64_t ldc) {
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < m; ++i) AT(c, ldc, i, j) = s * AT(a, lda, i, j);
}

/* X / s */
void or_div_scalar(int64_t m, int64_t n, double s, const double* a, int64_t lda, double* c,
                   int64_t ldc) {
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < m; ++i) AT(c, ldc, i, j) = AT(a, lda, i, j) / s;
}

/* X + s */
void or_add_scalar(int64_t m, int64_t n, double s, const double* a, int64_t lda, double* c,
                   int64_t ldc) {
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < m; ++i) AT(c, ldc, i, j) = AT(a, lda, i, j) + s;
}

/* -X */
void or_neg(int64_t m, int64_t n, const double* a, int64_t lda, double* c, int64_t ldc) {
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < m; ++i) AT(c, ldc, i, j) = -AT(a, lda, i, j);
}

/* ---- transpose as an explicit copy (the naive handling in Sec. III, expressions (2) and (8)) ---- */

/* C (n x m) = A^T for A (m x n) */
void or_trans(int64_t m, int64_t n, const double* a, int64_t lda, double* c, int64_t ldc) {
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < m; ++i) AT(c, ldc, j, i) = AT(a, lda, i, j);
}

/* ---- matrix product: the textbook triple loop ----
 * C (m x n) = A (m x k) * B (k x n), C_ij = sum_{l=0}^{k-1} A_il B_lj with
 * l increasing.  Columns of C are independent. */
void or_matmul(int64_t m, int64_t n, int64_t k, const double* a, int64_t lda, const double* b,
               int64_t ldb, double* c, int64_t ldc) {
  /* Row i of A is copied to a contiguous buffer first (pure data movement)
   * so that the inner loop walks memory in order; the sum is unchanged. */
  double* at = (double*)malloc(sizeof(double) * (size_t)(m * (k > 0 ? k : 1)));
  if (!at) return;
  for (int64_t l = 0; l < k; ++l)
    for (int64_t i = 0; i < m; ++i) at[i * k + l] = AT(a, lda, i, l);
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < m; ++i) {
      double s = 0.0;
      for (int64_t l = 0; l < k; ++l) s += at[i * k + l] * AT(b, ldb, l, j);
      AT(c, ldc, i, j) = s;
    }
  free(at);
}

/* Selected entries of A*B, each by the same increasing-l sum as or_matmul:
 * out[t] = sum_l A[ii[t], l] * B[l, jj[t]].  Used where the full product is
 * too large for the CPU (sampled parity at full size). */
void or_matmul_entries(int64_t k, const double* a, int64_t lda, const double* b, int64_t ldb,
                       const int64_t* ii, const int64_t* jj, int64_t count, double* out) {
#pragma omp parallel for schedule(static)
  for (int64_t t = 0; t < count; ++t) {
    double s = 0.0;
    for (int64_t l = 0; l < k; ++l) s += AT(a, lda, ii[t], l) * AT(b, ldb, l, jj[t]);
    out[t] = s;
  }
}

/* ---- diagmat (Sec. III, expressions (3), (4), (7)): only the main
 * diagonal is kept, every other element is treated as zero ---- */

/* vector v (n elements, stride inc) -> dense n x n diagonal matrix */
void or_diagmat_vec(int64_t n, const double* v, int64_t inc, double* c, int64_t ldc) {
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < n; ++i) AT(c, ldc, i, j) = (i == j) ? v[i * inc] : 0.0;
}

/* matrix X (m x n) -> same shape, off-diagonal elements zeroed */
void or_diagmat_mat(int64_t m, int64_t n, const double* a, int64_t lda, double* c, int64_t ldc) {
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < m; ++i) AT(c, ldc, i, j) = (i == j) ? AT(a, lda, i, j) : 0.0;
}

/* ---- scalar reductions ---- */

/* trace(X) = sum_{i < min(m,n)} X_ii (Sec. III, expression (5)) */
double or_trace(int64_t m, int64_t n, const double* a, int64_t lda) {
  double s = 0.0;
  int64_t d = m < n ? m : n;
  for (int64_t i = 0; i < d; ++i) s += AT(a, lda, i, i);
  return s;
}

/* accu(X) = sum of all elements, column-major order, one FP64 running sum */
double or_accu(int64_t m, int64_t n, const double* a, int64_t lda) {
  double s = 0.0;
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < m; ++i) s += AT(a, lda, i, j);
  return s;
}

/* norm(X, "fro") = sqrt(sum X_ij^2), no overflow scaling */
double or_norm_fro(int64_t m, int64_t n, const double* a, int64_t lda) {
  double s = 0.0;
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < m; ++i) s += AT(a, lda, i, j) * AT(a, lda, i, j);
  return sqrt(s);
}

/* ---- explicit inverse (the naive handling of inv(A)*b: Sec. I, Sec. III expression (9)) ----
 * Gauss-Jordan elimination on the augmented matrix [A | I] with partial
 * (row) pivoting; ties in |pivot| go to the smallest row index.
 * Returns 0 on success, or 1 + the column at which no non-zero pivot
 * remained (A singular); C (n x n) then holds no meaningful values. */
int or_inv(int64_t n, const double* a, int64_t lda, double* c, int64_t ldc) {
  int64_t w = 2 * n;
  double* t = (double*)malloc(sizeof(double) * (size_t)(n * w));
  if (!t) return -1;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < w; ++j)
      t[i * w + j] = (j < n) ? AT(a, lda, i, j) : ((j - n == i) ? 1.0 : 0.0);
  for (int64_t col = 0; col < n; ++col) {
    int64_t p = col;
    double best = fabs(t[col * w + col]);
    for (int64_t r = col + 1; r < n; ++r) {
      double v = fabs(t[r * w + col]);
      if (v > best) { best = v; p = r; }
    }
    if (best == 0.0) { free(t); return (int)(col + 1); }
    if (p != col)
      for (int64_t j = 0; j < w; ++j) {
        double x = t[col * w + j]; t[col * w + j] = t[p * w + j]; t[p * w + j] = x;
      }
    double piv = t[col * w + col];
    for (int64_t j = 0; j < w; ++j) t[col * w + j] /= piv;
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < n; ++r) {
      if (r == col) continue;
      double f = t[r * w + col];
      if (f == 0.0) continue;
      for (int64_t j = 0; j < w; ++j) t[r * w + j] -= f * t[col * w + j];
    }
  }
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < n; ++j) AT(c, ldc, i, j) = t[i * w + n + j];
  free(t);
  return 0;
}

/* ---- elementwise conversion helpers for the checks ---- */

/* Frobenius norm of (X - Y) and of Y, for relative errors, each in one
 * FP64 running sum. */
void or_diff_norms(int64_t m, int64_t n, const double* x, int64_t ldx, const double* y,
                   int64_t ldy, double* out2) {
  double d = 0.0, r = 0.0;
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < m; ++i) {
      double e = AT(x, ldx, i, j) - AT(y, ldy, i, j);
      d += e * e;
      r += AT(y, ldy, i, j) * AT(y, ldy, i, j);
    }
  out2[0] = sqrt(d);
  out2[1] = sqrt(r);
}

int or_num_threads(void) {
#ifdef _OPENMP
  extern int omp_get_max_threads(void);
  return omp_get_max_threads();
#else
  return 1;
#endif
}
