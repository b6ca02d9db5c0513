// Structured solves: the run-time analysis of the system matrix that picks
// a tailored solver (Sec. III (10); the band, triangular and symmetric
// checks of the solve trace in Fig. 3), and the diagonal and band solvers
// it can pick.  The triangular solver is the substitution of the LU path
// applied to the matrix itself (k_lu.cu).
//
//   analyse_kernel     one pass over A: lower and upper bandwidth (largest
//                      i - j and j - i over the non-zero elements), whether
//                      A equals A^T exactly, and the first zero on the
//                      diagonal.  32 x 32 tiles of the lower triangle, each
//                      read with its mirror tile so that the symmetry test
//                      needs no second pass.  Zero tests and comparisons
//                      work on the element bits with 32-bit integer
//                      operations.
//   diag_solve_kernel  X(i, c) = B(i, c) / A(i, i).
//   band_solve_kernel  Gaussian elimination with partial pivoting on the
//                      band (LAPACK's band LU: kl subdiagonals, ku
//                      superdiagonals, up to kl more superdiagonals of
//                      fill-in from the row interchanges), the right-hand
//                      sides eliminated alongside, then back substitution
//                      with the banded U.  One CTA: the band sits in shared
//                      memory when it fits (else in the workspace), one warp
//                      runs the elimination (lanes over the pivot
//                      candidates, the updated band elements and the
//                      right-hand sides) and the back substitution (lanes
//                      over right-hand sides).
#include <atomic>

#include "common.cuh"

namespace arma {
namespace {

__device__ __forceinline__ bool nz(double x) {
  return ((static_cast<uint32_t>(__double2hiint(x)) & 0x7FFFFFFFu) | static_cast<uint32_t>(__double2loint(x))) != 0u;
}
__device__ __forceinline__ bool nz(float x) { return (__float_as_uint(x) & 0x7FFFFFFFu) != 0u; }
__device__ __forceinline__ bool nz(__nv_bfloat16 x) { return (__bfloat16_as_ushort(x) & 0x7FFFu) != 0u; }

__device__ __forceinline__ bool same(double a, double b) {
  return (__double2hiint(a) == __double2hiint(b) && __double2loint(a) == __double2loint(b)) || (!nz(a) && !nz(b));
}
__device__ __forceinline__ bool same(float a, float b) {
  return __float_as_uint(a) == __float_as_uint(b) || (!nz(a) && !nz(b));
}
__device__ __forceinline__ bool same(__nv_bfloat16 a, __nv_bfloat16 b) {
  return __bfloat16_as_ushort(a) == __bfloat16_as_ushort(b) || (!nz(a) && !nz(b));
}

// tile (bi, bj) of the lower triangle (bi >= bj) and its mirror (bj, bi)
template <typename E>
__global__ void __launch_bounds__(256) analyse_kernel(const E* __restrict__ A, int64_t lda, int64_t n,
                                                      int32_t* props) {
  __shared__ E t[32][33];
  const int64_t bi = blockIdx.y, bj = blockIdx.x;
  if (bi < bj) return;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  int kl = 0, ku = 0, asym = 0, zd = 0, nonpos = 0;
  // mirror tile: element (r, c) = (32 bj + tx, 32 bi + q) kept as t[q][tx]
  for (int q = ty; q < 32; q += 8) {
    const int64_t r = bj * 32 + tx, c = bi * 32 + q;
    E v = E(0);
    if (r < n && c < n) {
      v = A[r + c * lda];
      if (bi != bj && nz(v)) ku = max(ku, (int)(c - r));   // c > r off the diagonal tile
    }
    t[q][tx] = v;
  }
  __syncthreads();
  // main tile: element (i, j) = (32 bi + tx, 32 bj + q); A(j, i) is t[tx][q]
  for (int q = ty; q < 32; q += 8) {
    const int64_t i = bi * 32 + tx, j = bj * 32 + q;
    if (i >= n || j >= n) continue;
    const E v = A[i + j * lda];
    const bool z = !nz(v);
    if (!z) {
      if (i > j) kl = max(kl, (int)(i - j));
      else if (j > i) ku = max(ku, (int)(j - i));
    } else if (i == j) {
      zd = max(zd, (int)(n - i));
    }
    if (i == j && !(v > E(0))) nonpos = 1;     // a diagonal element <= 0 (or NaN)
    if (!same(v, t[tx][q])) asym = 1;
  }
  kl = __reduce_max_sync(0xffffffffu, kl);
  ku = __reduce_max_sync(0xffffffffu, ku);
  asym = __reduce_or_sync(0xffffffffu, asym);
  zd = __reduce_max_sync(0xffffffffu, zd);
  nonpos = __reduce_or_sync(0xffffffffu, nonpos);
  if ((threadIdx.x & 31) == 0) {
    if (nonpos) atomicOr(props + SP_NONPOS, 1);
    if (kl) atomicMax(props + SP_KL, kl);
    if (ku) atomicMax(props + SP_KU, ku);
    if (asym) atomicOr(props + SP_ASYM, 1);
    if (zd) atomicMax(props + SP_ZDIAG, zd);
  }
}

template <typename T>
__global__ void diag_solve_kernel(const void* A, int64_t lda, int32_t adt, const void* B, int64_t ldb,
                                  int32_t bdt, void* X, int64_t ldx, int32_t xdt, int64_t n, int64_t nrhs) {
  const int64_t total = n * nrhs;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = t / n, i = t - c * n;
    const T b = B ? load_as<T>(B, i + c * ldb, bdt) : (T)(i == c ? 1 : 0);
    store_as<T>(X, i + c * ldx, xdt, b / load_as<T>(A, i + i * lda, adt));
  }
}

__global__ void set_props_kernel(int32_t* props, int32_t path, int32_t* status, int64_t* info, int64_t sing) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  props[SP_PATH] = path;
  if (sing > 0 && atomicCAS(status, 0, (int32_t)ARMA_ERR_SINGULAR) == 0) *info = sing;
}

__device__ __forceinline__ double rcp(double x) { return __drcp_rn(x); }
__device__ __forceinline__ float rcp(float x) { return __frcp_rn(x); }

// Magnitude of x as an integer key (non-negative floats order like their bit
// patterns), in 32-bit words: 64-bit integer work would share the FP64 pipe.
__device__ __forceinline__ void mag_key(double x, uint32_t& hi, uint32_t& lo) {
  hi = static_cast<uint32_t>(__double2hiint(x)) & 0x7FFFFFFFu;
  lo = static_cast<uint32_t>(__double2loint(x));
}
__device__ __forceinline__ void mag_key(float x, uint32_t& hi, uint32_t& lo) {
  hi = __float_as_uint(x) & 0x7FFFFFFFu;
  lo = 0u;
}

// The serial part (elimination, back substitution) uses 32-bit indices
// (the host keeps the work area below 2^31 elements) and no divisions.
template <typename T>
__global__ void __launch_bounds__(256) band_solve_kernel(const __grid_constant__ BandArgs a) {
  if (a.gate && *a.gate == 0) return;   // a fallback behind the tridiagonal kernel: not needed
  extern __shared__ __align__(16) unsigned char smraw[];
  T* base = a.in_smem ? reinterpret_cast<T*>(smraw) : static_cast<T*>(a.work);
  const int kl = a.kl, ku = a.ku, kv = kl + ku, ldab = 2 * kl + ku + 1;
  const int N = (int)a.n, R = (int)a.nrhs;
  T* AB = base;                              // A(i, j) at AB[j * ldab + kv + i - j]
  T* rinv = AB + N * ldab;                   // reciprocals of U's diagonal
  T* Xw = rinv + N;                          // right-hand sides, then the solution
  const int tid = threadIdx.x, nt = blockDim.x;
#pragma unroll 4
  for (int t = tid; t < N * ldab; t += nt) {
    const int j = t / ldab, i = j + (t - j * ldab) - kv;
    AB[t] = (i >= 0 && i < N && i >= j - ku) ? load_as<T>(a.A, i + (int64_t)j * a.lda, a.adt) : (T)0;
  }
#pragma unroll 4
  for (int t = tid; t < N * R; t += nt) {
    const int c = t / N, i = t - c * N;
    Xw[t] = a.B ? load_as<T>(a.B, i + (int64_t)c * a.ldb, a.bdt) : (T)(i == c ? 1 : 0);
  }
  __syncthreads();
  __shared__ int s_ok;
  if (tid < 32) {
    const int lane = tid;
    int ok = 1;
    for (int j = 0; j < N; ++j) {
      const int km = min(kl, N - 1 - j);
      T* colj = AB + j * ldab + kv;          // colj[l] = A(j + l, j)
      // pivot: the first largest magnitude among rows j .. j + km (lanes
      // past km hold key 0 and lose every tie to a lower lane)
      uint32_t khi = 0u, klo = 0u;
      if (lane <= km) mag_key(colj[lane], khi, klo);
      int bl = lane;
      for (int off = 1; off <= km; off <<= 1) {
        const uint32_t ohi = __shfl_xor_sync(0xffffffffu, khi, off);
        const uint32_t olo = __shfl_xor_sync(0xffffffffu, klo, off);
        const int ol = __shfl_xor_sync(0xffffffffu, bl, off);
        if (ohi > khi || (ohi == khi && (olo > klo || (olo == klo && ol < bl)))) {
          khi = ohi; klo = olo; bl = ol;
        }
      }
      bl = __shfl_sync(0xffffffffu, bl, 0);
      if ((__shfl_sync(0xffffffffu, khi, 0) | __shfl_sync(0xffffffffu, klo, 0)) == 0u) {
        if (lane == 0 && atomicCAS(a.status, 0, (int32_t)ARMA_ERR_SINGULAR) == 0) *a.info = j + 1;
        ok = 0;
        break;
      }
      const int ncol = min(kv, N - 1 - j);   // columns j + 1 .. j + ncol
      if (bl != 0) {
        for (int c = lane; c <= ncol; c += 32) {
          T* cc = AB + (j + c) * ldab + kv - c;   // cc[l] = A(j + l, j + c)
          const T u = cc[0];
          cc[0] = cc[bl];
          cc[bl] = u;
        }
        for (int r = lane; r < R; r += 32) {
          T* x = Xw + r * N + j;
          const T u = x[0];
          x[0] = x[bl];
          x[bl] = u;
        }
      }
      __syncwarp();
      const T rp = rcp(colj[0]);
      if (lane == 0) rinv[j] = rp;
      if (lane >= 1 && lane <= km) colj[lane] *= rp;
      __syncwarp();
      for (int l = 1; l <= km; ++l) {
        const T m = colj[l];
        for (int c = 1 + lane; c <= ncol; c += 32) {
          T* cc = AB + (j + c) * ldab + kv - c;
          cc[l] -= m * cc[0];
        }
        for (int r = lane; r < R; r += 32) {
          T* x = Xw + r * N + j;
          x[l] -= m * x[0];
        }
      }
      __syncwarp();
    }
    if (ok) {
      for (int r = lane; r < R; r += 32) {
        T* x = Xw + r * N;
        for (int j = N - 1; j >= 0; --j) {
          T sum = x[j];
          const int cmax = min(kv, N - 1 - j);
          const T* u = AB + (j + 1) * ldab + kv - 1;   // U(j, j + c) = u[c * (ldab - 1)]
          for (int c = 1; c <= cmax; ++c) sum -= u[(c - 1) * (ldab - 1)] * x[j + c];
          x[j] = sum * rinv[j];
        }
      }
    }
    if (lane == 0) s_ok = ok;
  }
  __syncthreads();
  if (!s_ok) return;
#pragma unroll 4
  for (int t = tid; t < N * R; t += nt) {
    const int c = t / N, i = t - c * N;
    store_as<T>(a.X, i + (int64_t)c * a.ldx, a.xdt, Xw[t]);
  }
}

// ---------------------------------------------------------------------------
// Tridiagonal systems (kl = ku = 1, the paper's expression (10)).  The same
// elimination with partial pivoting, but each step only decides between two
// rows, so one thread carries the state of the two live rows in registers:
// for step i, row i is (p, q) in columns (i, i + 1) and row i + 1 is
// (A(i+1, i), A(i+1, i+1), A(i+1, i+2)).  The larger of |p| and |A(i+1, i)|
// becomes the pivot row (ties keep row i); U gets that row (diagonal stored as
// its reciprocal, first and second superdiagonals), the multiplier and the
// interchange flag are kept for the right-hand sides, and the other row,
// reduced, carries on.  Each right-hand side is then solved by one thread:
// the recorded interchanges and multipliers forward, U backward.
//
// With FT = float for FP64 data the factors are FP32 and the solution is
// refined in FP64 inside the same launch: r = B - A X (from A itself),
// D = (LU)^-1 r, X += D, until the normwise backward error
// ||r|| / (||A|| ||X|| + ||B||) (Frobenius) is at most 1e-14, as for the
// general solve.  A zero or non-finite FP32 pivot, or no convergence after 10
// steps, sets the fallback word of the solve record; a direct FP64 band
// solve, launched behind this kernel and gated on that word, then runs.
// ---------------------------------------------------------------------------
constexpr int TRI_MAX_IR = 10;
constexpr double TRI_IR_TOL = 1e-14;

__host__ __device__ inline int64_t tri_align(int64_t b) { return (b + 15) / 16 * 16; }

// work area: the input diagonals (sub, main, super: n FT each), the factors
// dl, d (reciprocal), du, du2 (n FT each), interchange flags (n bytes), then
// X (n x nrhs DT, refinement only) and W (n x nrhs FT).  Inputs and factors
// live apart so that the elimination can load row i + 1 before it stores
// row i.
__host__ __device__ inline int64_t tri_bytes(int64_t n, int64_t nrhs, int dts, int fts, bool refine) {
  return tri_align((7 * n + 6) * fts) + tri_align(n) + (refine ? tri_align(n * nrhs * dts) : 0) +
         tri_align(n * nrhs * fts);
}

template <typename FT>
__device__ __forceinline__ bool finite_nz(FT x) { return x == x && x != (FT)0 && fabs(x) <= (FT)3.4e38; }
template <>
__device__ __forceinline__ bool finite_nz<double>(double x) {
  const uint32_t hi = static_cast<uint32_t>(__double2hiint(x)) & 0x7FFFFFFFu;
  return hi < 0x7FF00000u && (hi | static_cast<uint32_t>(__double2loint(x))) != 0u;
}

// reciprocal of a pivot: FP32 factors that FP64 refinement corrects take the
// hardware approximation (about 1 ulp); direct solves the rounded one
template <typename FT, bool APPROX>
__device__ __forceinline__ FT pivot_rcp(FT x) {
  if constexpr (APPROX && sizeof(FT) == 4) {
    float r;
    asm("rcp.approx.f32 %0, %1;" : "=f"(r) : "f"((float)x));
    return (FT)r;
  } else {
    return rcp(x);
  }
}

// one right-hand side w (n values) through the recorded factors; the next
// row's operands are loaded one step ahead of the dependent arithmetic
template <typename FT>
__device__ __forceinline__ void tri_apply(const FT* __restrict__ dl, const FT* __restrict__ rd,
                                          const FT* __restrict__ du, const FT* __restrict__ du2,
                                          const unsigned char* __restrict__ piv, FT* __restrict__ w, int N) {
  FT cur = w[0];
  FT nxt = N > 1 ? w[1] : (FT)0, m = dl[0];
  unsigned char sw = piv[0];
#pragma unroll 4
  for (int i = 0; i + 1 < N; ++i) {
    const FT nn = i + 2 < N ? w[i + 2] : (FT)0, mn = dl[i + 1];
    const unsigned char swn = piv[i + 1];
    const FT lo = sw ? nxt : cur, hi = sw ? cur : nxt;
    w[i] = lo;
    cur = hi - m * lo;
    nxt = nn; m = mn; sw = swn;
  }
  w[N - 1] = cur;
  FT x1 = 0, x2 = 0;
  FT wi = w[N - 1], ui = du[N - 1], u2 = du2[N - 1], ri = rd[N - 1];
#pragma unroll 4
  for (int i = N - 1; i >= 0; --i) {
    FT wn = 0, un = 0, u2n = 0, rn = 0;
    if (i > 0) { wn = w[i - 1]; un = du[i - 1]; u2n = du2[i - 1]; rn = rd[i - 1]; }
    const FT v = (wi - ui * x1 - u2 * x2) * ri;
    w[i] = v;
    x2 = x1; x1 = v;
    wi = wn; ui = un; u2 = u2n; ri = rn;
  }
}

// SMEM: the work area is this CTA's shared memory (then every access is a
// 32-bit shared-memory access), else the workspace.
template <typename DT, typename FT, bool REFINE, bool SMEM>
__global__ void __launch_bounds__(256) tridiag_kernel(const __grid_constant__ BandArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  unsigned char* base;
  if constexpr (SMEM) base = smraw;
  else base = static_cast<unsigned char*>(a.work);
  const int N = (int)a.n, R = (int)a.nrhs, tid = threadIdx.x, nt = blockDim.x;
  FT* a_dl = reinterpret_cast<FT*>(base);   // input diagonals (N + 2 each)
  FT* a_d = a_dl + (N + 2);
  FT* a_du = a_d + (N + 2);
  FT* dl = a_du + (N + 2);                    // factors
  FT* rd = dl + N;
  FT* du = rd + N;
  FT* du2 = du + N;
  unsigned char* piv = base + tri_align((7 * (int64_t)N + 6) * sizeof(FT));
  DT* X = reinterpret_cast<DT*>(piv + tri_align(N));
  FT* W = reinterpret_cast<FT*>(reinterpret_cast<unsigned char*>(X) +
                                (REFINE ? tri_align((int64_t)N * R * sizeof(DT)) : 0));
  auto Aat = [&](int i, int j) { return load_as<DT>(a.A, i + (int64_t)j * a.lda, a.adt); };
  auto Bat = [&](int i, int c) { return a.B ? load_as<DT>(a.B, i + (int64_t)c * a.ldb, a.bdt) : (DT)(i == c); };
  // the three diagonals (dl[i] = A(i+1, i), du[i] = A(i, i+1)) and W = B
  for (int i = tid; i < N + 2; i += nt) {
    a_d[i] = i < N ? (FT)Aat(i, i) : (FT)0;
    a_dl[i] = i + 1 < N ? (FT)Aat(i + 1, i) : (FT)0;
    a_du[i] = i + 1 < N ? (FT)Aat(i, i + 1) : (FT)0;
  }
  for (int t = tid; t < N * R; t += nt) {
    const int c = t / N, i = t - c * N;
    W[t] = (FT)Bat(i, c);
  }
  __shared__ int s_bad;
  __syncthreads();
  if (tid == 0) {
    int bad = 0;
    FT p = a_d[0], q = a_du[0];
    FT l = a_dl[0], d1 = a_d[1], u1 = N > 2 ? a_du[1] : (FT)0;
    // (a_d and a_du hold a zero past the last row, read by the look-ahead)
#pragma unroll 4
    for (int i = 0; i + 1 < N; ++i) {
      // row i + 2's operands, ahead of the dependent arithmetic
      const FT ln = a_dl[i + 1], dn = a_d[i + 2], un = a_du[i + 2];
      const bool swap = fabs(l) > fabs(p);
      const FT piv_v = swap ? l : p;
      bad = (bad == 0 && !finite_nz(piv_v)) ? i + 1 : bad;   // first bad pivot, no branch
      const FT r = pivot_rcp<FT, REFINE>(piv_v);
      const FT f = (swap ? p : l) * r;
      dl[i] = f;
      piv[i] = swap ? 1 : 0;
      rd[i] = r;
      du[i] = swap ? d1 : q;
      du2[i] = swap ? u1 : (FT)0;
      const FT np = swap ? q - f * d1 : d1 - f * q;
      q = swap ? -f * u1 : u1;
      p = np;
      l = ln; d1 = dn; u1 = un;
    }
    if (!bad) {
      if (!finite_nz(p)) bad = N;
      else rd[N - 1] = pivot_rcp<FT, REFINE>(p);
      du[N - 1] = (FT)0;
      du2[N - 1] = (FT)0;
      if (N > 1) du2[N - 2] = (FT)0;
    }
    s_bad = bad;
  }
  __syncthreads();
  if (s_bad) {
    if (tid == 0) {
      if (REFINE) *a.fallback = 1;                  // FP32 broke down: the FP64 solve decides
      else if (atomicCAS(a.status, 0, (int32_t)ARMA_ERR_SINGULAR) == 0) *a.info = s_bad;
    }
    return;
  }
  for (int c = tid; c < R; c += nt) tri_apply(dl, rd, du, du2, piv, W + (int64_t)c * N, N);
  __syncthreads();
  if constexpr (!REFINE) {
    for (int t = tid; t < N * R; t += nt) {
      const int c = t / N, i = t - c * N;
      store_as<DT>(a.X, i + (int64_t)c * a.ldx, a.xdt, (DT)W[t]);
    }
  } else {
    __shared__ double s_norm[2];
    __shared__ int s_done;
    for (int t = tid; t < N * R; t += nt) X[t] = (DT)W[t];
    // ||A||_F (the three diagonals) and ||B||_F, once
    double sa = 0.0, sb = 0.0;
    for (int i = tid; i < N; i += nt) {
      const double v0 = Aat(i, i), v1 = i + 1 < N ? (double)Aat(i + 1, i) : 0.0,
                   v2 = i + 1 < N ? (double)Aat(i, i + 1) : 0.0;
      sa += v0 * v0 + v1 * v1 + v2 * v2;
    }
    for (int t = tid; t < N * R; t += nt) {
      const int c = t / N, i = t - c * N;
      const double v = Bat(i, c);
      sb += v * v;
    }
    block_sum2(sa, sb);
    if (tid == 0) { s_norm[0] = sqrt(sa); s_norm[1] = sqrt(sb); s_done = 0; }
    __syncthreads();
    const double nA = s_norm[0], nB = s_norm[1];
    int step = 0;
    for (step = 1; step <= TRI_MAX_IR; ++step) {
      // r = B - A X in FP64, rounded into W for the correction solve
      double sr = 0.0, sx = 0.0;
      for (int t = tid; t < N * R; t += nt) {
        const int c = t / N, i = t - c * N;
        const DT* x = X + (int64_t)c * N;
        double r = (double)Bat(i, c) - (double)Aat(i, i) * (double)x[i];
        if (i > 0) r -= (double)Aat(i, i - 1) * (double)x[i - 1];
        if (i + 1 < N) r -= (double)Aat(i, i + 1) * (double)x[i + 1];
        W[t] = (FT)r;
        sr += r * r;
        sx += (double)x[i] * (double)x[i];
      }
      block_sum2(sr, sx);
      if (tid == 0) {
        const double nr = sqrt(sr), den = nA * sqrt(sx) + nB;
        const double bwd = den > 0.0 ? nr / den : nr;
        s_done = bwd <= TRI_IR_TOL ? 1 : (bwd == bwd && bwd <= 1e300) ? 0 : -1;
      }
      __syncthreads();
      if (s_done != 0) break;
      for (int c = tid; c < R; c += nt) tri_apply(dl, rd, du, du2, piv, W + (int64_t)c * N, N);
      __syncthreads();
      for (int t = tid; t < N * R; t += nt) X[t] += (DT)W[t];
      __syncthreads();
    }
    if (s_done != 1) {
      if (tid == 0) *a.fallback = 1;
      return;
    }
    if (tid == 0 && *a.status == 0) *a.info = step;   // refinement steps taken
    for (int t = tid; t < N * R; t += nt) {
      const int c = t / N, i = t - c * N;
      store_as<DT>(a.X, i + (int64_t)c * a.ldx, a.xdt, X[t]);
    }
  }
}

}  // namespace

int64_t band_work_bytes(int64_t n, int64_t nrhs, int32_t kl, int32_t ku, int32_t es) {
  const int64_t general = ((int64_t)(2 * kl + ku + 1) * n + n + n * nrhs) * es;
  const int64_t tri = tri_bytes(n, nrhs, 8, 8, true);
  return general > tri ? general : tri;
}

cudaError_t launch_analyse(const void* A, int64_t lda, int32_t adt, int64_t n, int32_t* props, cudaStream_t s,
                           int* launches) {
  if (n < 1) return cudaSuccess;
  const int64_t T = (n + 31) / 32;
  if (T > 65535) return cudaErrorInvalidConfiguration;
  dim3 grid((unsigned)T, (unsigned)T);
  if (adt == ARMA_F64) analyse_kernel<double><<<grid, 256, 0, s>>>(static_cast<const double*>(A), lda, n, props);
  else if (adt == ARMA_F32) analyse_kernel<float><<<grid, 256, 0, s>>>(static_cast<const float*>(A), lda, n, props);
  else analyse_kernel<__nv_bfloat16><<<grid, 256, 0, s>>>(static_cast<const __nv_bfloat16*>(A), lda, n, props);
  if (launches) ++*launches;
  return cudaGetLastError();
}

cudaError_t launch_set_props(int32_t* props, int32_t path, int32_t* status, int64_t* info, int64_t singular_at,
                             cudaStream_t s, int* launches) {
  set_props_kernel<<<1, 32, 0, s>>>(props, path, status, info, singular_at);
  if (launches) ++*launches;
  return cudaGetLastError();
}

cudaError_t launch_diag_solve(const SolveArgs& a, bool f64, cudaStream_t s, int* launches) {
  const int64_t total = a.n * a.nrhs;
  int64_t blocks = (total + 255) / 256, cap = (int64_t)device_sm_count() * 8;
  const unsigned g = (unsigned)(blocks < 1 ? 1 : blocks < cap ? blocks : cap);
  if (f64)
    diag_solve_kernel<double><<<g, 256, 0, s>>>(a.A, a.lda, a.adt, a.B, a.ldb, a.bdt, a.X, a.ldx, a.xdt, a.n, a.nrhs);
  else
    diag_solve_kernel<float><<<g, 256, 0, s>>>(a.A, a.lda, a.adt, a.B, a.ldb, a.bdt, a.X, a.ldx, a.xdt, a.n, a.nrhs);
  if (launches) ++*launches;
  return cudaGetLastError();
}

template <typename DT, typename FT, bool REFINE>
cudaError_t launch_tridiag(BandArgs a, cudaStream_t s) {
  const int64_t bytes = tri_bytes(a.n, a.nrhs, sizeof(DT), sizeof(FT), REFINE);
  constexpr int64_t SMEM_CAP = 200 * 1024;
  a.in_smem = bytes <= SMEM_CAP ? 1 : 0;
  if (!a.in_smem) {
    if (!a.work) return cudaErrorInvalidValue;
    tridiag_kernel<DT, FT, REFINE, false><<<1, 256, 0, s>>>(a);
    return cudaGetLastError();
  }
  static std::atomic<bool> attr[64];
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (!attr[dev].load(std::memory_order_acquire)) {
    cudaError_t e = cudaFuncSetAttribute(tridiag_kernel<DT, FT, REFINE, true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_CAP);
    if (e != cudaSuccess) return e;
    attr[dev].store(true, std::memory_order_release);
  }
  tridiag_kernel<DT, FT, REFINE, true><<<1, 256, (size_t)bytes, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_band_solve(BandArgs a, bool f64, cudaStream_t s, int* launches) {
  if (a.n >= (1ll << 31) || a.nrhs >= (1ll << 31) || a.n * a.nrhs >= (1ll << 31)) return cudaErrorInvalidValue;
  if (a.kl == 1 && a.ku == 1 && a.n >= 2) {
    cudaError_t e;
    if (!f64) {
      e = launch_tridiag<float, float, false>(a, s);
      if (launches) ++*launches;
      return e;
    }
    if (!a.refine) {
      e = launch_tridiag<double, double, false>(a, s);
      if (launches) ++*launches;
      return e;
    }
    e = launch_tridiag<double, float, true>(a, s);
    if (launches) ++*launches;
    if (e != cudaSuccess) return e;
    a.gate = a.fallback;                  // the direct FP64 band solve, only if needed
  }
  const int es = f64 ? 8 : 4;
  const int64_t bytes = band_work_bytes(a.n, a.nrhs, a.kl, a.ku, es);
  if (bytes / es >= (1ll << 31) || a.n >= (1ll << 31) || a.nrhs >= (1ll << 31)) return cudaErrorInvalidValue;
  constexpr int64_t SMEM_CAP = 200 * 1024;
  a.in_smem = bytes <= SMEM_CAP ? 1 : 0;
  if (!a.in_smem && !a.work) return cudaErrorInvalidValue;
  const size_t smem = a.in_smem ? (size_t)bytes : 0;
  cudaError_t e;
  if (f64) {
    e = cudaFuncSetAttribute(band_solve_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_CAP);
    if (e != cudaSuccess) return e;
    band_solve_kernel<double><<<1, 256, smem, s>>>(a);
  } else {
    e = cudaFuncSetAttribute(band_solve_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_CAP);
    if (e != cudaSuccess) return e;
    band_solve_kernel<float><<<1, 256, smem, s>>>(a);
  }
  if (launches) ++*launches;
  return cudaGetLastError();
}

}  // namespace arma
