// X = inv(A) * B as a solve: the paper's rewrite of inv(A)*b (Sec. I;
// Sec. II, the Glue<Op<Mat,op_inv>,Vec,glue_times> pattern mapped to xGESV;
// Sec. III (9)).  Blocked right-looking LU with partial pivoting (ties go to
// the smallest row index), then forward and back substitution, and for the
// mixed-precision tiers FP64 iterative refinement.
//
//   panel      one cooperative launch per 64-column panel: each CTA keeps its
//              block of panel rows in shared memory; per column the CTAs
//              publish their local pivot candidate and meet at one grid
//              barrier (bounded spin), then all pick the same pivot, swap and
//              update locally
//   laswp      the panel's row swaps applied to the other columns
//   trsm       U12 = L11^-1 A12
//   update     A22 -= L21 U12 through the product kernels: DFMA for the FP64
//              tier, split-BF16 tcgen05 (FP32-accurate) or BF16 tcgen05
//   trsv       one CTA per right-hand side: L then U substitution in smem
//   refine     r = B - A x in FP64 (DFMA), correction solved with the FP32
//              factors, x += d in FP64, until the normwise backward error
//              |r| / (|A||x| + |B|) <= 1e-14 or the step limit
//
// Numerical failures never trap: a zero pivot records ARMA_ERR_SINGULAR and
// its 1-based column in the workspace status; refinement that does not reach
// its tolerance records ARMA_ERR_NOCONVERGE.
#include <cooperative_groups.h>

#include "common.cuh"

namespace arma {

namespace lu {

constexpr int NB = 64;          // panel width
constexpr int PT = 256;         // panel threads per CTA
constexpr int MAX_CTAS = 64;
constexpr int MAX_IR = 10;
constexpr double IR_TOL = 1e-14;
constexpr unsigned int SPIN_LIMIT = 1u << 26;

struct Ctl {                    // device control block in the solve scratch
  unsigned int bar_count, bar_gen;
  int err;                      // barrier timeout
  int done;                     // refinement converged
  int steps;                    // refinement steps taken
  int pad;
  double nrmA, nrmB, nrmR, nrmX;
};

__device__ __forceinline__ bool grid_barrier(Ctl* c, unsigned int nblocks, int32_t* status) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned int* gen = &c->bar_gen;
    const unsigned int g = *gen;
    __threadfence();
    const unsigned int arrived = atomicAdd(&c->bar_count, 1u) + 1u;
    if (arrived == nblocks) {
      c->bar_count = 0u;
      __threadfence();
      atomicAdd(&c->bar_gen, 1u);
    } else {
      unsigned int i = 0;
      while (*gen == g) {
        if (++i > SPIN_LIMIT || *(volatile int*)&c->err) {
          atomicExch(&c->err, 1);
          atomicCAS(status, 0, (int32_t)ARMA_ERR_CUDA);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

template <typename T>
struct PanelArgs {
  T* A; int64_t ld, n;
  int64_t j;              // first panel column (and row)
  int32_t w;              // panel width
  int64_t rows_per_cta;
  int32_t* piv;
  double* cand_val;       // [2][MAX_CTAS]
  int64_t* cand_row;      // [2][MAX_CTAS]
  T* cand_data;           // [2][MAX_CTAS][NB]
  T* drow;                // [2][NB]
  Ctl* ctl;
  int32_t* status; int64_t* info;
};

template <typename T>
__global__ void __launch_bounds__(PT) panel_kernel(const __grid_constant__ PanelArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sm = reinterpret_cast<T*>(smraw);   // [w][R] column-major
  __shared__ double red_v[PT / 32];
  __shared__ int64_t red_r[PT / 32];
  __shared__ int64_t s_p;
  __shared__ int s_win;
  __shared__ T s_u[NB];
  const int64_t R = a.rows_per_cta;
  const int64_t r0 = a.j + (int64_t)blockIdx.x * R;             // first owned row
  const int64_t r1 = min(r0 + R, a.n);                          // one past last
  const int64_t nown = r1 > r0 ? r1 - r0 : 0;
  const int w = a.w;
  for (int64_t t = threadIdx.x; t < nown * w; t += PT) {
    const int64_t c = t / nown, r = t - c * nown;
    sm[c * R + r] = a.A[(r0 + r) + (a.j + c) * a.ld];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int c = 0; c < w; ++c) {
    const int64_t d = a.j + c;                 // global row of the diagonal
    const int ph = c & 1;
    // 1. local pivot candidate among owned rows >= d
    double bv = -1.0;
    int64_t br = INT64_MAX;
    for (int64_t r = threadIdx.x; r < nown; r += PT) {
      const int64_t g = r0 + r;
      if (g < d) continue;
      const double v = fabs((double)sm[c * R + r]);
      if (v > bv || (v == bv && g < br)) { bv = v; br = g; }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const double ov = __shfl_down_sync(0xffffffffu, bv, off);
      const int64_t orr = __shfl_down_sync(0xffffffffu, br, off);
      if (ov > bv || (ov == bv && orr < br)) { bv = ov; br = orr; }
    }
    if (lane == 0) { red_v[wid] = bv; red_r[wid] = br; }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int q = 1; q < PT / 32; ++q)
        if (red_v[q] > bv || (red_v[q] == bv && red_r[q] < br)) { bv = red_v[q]; br = red_r[q]; }
      a.cand_val[ph * MAX_CTAS + blockIdx.x] = bv;
      a.cand_row[ph * MAX_CTAS + blockIdx.x] = br;
      s_p = br;
    }
    __syncthreads();
    // publish the candidate row and, if owned here, row d (panel columns only)
    if (s_p >= r0 && s_p < r1)
      for (int q = threadIdx.x; q < w; q += PT)
        a.cand_data[((int64_t)ph * MAX_CTAS + blockIdx.x) * NB + q] = sm[q * R + (s_p - r0)];
    if (d >= r0 && d < r1)
      for (int q = threadIdx.x; q < w; q += PT) a.drow[ph * NB + q] = sm[q * R + (d - r0)];
    __threadfence();
    // 2. all CTAs meet
    if (!grid_barrier(a.ctl, gridDim.x, a.status)) return;
    // 3. every CTA picks the same pivot
    if (threadIdx.x == 0) {
      double v = -1.0;
      int64_t p = INT64_MAX;
      int win = -1;
      for (unsigned int b = 0; b < gridDim.x; ++b) {
        const double cv = __ldcg(a.cand_val + ph * MAX_CTAS + b);
        const int64_t cr = __ldcg(reinterpret_cast<const long long*>(a.cand_row) + ph * MAX_CTAS + b);
        if (cv > v || (cv == v && cr < p)) { v = cv; p = cr; win = (int)b; }
      }
      if (v <= 0.0) {             // exact zero column: singular, keep going
        if (atomicCAS(a.status, 0, (int32_t)ARMA_ERR_SINGULAR) == 0) *a.info = d + 1;
        p = d;
        win = -1;
      }
      s_p = p;
      s_win = win;
      if (blockIdx.x == 0) a.piv[d] = (int32_t)p;
    }
    __syncthreads();
    const int64_t p = s_p;
    const int win = s_win;
    // pivot row values (panel columns)
    for (int q = threadIdx.x; q < w; q += PT) {
      T u;
      if (win >= 0) u = __ldcg(a.cand_data + ((int64_t)ph * MAX_CTAS + win) * NB + q);
      else u = __ldcg(a.drow + ph * NB + q);
      s_u[q] = u;
    }
    __syncthreads();
    // 4. swap rows d and p inside the panel
    if (p != d) {
      if (d >= r0 && d < r1)
        for (int q = threadIdx.x; q < w; q += PT) sm[q * R + (d - r0)] = s_u[q];
      if (p >= r0 && p < r1)
        for (int q = threadIdx.x; q < w; q += PT) sm[q * R + (p - r0)] = __ldcg(a.drow + ph * NB + q);
    }
    __syncthreads();
    // 5. scale the column below the pivot and update the rest of the panel
    const T pv = s_u[c];
    if (win >= 0) {
      for (int64_t r = threadIdx.x; r < nown; r += PT) {
        if (r0 + r <= d) continue;
        const T l = sm[c * R + r] / pv;
        sm[c * R + r] = l;
        for (int q = c + 1; q < w; ++q) sm[q * R + r] -= l * s_u[q];
      }
    }
    __syncthreads();
  }
  for (int64_t t = threadIdx.x; t < nown * w; t += PT) {
    const int64_t c = t / nown, r = t - c * nown;
    a.A[(r0 + r) + (a.j + c) * a.ld] = sm[c * R + r];
  }
}

// the panel's row swaps applied to columns outside [j, j + w)
template <typename T>
__global__ void laswp_kernel(T* A, int64_t ld, int64_t n, int64_t j, int w, const int32_t* piv) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t others = n - w;
  if (k >= others) return;
  const int64_t col = k < j ? k : k + w;
  for (int c = 0; c < w; ++c) {
    const int64_t d = j + c, p = piv[d];
    if (p != d) {
      const T t = A[d + col * ld];
      A[d + col * ld] = A[p + col * ld];
      A[p + col * ld] = t;
    }
  }
}

// U12 = L11^-1 A12 (L11 unit lower w x w), one thread per column of A12
template <typename T>
__global__ void trsm_kernel(T* A, int64_t ld, int64_t n, int64_t j, int w) {
  __shared__ T L[NB * NB];
  for (int t = threadIdx.x; t < w * w; t += blockDim.x) {
    const int r = t % w, c = t / w;
    L[c * NB + r] = A[(j + r) + (j + c) * ld];
  }
  __syncthreads();
  const int64_t col = j + w + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= n) return;
  T x[NB];
  for (int r = 0; r < w; ++r) x[r] = A[(j + r) + col * ld];
  for (int r = 0; r < w; ++r)
    for (int r2 = r + 1; r2 < w; ++r2) x[r2] -= L[r * NB + r2] * x[r];
  for (int r = 0; r < w; ++r) A[(j + r) + col * ld] = x[r];
}

// perm = composition of the row swaps; Y(:, c) = P * B(:, c) (B null: identity)
__global__ void perm_kernel(const int32_t* piv, int32_t* perm, int64_t n) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
  for (int64_t d = 0; d < n; ++d) {
    const int64_t p = piv[d];
    const int32_t t = perm[d];
    perm[d] = perm[p];
    perm[p] = t;
  }
}

template <typename T>
__global__ void gather_kernel(const void* B, int64_t ldb, int32_t bdt, const int32_t* perm, T* Y, int64_t n,
                              int64_t nrhs, const int* skip) {
  if (skip && *skip) return;
  const int64_t total = n * nrhs;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = t / n, i = t - c * n;
    const int64_t src = perm[i];
    T v;
    if (B) v = load_as<T>(B, src + c * ldb, bdt);
    else v = (src == c) ? (T)1 : (T)0;
    Y[i + c * n] = v;
  }
}

// one CTA per right-hand side: y := U^-1 L^-1 y, y in shared memory
template <typename T>
__global__ void __launch_bounds__(256) trsv_kernel(const T* LU, int64_t ld, int64_t n, T* Y, int64_t ldy,
                                                  const int* skip) {
  if (skip && *skip) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* y = reinterpret_cast<T*>(smraw);
  T* col = Y + (int64_t)blockIdx.x * ldy;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) y[i] = col[i];
  __syncthreads();
  for (int64_t i = 0; i < n; ++i) {            // unit lower
    const T yi = y[i];
    for (int64_t r = i + 1 + threadIdx.x; r < n; r += blockDim.x) y[r] -= LU[r + i * ld] * yi;
    __syncthreads();
  }
  for (int64_t i = n - 1; i >= 0; --i) {       // upper
    __shared__ T s_yi;
    if (threadIdx.x == 0) {
      const T piv = LU[i + i * ld];
      s_yi = piv != (T)0 ? y[i] / piv : (T)0;
      y[i] = s_yi;
    }
    __syncthreads();
    const T yi = s_yi;
    for (int64_t r = threadIdx.x; r < i; r += blockDim.x) y[r] -= LU[r + i * ld] * yi;
    __syncthreads();
  }
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) col[i] = y[i];
}

// convert A into the LU work matrix
template <typename T>
__global__ void copy_kernel(const void* A, int64_t lda, int32_t adt, T* W, int64_t n) {
  const int64_t total = n * n;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = t / n, i = t - c * n;
    W[t] = load_as<T>(A, i + c * lda, adt);
  }
}

// X (output, any type) = Y
template <typename T>
__global__ void store_kernel(const T* Y, int64_t n, int64_t nrhs, void* X, int64_t ldx, int32_t xdt) {
  const int64_t total = n * nrhs;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = t / n, i = t - c * n;
    store_as<double>(X, i + c * ldx, xdt, (double)Y[t]);
  }
}

// refinement bookkeeping: sum of squares -> convergence flag
__global__ void ir_check_kernel(Ctl* c, const double* sq, int step, int32_t* status, int64_t* info, int last) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (c->done) return;
  const double nr = sqrt(sq[0]), nx = sqrt(sq[1]);
  const double denom = c->nrmA * nx + c->nrmB;
  const double bwd = denom > 0.0 ? nr / denom : nr;
  c->steps = step;
  if (bwd <= IR_TOL) {
    c->done = 1;
  } else if (last) {
    if (atomicCAS(status, 0, (int32_t)ARMA_ERR_NOCONVERGE) == 0) *info = step;
  }
}

__global__ void norms_init_kernel(Ctl* c, const double* sq) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  c->nrmA = sqrt(sq[0]);
  c->nrmB = sqrt(sq[1]);
}

// x += d (FP64), skipped once converged
__global__ void ir_update_kernel(double* X, const float* D, int64_t total, const int* skip) {
  if (*skip) return;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x)
    X[t] += (double)D[t];
}

// second stage of a sum of squares: add the per-block partials in order
__global__ void sum_partials_kernel(const double* part, int count, double* out, int k) {
  double s = 0.0;
  for (int t = threadIdx.x; t < count; t += blockDim.x) s += part[t];
  double q = 0.0;
  block_sum2(s, q);
  if (threadIdx.x == 0) out[k] = s;
}

__global__ void sumsq_any_kernel(const void* x, int32_t dt, int64_t ld, int64_t rows, int64_t cols,
                                 double* partial) {
  // per-block sums of squares, added up by sum_partials_kernel
  double s = 0.0;
  const int64_t total = rows * cols;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = t / rows, i = t - c * rows;
    const double v = load_as<double>(x, i + c * ld, dt);
    s = fma(v, v, s);
  }
  double q = 0.0;
  block_sum2(s, q);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

struct Layout {
  int64_t lu, piv, perm, cand_val, cand_row, cand_data, drow, ctl, gemm, y, x64, r64, sq, part, total;
  int64_t gemm_bytes;
  bool f64;
  bool refine;
};

Layout layout(int64_t n, int64_t nrhs, int32_t tier) {
  Layout L;
  L.f64 = tier == ARMA_TIER_F64;
  L.refine = tier == ARMA_TIER_LU32_IR64 || tier == ARMA_TIER_BF16;
  const int64_t es = L.f64 ? 8 : 4;
  int64_t off = 0;
  auto take = [&](int64_t bytes) { int64_t o = off; off += (bytes + 255) / 256 * 256; return o; };
  L.lu = take(n * n * es);
  L.piv = take(n * 4);
  L.perm = take(n * 4);
  L.cand_val = take(2 * MAX_CTAS * 8);
  L.cand_row = take(2 * MAX_CTAS * 8);
  L.cand_data = take(2 * MAX_CTAS * NB * es);
  L.drow = take(2 * NB * es);
  L.ctl = take(sizeof(Ctl));
  const int32_t gt = L.f64 ? ARMA_TIER_F64 : tier == ARMA_TIER_BF16 ? ARMA_TIER_BF16 : ARMA_TIER_SPLIT_BF16;
  int64_t gb = gemm_tc_scratch_bytes(n, n, NB, gt);
  if (gb < 64 * n * 8) gb = 64 * n * 8;            // GEMV partials for 1-wide updates
  if (L.f64) {
    const int64_t sb = gemm_simt_scratch_bytes(n, n, NB);
    if (gb < sb) gb = sb;
  }
  if (L.refine) {
    const int64_t rb = gemm_simt_scratch_bytes(n, nrhs, n);   // FP64 residual
    if (gb < rb) gb = rb;
  }
  L.gemm_bytes = gb;
  L.gemm = take(gb);
  L.y = take(n * nrhs * es);
  L.x64 = L.refine ? take(n * nrhs * 8) : 0;
  L.r64 = L.refine ? take(n * nrhs * 8) : 0;
  L.sq = take(8 * 8);
  L.part = take(1024 * 8);
  L.total = off + 256;
  return L;
}

template <typename T>
cudaError_t factor(const SolveArgs& a, const Layout& L, char* base, cudaStream_t s, int* launches) {
  const int64_t n = a.n;
  T* W = reinterpret_cast<T*>(base + L.lu);
  int32_t* piv = reinterpret_cast<int32_t*>(base + L.piv);
  Ctl* ctl = reinterpret_cast<Ctl*>(base + L.ctl);
  const int sms = device_sm_count();
  {
    int64_t blocks = (n * n + 255) / 256, cap = (int64_t)sms * 8;
    copy_kernel<T><<<(unsigned)(blocks < cap ? blocks : cap), 256, 0, s>>>(a.A, a.lda, a.adt, W, n);
    if (launches) ++*launches;
  }
  const int32_t gt = L.f64 ? ARMA_TIER_F64 : a.tier == ARMA_TIER_BF16 ? ARMA_TIER_BF16 : ARMA_TIER_SPLIT_BF16;
  for (int64_t j = 0; j < n; j += NB) {
    const int w = (int)(n - j < NB ? n - j : NB);
    // panel
    PanelArgs<T> pa;
    pa.A = W; pa.ld = n; pa.n = n; pa.j = j; pa.w = w;
    int64_t rows = n - j;
    int ctas = (int)((rows + PT - 1) / PT);
    if (ctas < 1) ctas = 1;
    if (ctas > MAX_CTAS) ctas = MAX_CTAS;
    if (ctas > sms) ctas = sms;
    pa.rows_per_cta = (rows + ctas - 1) / ctas;
    ctas = (int)((rows + pa.rows_per_cta - 1) / pa.rows_per_cta);
    pa.piv = piv;
    pa.cand_val = reinterpret_cast<double*>(base + L.cand_val);
    pa.cand_row = reinterpret_cast<int64_t*>(base + L.cand_row);
    pa.cand_data = reinterpret_cast<T*>(base + L.cand_data);
    pa.drow = reinterpret_cast<T*>(base + L.drow);
    pa.ctl = ctl;
    pa.status = a.status_code;
    pa.info = a.status_info;
    const size_t smem = (size_t)pa.rows_per_cta * w * sizeof(T);
    if (smem > 200 * 1024) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(panel_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    void* kargs[] = {&pa};
    e = cudaLaunchCooperativeKernel((const void*)panel_kernel<T>, dim3(ctas), dim3(PT), kargs, smem, s);
    if (e != cudaSuccess) return e;
    if (launches) ++*launches;
    if (n > w) {
      const int64_t others = n - w;
      laswp_kernel<T><<<(unsigned)((others + 255) / 256), 256, 0, s>>>(W, n, n, j, w, piv);
      if (launches) ++*launches;
    }
    const int64_t rest = n - j - w;
    if (rest > 0) {
      trsm_kernel<T><<<(unsigned)((rest + 127) / 128), 128, 0, s>>>(W, n, n, j, w);
      if (launches) ++*launches;
      GemmArgs g;
      memset(&g, 0, sizeof g);
      const int dt = L.f64 ? ARMA_F64 : ARMA_F32;
      g.m = rest; g.n = rest; g.k = w;
      g.A = W + (j + w) + j * n; g.lda = n; g.ta = 0; g.adt = dt;
      g.B = W + j + (j + w) * n; g.ldb = n; g.tb = 0; g.bdt = dt;
      g.C = W + (j + w) + (j + w) * n; g.ldc = n; g.cdt = dt;
      g.D = W + (j + w) + (j + w) * n; g.ldd = n; g.ddt = dt;
      g.alpha = -1.0; g.beta = 1.0;
      g.tier = gt;
      g.scratch = base + L.gemm; g.scratch_bytes = L.gemm_bytes;
      g.status = a.status_code;
      e = launch_gemm(g, s, launches);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t substitute(const T* W, int64_t n, T* Y, int64_t nrhs, const int* skip, cudaStream_t s, int* launches) {
  const size_t smem = (size_t)n * sizeof(T);
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(trsv_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  trsv_kernel<T><<<(unsigned)nrhs, 256, smem, s>>>(W, n, n, Y, n, skip);
  if (launches) ++*launches;
  return cudaGetLastError();
}

}  // namespace lu

int64_t solve_scratch_bytes(int64_t n, int64_t nrhs, int32_t tier) {
  return lu::layout(n, nrhs, tier).total;
}

cudaError_t launch_solve(const SolveArgs& a, cudaStream_t s, int* launches) {
  using namespace lu;
  const int64_t n = a.n, nrhs = a.nrhs;
  if (n == 0 || nrhs == 0) return cudaSuccess;
  Layout L = layout(n, nrhs, a.tier);
  if (a.scratch_bytes < L.total) return cudaErrorInvalidValue;
  char* base = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(a.scratch) + 255) & ~uintptr_t(255));
  Ctl* ctl = reinterpret_cast<Ctl*>(base + L.ctl);
  cudaError_t e = cudaMemsetAsync(ctl, 0, sizeof(Ctl), s);
  if (e != cudaSuccess) return e;
  const int sms = device_sm_count();
  int32_t* piv = reinterpret_cast<int32_t*>(base + L.piv);
  int32_t* perm = reinterpret_cast<int32_t*>(base + L.perm);
  auto grid_for = [&](int64_t total) {
    int64_t b = (total + 255) / 256, cap = (int64_t)sms * 8;
    return (unsigned)(b < 1 ? 1 : b < cap ? b : cap);
  };
  if (L.f64) {
    e = factor<double>(a, L, base, s, launches);
    if (e != cudaSuccess) return e;
    double* Y = reinterpret_cast<double*>(base + L.y);
    perm_kernel<<<1, 32, 0, s>>>(piv, perm, n);
    gather_kernel<double><<<grid_for(n * nrhs), 256, 0, s>>>(a.B, a.ldb, a.bdt, perm, Y, n, nrhs, nullptr);
    e = substitute<double>(reinterpret_cast<double*>(base + L.lu), n, Y, nrhs, nullptr, s, launches);
    if (e != cudaSuccess) return e;
    store_kernel<double><<<grid_for(n * nrhs), 256, 0, s>>>(Y, n, nrhs, a.X, a.ldx, a.xdt);
    if (launches) *launches += 3;
    return cudaGetLastError();
  }
  e = factor<float>(a, L, base, s, launches);
  if (e != cudaSuccess) return e;
  const float* W = reinterpret_cast<const float*>(base + L.lu);
  float* Y = reinterpret_cast<float*>(base + L.y);
  perm_kernel<<<1, 32, 0, s>>>(piv, perm, n);
  gather_kernel<float><<<grid_for(n * nrhs), 256, 0, s>>>(a.B, a.ldb, a.bdt, perm, Y, n, nrhs, nullptr);
  e = substitute<float>(W, n, Y, nrhs, nullptr, s, launches);
  if (e != cudaSuccess) return e;
  if (launches) *launches += 2;
  if (!L.refine || !a.B) {
    store_kernel<float><<<grid_for(n * nrhs), 256, 0, s>>>(Y, n, nrhs, a.X, a.ldx, a.xdt);
    if (launches) ++*launches;
    return cudaGetLastError();
  }
  // ---- FP64 iterative refinement ----
  double* X64 = reinterpret_cast<double*>(base + L.x64);
  double* R64 = reinterpret_cast<double*>(base + L.r64);
  double* sq = reinterpret_cast<double*>(base + L.sq);
  double* part = reinterpret_cast<double*>(base + L.part);
  store_kernel<float><<<grid_for(n * nrhs), 256, 0, s>>>(Y, n, nrhs, X64, n, ARMA_F64);
  // |A|_F, |B|_F once
  sumsq_any_kernel<<<512, 256, 0, s>>>(a.A, a.adt, a.lda, n, n, part);
  sum_partials_kernel<<<1, 256, 0, s>>>(part, 512, sq, 0);
  sumsq_any_kernel<<<512, 256, 0, s>>>(a.B, a.bdt, a.ldb, n, nrhs, part);
  sum_partials_kernel<<<1, 256, 0, s>>>(part, 512, sq, 1);
  norms_init_kernel<<<1, 32, 0, s>>>(ctl, sq);
  if (launches) *launches += 6;
  for (int it = 1; it <= MAX_IR; ++it) {
    // r = B - A x (FP64)
    GemmArgs g;
    memset(&g, 0, sizeof g);
    g.m = n; g.n = nrhs; g.k = n;
    g.A = a.A; g.lda = a.lda; g.ta = 0; g.adt = a.adt;
    g.B = X64; g.ldb = n; g.tb = 0; g.bdt = ARMA_F64;
    g.C = a.B; g.ldc = a.ldb; g.cdt = a.bdt;
    g.D = R64; g.ldd = n; g.ddt = ARMA_F64;
    g.alpha = -1.0; g.beta = 1.0;
    g.tier = ARMA_TIER_F64;
    g.scratch = base + L.gemm; g.scratch_bytes = L.gemm_bytes;
    g.status = a.status_code;
    g.skip = &ctl->done;
    e = launch_gemm(g, s, launches);
    if (e != cudaSuccess) return e;
    sumsq_any_kernel<<<512, 256, 0, s>>>(R64, ARMA_F64, n, n, nrhs, part);
    sum_partials_kernel<<<1, 256, 0, s>>>(part, 512, sq + 2, 0);
    sumsq_any_kernel<<<512, 256, 0, s>>>(X64, ARMA_F64, n, n, nrhs, part);
    sum_partials_kernel<<<1, 256, 0, s>>>(part, 512, sq + 2, 1);
    ir_check_kernel<<<1, 32, 0, s>>>(ctl, sq + 2, it, a.status_code, a.status_info, it == MAX_IR);
    // d = (LU)^-1 P r in FP32; x += d
    gather_kernel<float><<<grid_for(n * nrhs), 256, 0, s>>>(R64, n, ARMA_F64, perm, Y, n, nrhs, &ctl->done);
    e = substitute<float>(W, n, Y, nrhs, &ctl->done, s, launches);
    if (e != cudaSuccess) return e;
    ir_update_kernel<<<grid_for(n * nrhs), 256, 0, s>>>(X64, Y, n * nrhs, &ctl->done);
    if (launches) *launches += 7;
  }
  store_kernel<double><<<grid_for(n * nrhs), 256, 0, s>>>(X64, n, nrhs, a.X, a.ldx, a.xdt);
  if (launches) ++*launches;
  return cudaGetLastError();
}

}  // namespace arma
