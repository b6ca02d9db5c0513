// Product kernels that need no tensor cores: the FP64 DFMA GEMM (the FP64
// tier and the refinement residual), GEMV for matrix-vector chains, the
// diagonal-only product behind trace(A*B) (Sec. III (5)), and the explicit
// transpose / dense-diagonal copies that only the literal plan uses.
//
// Column-major everywhere; op(X) is X or X^T.  The product kernels fold
// alpha, beta*C, a row scaling diag(r) and a column scaling diag(c) into
// their epilogue, so 2*A*B + C, trans(A)*B and diagmat(v)*(A*B) are single
// launches (Sec. II, the folded scalar and transpose flags of Fig. 3).
#include "common.cuh"

namespace arma {

cudaError_t launch_gemm_tc(const GemmArgs& a, cudaStream_t s, int* launches);
bool gemm_tc_supported(const GemmArgs& a);

namespace {

// ---------------------------------------------------------------------------
// SIMT GEMM: 64 x 64 tile, BK = 16, 256 threads, 4 x 4 outputs per thread.
// Accumulates in AT (double for the FP64 tier, float otherwise).
// ---------------------------------------------------------------------------
constexpr int BM = 64, BN = 64, BK = 16;

// blockIdx.z selects a K range when the output has too few tiles to fill
// the GPU; those partial sums go to scratch (FP64) and a second kernel
// combines them in a fixed order.
template <typename AT>
__global__ void __launch_bounds__(256) gemm_simt_kernel(const __grid_constant__ GemmArgs a) {
  if (a.skip && *a.skip) return;
  __shared__ AT As[BK][BM + 1];
  __shared__ AT Bs[BK][BN + 1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  int64_t ti = blockIdx.x, tj = blockIdx.y;
  if (a.sym) {
    // lower-triangle tiles only, row by row: tile row ti holds ti + 1 tiles
    const int64_t b = blockIdx.x;
    ti = (int64_t)((sqrtf(8.f * (float)b + 1.f) - 1.f) * 0.5f);
    while (ti * (ti + 1) / 2 > b) --ti;
    while ((ti + 1) * (ti + 2) / 2 <= b) ++ti;
    tj = b - ti * (ti + 1) / 2;
  }
  const int64_t i0 = ti * BM, j0 = tj * BN;
  const int64_t kchunk = (a.k + gridDim.z - 1) / gridDim.z;
  const int64_t kbeg = (int64_t)blockIdx.z * kchunk;
  const int64_t kend = kbeg + kchunk < a.k ? kbeg + kchunk : a.k;
  AT acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = 0;
  for (int64_t l0 = kbeg; l0 < kend; l0 += BK) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int e = tid + r * 256;
      int ii, ll;
      if (!a.ta) { ii = e & 63; ll = e >> 6; } else { ll = e & 15; ii = e >> 4; }
      int64_t gi = i0 + ii, gl = l0 + ll;
      AT v = 0;
      if (gi < a.m && gl < kend) v = load_as<AT>(a.A, a.ta ? gl + gi * a.lda : gi + gl * a.lda, a.adt);
      As[ll][ii] = v;
      int jj;
      if (!a.tb) { ll = e & 15; jj = e >> 4; } else { jj = e & 63; ll = e >> 6; }
      int64_t gj = j0 + jj;
      gl = l0 + ll;
      AT w = 0;
      if (gl < kend && gj < a.n) w = load_as<AT>(a.B, a.tb ? gj + gl * a.ldb : gl + gj * a.ldb, a.bdt);
      Bs[ll][jj] = w;
    }
    __syncthreads();
#pragma unroll
    for (int l = 0; l < BK; ++l) {
      AT av[4], bv[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) av[r] = As[l][tx + 16 * r];
#pragma unroll
      for (int c = 0; c < 4; ++c) bv[c] = Bs[l][ty + 16 * c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = fma(av[r], bv[c], acc[r][c]);
    }
    __syncthreads();
  }
  if (gridDim.z > 1) {
    double* P = static_cast<double*>(a.scratch) + (int64_t)blockIdx.z * a.m * a.n;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      int64_t j = j0 + ty + 16 * c;
      if (j >= a.n) continue;
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        int64_t i = i0 + tx + 16 * r;
        if (i < a.m) P[i + j * a.m] = (double)acc[r][c];
      }
    }
    return;
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    int64_t j = j0 + ty + 16 * c;
    if (j >= a.n) continue;
    double cj = a.cs ? load_as<double>(a.cs, j * a.cs_inc, a.csdt) : 1.0;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int64_t i = i0 + tx + 16 * r;
      if (i >= a.m) continue;
      double v = a.alpha * (double)acc[r][c];
      if (a.rs) v *= load_as<double>(a.rs, i * a.rs_inc, a.rsdt);
      v *= cj;
      if (a.C && a.beta != 0.0) v += a.beta * load_as<double>(a.C, i + j * a.ldc, a.cdt);
      store_as<double>(a.D, i + j * a.ldd, a.ddt, v);
    }
  }
}

__global__ void __launch_bounds__(256) gemm_simt_combine_kernel(const __grid_constant__ GemmArgs a, int splits) {
  if (a.skip && *a.skip) return;
  const int64_t total = a.m * a.n;
  const double* P = static_cast<const double*>(a.scratch);
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = t / a.m, i = t - j * a.m;
    if (a.sym && i < j) continue;   // not computed; mirrored afterwards
    double s = 0.0;
    for (int z = 0; z < splits; ++z) s += P[(int64_t)z * total + t];
    double v = a.alpha * s;
    if (a.rs) v *= load_as<double>(a.rs, i * a.rs_inc, a.rsdt);
    if (a.cs) v *= load_as<double>(a.cs, j * a.cs_inc, a.csdt);
    if (a.C && a.beta != 0.0) v += a.beta * load_as<double>(a.C, i + j * a.ldc, a.cdt);
    store_as<double>(a.D, i + j * a.ldd, a.ddt, v);
  }
}

// The K split minimises the busiest SM's share of the multiply-adds (the
// FP64 pipe does 2 per SM and clock here, so even a 64 x 64 x 16 piece is
// 32k clocks) plus the combine pass: s partial sums written and read back at
// HBM speed and one more launch, all in SM clocks.  Every K piece is at
// least one BK block, and the partial sums stay within 256 MB.
int simt_splits(int64_t m, int64_t n, int64_t k) {
  constexpr int64_t SMS = 152;
  const int64_t tiles = ((m + BM - 1) / BM) * ((n + BN - 1) / BN);
  int best = 1;
  double best_cost = 0.0;
  for (int s = 1; s <= 64; s *= 2) {
    if (s > 1 && ((k + s - 1) / s < BK || (double)s * (double)m * (double)n * 8.0 > 256e6)) break;
    const int64_t waves = (tiles * s + SMS - 1) / SMS;
    double cost = (double)waves * (double)((k + s - 1) / s) * (BM * BN / 2);
    if (s > 1) cost += (double)s * (double)m * (double)n * 16.0 * 3.04e-4 + 4000.0;
    if (s == 1 || cost < best_cost) { best = s; best_cost = cost; }
  }
  return best;
}

// ---------------------------------------------------------------------------
// GEMV: y_i = alpha * sum_l M(i, l) x_l, M(i, l) at M[i*rsm + l*csm].
// ---------------------------------------------------------------------------
struct GemvArgs {
  int64_t rows, k;
  const void* M; int64_t rsm, csm; int32_t mdt;
  const void* x; int64_t incx; int32_t xdt;
  void* y; int64_t incy; int32_t ydt;
  const void* c; int64_t incc; int32_t cdt; double beta;
  double alpha;
  const void* rsv; int64_t rs_inc; int32_t rsdt;   // per-output scale
  const void* sv; int32_t svdt;                     // one scale factor (1 x 1 diagonal)
  double scal;
  double* partials;  // [splits][rows] when splits > 1
  int32_t splits;
  const int* skip;
};

__device__ __forceinline__ void gemv_out(const GemvArgs& a, int64_t i, double sum) {
  double v = a.alpha * a.scal * sum;
  if (a.rsv) v *= load_as<double>(a.rsv, i * a.rs_inc, a.rsdt);
  if (a.sv) v *= load_as<double>(a.sv, 0, a.svdt);
  if (a.c && a.beta != 0.0) v += a.beta * load_as<double>(a.c, i * a.incc, a.cdt);
  store_as<double>(a.y, i * a.incy, a.ydt, v);
}

// rows contiguous in memory (rsm == 1): one thread per row, k split in chunks
__global__ void __launch_bounds__(256) gemv_rows_kernel(const __grid_constant__ GemvArgs a) {
  if (a.skip && *a.skip) return;
  __shared__ double xs[256];
  const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
  const int64_t chunk = (a.k + a.splits - 1) / a.splits;
  const int64_t lb = (int64_t)blockIdx.y * chunk;
  const int64_t le = lb + chunk < a.k ? lb + chunk : a.k;
  double sum = 0.0;
  for (int64_t l0 = lb; l0 < le; l0 += 256) {
    int64_t l = l0 + threadIdx.x;
    xs[threadIdx.x] = l < le ? load_as<double>(a.x, l * a.incx, a.xdt) : 0.0;
    __syncthreads();
    int64_t cnt = le - l0 < 256 ? le - l0 : 256;
    if (i < a.rows) {
      if (a.mdt == ARMA_F64) {
        // four independent accumulators: the DFMA latency is not a chain
        const double* M = static_cast<const double*>(a.M) + i + l0 * a.csm;
        double s4[4] = {0.0, 0.0, 0.0, 0.0};
        int u = 0;
        for (; u + 4 <= cnt; u += 4) {
#pragma unroll
          for (int q = 0; q < 4; ++q) s4[q] = fma(M[(int64_t)(u + q) * a.csm], xs[u + q], s4[q]);
        }
        for (; u < cnt; ++u) s4[0] = fma(M[(int64_t)u * a.csm], xs[u], s4[0]);
        sum += (s4[0] + s4[1]) + (s4[2] + s4[3]);
      } else {
        for (int u = 0; u < cnt; ++u) sum = fma(load_as<double>(a.M, i + (l0 + u) * a.csm, a.mdt), xs[u], sum);
      }
    }
    __syncthreads();
  }
  if (i >= a.rows) return;
  if (a.splits == 1) gemv_out(a, i, sum);
  else a.partials[(int64_t)blockIdx.y * a.rows + i] = sum;
}

__global__ void gemv_finish_kernel(const __grid_constant__ GemvArgs a) {
  if (a.skip && *a.skip) return;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.rows) return;
  double sum = 0.0;
  for (int s = 0; s < a.splits; ++s) sum += a.partials[(int64_t)s * a.rows + i];
  gemv_out(a, i, sum);
}

// the reduction index contiguous (csm == 1): one warp per output
__global__ void __launch_bounds__(256) gemv_cols_kernel(const __grid_constant__ GemvArgs a) {
  if (a.skip && *a.skip) return;
  const int lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (i >= a.rows) return;
  double sum = 0.0;
  for (int64_t l = lane; l < a.k; l += 32)
    sum = fma(load_as<double>(a.M, i * a.rsm + l, a.mdt), load_as<double>(a.x, l * a.incx, a.xdt), sum);
  sum = warp_sum(sum);
  if (lane == 0) gemv_out(a, i, sum);
}

// K splits of the row kernel: enough CTAs for 4 per SM, chunks of at least
// 32 columns, at most 64 splits (the partials buffer holds 64 x rows).  A
// short, wide GEMV (512 x 4096, or 8192 x 512) would otherwise run on a few
// dozen CTAs and leave the GPU latency-bound.
int gemv_splits(int64_t rows, int64_t k) {
  int64_t blocks = (rows + 255) / 256;
  int64_t want = (int64_t)device_sm_count() * 4;
  int64_t s = (want + blocks - 1) / blocks;
  int64_t smax = (k + 31) / 32;
  if (s > smax) s = smax;
  if (s > 64) s = 64;
  return s < 1 ? 1 : (int)s;
}

cudaError_t launch_gemv(const GemmArgs& a, cudaStream_t s, int* launches) {
  GemvArgs g;
  memset(&g, 0, sizeof g);
  g.alpha = a.alpha;
  g.beta = a.beta;
  g.scal = 1.0;
  g.skip = a.skip;
  if (a.n == 1) {
    // y (m) = op(A) (m x k) * op(B)(:, 0)
    g.rows = a.m; g.k = a.k;
    g.M = a.A; g.mdt = a.adt;
    if (a.ta) { g.rsm = a.lda; g.csm = 1; } else { g.rsm = 1; g.csm = a.lda; }
    g.x = a.B; g.xdt = a.bdt; g.incx = a.tb ? a.ldb : 1;
    g.y = a.D; g.incy = 1; g.ydt = a.ddt;
    g.c = a.C; g.incc = 1; g.cdt = a.cdt;
    g.rsv = a.rs; g.rs_inc = a.rs_inc; g.rsdt = a.rsdt;
    g.sv = a.cs; g.svdt = a.csdt;
  } else {
    // y^T (n) = op(A)(0, :) (1 x k) * op(B) (k x n)  ->  y_j = sum_l op(B)(l, j) x_l
    g.rows = a.n; g.k = a.k;
    g.M = a.B; g.mdt = a.bdt;
    if (a.tb) { g.rsm = 1; g.csm = a.ldb; } else { g.rsm = a.ldb; g.csm = 1; }
    g.x = a.A; g.xdt = a.adt; g.incx = a.ta ? 1 : a.lda;
    g.y = a.D; g.incy = a.ldd; g.ydt = a.ddt;
    g.c = a.C; g.incc = a.ldc; g.cdt = a.cdt;
    g.rsv = a.cs; g.rs_inc = a.cs_inc; g.rsdt = a.csdt;
    g.sv = a.rs; g.svdt = a.rsdt;
  }
  cudaError_t e;
  if (g.rsm == 1 || g.k == 0) {
    g.splits = (g.k == 0 || a.nosplit) ? 1 : gemv_splits(g.rows, g.k);
    if (g.splits > 1 && (!a.scratch || a.scratch_bytes < (int64_t)g.splits * g.rows * 8)) g.splits = 1;
    g.partials = static_cast<double*>(a.scratch);
    dim3 grid((unsigned)((g.rows + 255) / 256), (unsigned)g.splits);
    gemv_rows_kernel<<<grid, 256, 0, s>>>(g);
    if (launches) ++*launches;
    if (g.splits > 1) {
      gemv_finish_kernel<<<(unsigned)((g.rows + 255) / 256), 256, 0, s>>>(g);
      if (launches) ++*launches;
    }
  } else {
    gemv_cols_kernel<<<(unsigned)((g.rows + 7) / 8), 256, 0, s>>>(g);
    if (launches) ++*launches;
  }
  e = cudaGetLastError();
  return e;
}

// ---------------------------------------------------------------------------
// trace(op(A) op(B)) = sum_{i < min(m,n)} sum_l op(A)(i,l) op(B)(l,i).
// 32 x 32 tiles over (i, l); each operand is loaded along its contiguous
// index and met in shared memory, so both reads are coalesced.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) diagdot_kernel(const __grid_constant__ DotArgs a) {
  __shared__ double As[32][33];
  __shared__ double Bs[32][33];
  const int64_t d = a.m < a.n ? a.m : a.n;
  const int64_t ti = (d + 31) / 32, tl = (a.k + 31) / 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  double sum = 0.0;
  for (int64_t t = blockIdx.x; t < ti * tl; t += gridDim.x) {
    int64_t i0 = (t % ti) * 32, l0 = (t / ti) * 32;
    // op(A)(i, l): contiguous along i when A is not transposed
    for (int r = ty; r < 32; r += 8) {
      int ii = a.ta ? r : tx, ll = a.ta ? tx : r;
      int64_t gi = i0 + ii, gl = l0 + ll;
      double v = 0.0;
      if (gi < d && gl < a.k) v = load_as<double>(a.A, a.ta ? gl + gi * a.lda : gi + gl * a.lda, a.adt);
      As[ii][ll] = v;
      // op(B)(l, i): contiguous along l when B is not transposed
      ll = a.tb ? r : tx;
      ii = a.tb ? tx : r;
      gi = i0 + ii; gl = l0 + ll;
      double w = 0.0;
      if (gi < d && gl < a.k) w = load_as<double>(a.B, a.tb ? gi + gl * a.ldb : gl + gi * a.ldb, a.bdt);
      Bs[ii][ll] = w;
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) sum = fma(As[r][tx], Bs[r][tx], sum);
    __syncthreads();
  }
  reduce_finish(sum, 0.0, a.partials, a.ticket, a.out, nullptr, a.alpha);
}

// the diagonal of op(A) op(B) alone (diagmat of a product, Sec. III (4)):
// a CTA per 32 diagonal elements walks K in 32-wide tiles, read as in the
// trace kernel; each warp keeps the sums of its rows and reduces them across
// the K lanes at the end.  out[i] = alpha * sum_l op(A)(i, l) op(B)(l, i).
// blockIdx.y selects one of gridDim.y K chunks; with more than one chunk
// the sums go to partials[chunk][i] and diagvec_finish adds them in chunk
// order (deterministic)
__global__ void __launch_bounds__(256) diagvec_kernel(const __grid_constant__ DotArgs a) {
  __shared__ double As[32][33];
  __shared__ double Bs[32][33];
  const int64_t d = a.m < a.n ? a.m : a.n;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  const int64_t i0 = (int64_t)blockIdx.x * 32;
  const int64_t kt = (a.k + 31) / 32, per = (kt + gridDim.y - 1) / gridDim.y;
  const int64_t lb = (int64_t)blockIdx.y * per * 32, le = min(a.k, lb + per * 32);
  double sum[4] = {0.0, 0.0, 0.0, 0.0};                 // rows ty, ty + 8, ty + 16, ty + 24
  for (int64_t l0 = lb; l0 < le; l0 += 32) {
    for (int r = ty; r < 32; r += 8) {
      int ii = a.ta ? r : tx, ll = a.ta ? tx : r;
      int64_t gi = i0 + ii, gl = l0 + ll;
      double v = 0.0;
      if (gi < d && gl < le) v = load_as<double>(a.A, a.ta ? gl + gi * a.lda : gi + gl * a.lda, a.adt);
      As[ii][ll] = v;
      ll = a.tb ? r : tx;
      ii = a.tb ? tx : r;
      gi = i0 + ii; gl = l0 + ll;
      double w = 0.0;
      if (gi < d && gl < le) w = load_as<double>(a.B, a.tb ? gi + gl * a.ldb : gl + gi * a.ldb, a.bdt);
      Bs[ii][ll] = w;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) sum[q] = fma(As[ty + 8 * q][tx], Bs[ty + 8 * q][tx], sum[q]);
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const double t = warp_sum(sum[q]);
    const int64_t i = i0 + ty + 8 * q;
    if (tx == 0 && i < d) {
      if (gridDim.y == 1) a.out[i] = a.alpha * t;
      else a.partials[(int64_t)blockIdx.y * d + i] = t;
    }
  }
}

__global__ void diagvec_finish_kernel(const __grid_constant__ DotArgs a, int chunks) {
  const int64_t d = a.m < a.n ? a.m : a.n;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d) return;
  double t = 0.0;
  for (int c = 0; c < chunks; ++c) t += a.partials[(int64_t)c * d + i];
  a.out[i] = a.alpha * t;
}

// ---------------------------------------------------------------------------
// literal-plan copies
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) transpose_kernel(const __grid_constant__ CopyArgs a) {
  __shared__ double t[32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t i0 = (int64_t)blockIdx.x * 32, j0 = (int64_t)blockIdx.y * 32;
  for (int r = ty; r < 32; r += 8) {
    int64_t i = i0 + tx, j = j0 + r;
    if (i < a.m && j < a.n) t[r][tx] = load_as<double>(a.src, i + j * a.lds, a.sdt);
  }
  __syncthreads();
  // dst (n x m): dst[j + i*ldd] = src(i, j)
  for (int r = ty; r < 32; r += 8) {
    int64_t j = j0 + tx, i = i0 + r;
    if (i < a.m && j < a.n) store_as<double>(a.dst, j + i * a.ldd, a.ddt, t[tx][r]);
  }
}

__global__ void __launch_bounds__(256) diag_build_kernel(const __grid_constant__ CopyArgs a) {
  int64_t total = a.m * a.n;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    int64_t j = t / a.m, i = t - j * a.m;
    double v = (i == j) ? load_as<double>(a.src, i * a.inc, a.sdt) : 0.0;
    store_as<double>(a.dst, i + j * a.ldd, a.ddt, v);
  }
}

// D(i, j) = D(j, i) for i < j, in 32 x 32 blocks through shared memory: the
// block of the lower triangle is read along its columns and written
// transposed into the upper triangle (element bits copied unchanged)
template <typename E>
__global__ void __launch_bounds__(256) mirror_lower_kernel(E* D, int64_t n, int64_t ldd) {
  __shared__ E t[32][33];
  const int64_t bi = blockIdx.y, bj = blockIdx.x;   // destination block (upper: bi <= bj)
  if (bi > bj) return;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int q = ty; q < 32; q += 8) {
    const int64_t r = bj * 32 + tx, c = bi * 32 + q;
    if (r < n && c < n) t[q][tx] = D[r + c * ldd];
  }
  __syncthreads();
  for (int q = ty; q < 32; q += 8) {
    const int64_t i = bi * 32 + tx, j = bj * 32 + q;
    if (i < j && j < n) D[i + j * ldd] = t[tx][q];
  }
}

}  // namespace

cudaError_t launch_mirror_lower(void* D, int64_t n, int64_t ldd, int32_t ddt, cudaStream_t s, int* launches) {
  if (n < 2) return cudaSuccess;
  const int64_t T = (n + 31) / 32;
  if (T > 65535) return cudaErrorInvalidConfiguration;
  dim3 grid((unsigned)T, (unsigned)T);
  if (ddt == ARMA_F64) mirror_lower_kernel<unsigned long long><<<grid, 256, 0, s>>>(static_cast<unsigned long long*>(D), n, ldd);
  else if (ddt == ARMA_F32) mirror_lower_kernel<unsigned int><<<grid, 256, 0, s>>>(static_cast<unsigned int*>(D), n, ldd);
  else mirror_lower_kernel<unsigned short><<<grid, 256, 0, s>>>(static_cast<unsigned short*>(D), n, ldd);
  if (launches) ++*launches;
  return cudaGetLastError();
}

// the DFMA kernel's K splits: the model's, or as many as asked for (at most
// one per BK block of K, partial sums within 256 MB)
int simt_split_count(int64_t m, int64_t n, int64_t k, bool nosplit, int32_t req) {
  if (nosplit) return 1;
  if (req <= 0) return simt_splits(m, n, k);
  int s = req;
  const int64_t kb = (k + BK - 1) / BK;
  if (s > kb) s = kb > 0 ? (int)kb : 1;
  while (s > 1 && (double)s * (double)m * (double)n * 8.0 > 256e6) --s;
  return s < 1 ? 1 : s;
}

int64_t gemm_simt_scratch_bytes(int64_t m, int64_t n, int64_t k, int32_t split_req) {
  const int s = simt_split_count(m, n, k, false, split_req);
  return s > 1 ? (int64_t)s * m * n * 8 : 0;
}

// K splits (CTAs per output tile) the product kernels will use for a step,
// and the tiles of its output; host only (152 SMs assumed for the
// matrix-vector rule, whose launch reads the device)
void gemm_step_shape(const GemmStep& g, int* splits, double* tiles) {
  if (g.m == 1 || g.n == 1) {
    const int64_t rows = g.n == 1 ? g.m : g.n;
    const int64_t blocks = (rows + 255) / 256;
    int64_t s = (152 * 4 + blocks - 1) / blocks;
    const int64_t smax = (g.k + 31) / 32;
    if (s > smax) s = smax;
    if (s > 64) s = 64;
    *splits = g.nosplit || s < 1 ? 1 : (int)s;
    *tiles = (double)blocks;
    return;
  }
  const bool tc = g.tier == ARMA_TIER_SPLIT_BF16 || g.tier == ARMA_TIER_BF16;
  if (tc) {
    *splits = gemm_tc_splits(g.m, g.n, g.k, g.tier, g.sym != 0, g.nosplit != 0, g.split_req);
    *tiles = (double)((g.m + 127) / 128) * (double)((g.n + 255) / 256);
  } else {
    *splits = simt_split_count(g.m, g.n, g.k, g.nosplit != 0, g.split_req);
    *tiles = (double)((g.m + BM - 1) / BM) * (double)((g.n + BN - 1) / BN);
  }
}

int64_t gemm_scratch_bytes(const GemmStep& g) {
  if (g.n == 1 || g.m == 1) {
    int64_t rows = g.n == 1 ? g.m : g.n;
    return 64 * rows * 8;
  }
  const int64_t tc = gemm_tc_scratch_bytes(g.m, g.n, g.k, g.tier, g.split_req);
  const int64_t simt = gemm_simt_scratch_bytes(g.m, g.n, g.k, g.split_req);
  int64_t b = tc > simt ? tc : simt;
  if (g.tier == ARMA_TIER_F64_SLICED) {
    const int64_t oz = gemm_ozaki_scratch_bytes(g.m, g.n, g.k);
    if (oz > b) b = oz;
  }
  return b;
}

// sym 1: a symmetric product (no beta*C), mirrored; sym 2: only the lower
// triangle of D is computed (with beta*C), the upper triangle is untouched
int gemm_sym_valid(const GemmArgs& a) {
  if (!(a.sym == 1 || a.sym == 2) || a.m != a.n || a.A != a.B || a.lda != a.ldb || a.adt != a.bdt ||
      a.ta == a.tb || a.rs || a.cs)
    return 0;
  if (a.sym == 1 && a.C && a.beta != 0.0) return 0;
  return a.sym;
}

cudaError_t launch_gemm(const GemmArgs& a0, cudaStream_t s, int* launches) {
  if (a0.m == 0 || a0.n == 0) return cudaSuccess;
  if ((a0.n == 1 || a0.m == 1) && !a0.no_gemv) return launch_gemv(a0, s, launches);
  GemmArgs a = a0;
  a.sym = gemm_sym_valid(a0);   // anything else is a general product
  if (a.tier == ARMA_TIER_F64_SLICED && gemm_ozaki_supported(a)) return launch_gemm_ozaki(a, s, launches);
  if (a.tier != ARMA_TIER_F64 && gemm_tc_supported(a)) return launch_gemm_tc(a, s, launches);
  int splits = simt_split_count(a.m, a.n, a.k, a.nosplit != 0, a.split_req);
  if (splits > 1 && (!a.scratch || a.scratch_bytes < (int64_t)splits * a.m * a.n * 8)) splits = 1;
  const int64_t tm = (a.m + BM - 1) / BM, tn = (a.n + BN - 1) / BN;
  dim3 grid((unsigned)(a.sym ? tm * (tm + 1) / 2 : tm), (unsigned)(a.sym ? 1 : tn), (unsigned)splits);
  if (grid.y > 65535) return cudaErrorInvalidConfiguration;
  if (a.tier == ARMA_TIER_F64 || a.adt == ARMA_F64 || a.bdt == ARMA_F64)
    gemm_simt_kernel<double><<<grid, 256, 0, s>>>(a);
  else
    gemm_simt_kernel<float><<<grid, 256, 0, s>>>(a);
  if (launches) ++*launches;
  if (splits > 1) {
    const int64_t total = a.m * a.n;
    int64_t blocks = (total + 255) / 256, cap = (int64_t)device_sm_count() * 8;
    gemm_simt_combine_kernel<<<(unsigned)(blocks < cap ? blocks : cap), 256, 0, s>>>(a, splits);
    if (launches) ++*launches;
  }
  if (a.sym == 1) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_mirror_lower(a.D, a.n, a.ldd, a.ddt, s, launches);
  }
  return cudaGetLastError();
}

cudaError_t launch_diagdot(const DotArgs& a, cudaStream_t s, int* launches) {
  int64_t d = a.m < a.n ? a.m : a.n;
  int64_t tiles = ((d + 31) / 32) * ((a.k + 31) / 32);
  int64_t cap = (int64_t)device_sm_count() * 8;
  if (cap > kMaxRedBlocks) cap = kMaxRedBlocks;
  int grid = (int)(tiles < 1 ? 1 : tiles > cap ? cap : tiles);
  if (a.per_diag) {
    if (d == 0) return cudaSuccess;
    // K chunks: about 4 CTAs per SM, each chunk at least 128 of K, at most
    // DIAGVEC_MAX_CHUNKS (the partials buffer holds that many rows of d)
    const int64_t rb = (d + 31) / 32;
    int64_t chunks = ((int64_t)device_sm_count() * 4 + rb - 1) / rb;
    const int64_t cmax = (a.k + 127) / 128;
    if (chunks > cmax) chunks = cmax;
    if (chunks > DIAGVEC_MAX_CHUNKS) chunks = DIAGVEC_MAX_CHUNKS;
    if (chunks < 1 || !a.partials) chunks = 1;
    diagvec_kernel<<<dim3((unsigned)rb, (unsigned)chunks), 256, 0, s>>>(a);
    if (chunks > 1) {
      if (launches) ++*launches;
      diagvec_finish_kernel<<<(unsigned)((d + 255) / 256), 256, 0, s>>>(a, (int)chunks);
    }
  } else {
    diagdot_kernel<<<grid, 256, 0, s>>>(a);
  }
  if (launches) ++*launches;
  return cudaGetLastError();
}

cudaError_t launch_transpose(const CopyArgs& a, cudaStream_t s, int* launches) {
  if (a.m == 0 || a.n == 0) return cudaSuccess;
  dim3 grid((unsigned)((a.m + 31) / 32), (unsigned)((a.n + 31) / 32));
  transpose_kernel<<<grid, 256, 0, s>>>(a);
  if (launches) ++*launches;
  return cudaGetLastError();
}

cudaError_t launch_diag_build(const CopyArgs& a, cudaStream_t s, int* launches) {
  int64_t total = a.m * a.n;
  if (total == 0) return cudaSuccess;
  int64_t need = (total + 255) / 256, cap = (int64_t)device_sm_count() * 8;
  diag_build_kernel<<<(unsigned)(need < cap ? need : cap), 256, 0, s>>>(a);
  if (launches) ++*launches;
  return cudaGetLastError();
}

}  // namespace arma
