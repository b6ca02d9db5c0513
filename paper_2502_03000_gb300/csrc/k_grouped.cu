// Grouped evaluation of many independent small products of uneven sizes in
// one persistent launch: for every problem g,
//     D_g = alpha * op(A_g) * op(B_g) + beta * C_g,   t_g = trace(op(A_g) op(B_g))
// (the batched form of the paper's folded product and diagonal-only trace,
// Sec. II xGEMM paragraph, Sec. III (5)).  A host-built tile list spans all
// problems, ordered by decreasing work; the CTAs of one resident wave take
// tiles from a shared counter (longest first), so there is one launch for the
// whole batch (plus a small trace finalisation) instead of one or more
// launches per problem, and the pair of launches can be captured in a CUDA
// graph.  Per problem the tile shape is 32 x 32 or 64 x 64, picked on the host
// by a padded-work cost model.  Accumulation is FP32 (BF16 inputs are
// widened exactly); traces are accumulated per diagonal tile in FP64 and
// summed in a fixed order.
#include "common.cuh"
#include "grouped.h"

namespace arma {
namespace {

constexpr int GBK = 32;   // K per shared-memory stage

__device__ __forceinline__ float widen(float x) { return x; }
__device__ __forceinline__ float widen(__nv_bfloat16 x) { return __bfloat162float(x); }

// One output tile.  AT is the storage type of A and B (FP32 or BF16, widened
// exactly); the element type is a template parameter so that no load carries
// conversion code for the other types.  The next K block is fetched into
// registers while the current one is multiplied out of shared memory.
constexpr int SROW = 68;  // shared row stride in floats: 16-byte aligned rows for vector reads

// thread (tx, ty) owns rows R tx .. R tx + R - 1 and columns R ty .. R ty + R - 1
// of the tile, read from shared memory as R-wide vectors
template <int R>
__device__ __forceinline__ void ldsR(const float* p, float (&v)[R]) {
  if constexpr (R == 4) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  } else {
    const float2 t = *reinterpret_cast<const float2*>(p);
    v[0] = t.x; v[1] = t.y;
  }
}

template <typename AT, int T>   // tile edge: 32 or 64; 256 threads, (T/16)^2 outputs each
__device__ __forceinline__ void grouped_tile(const GroupedProblem& pb, int tm, int tn, const GroupedArgs& g,
                                             float (&As)[GBK][SROW], float (&Bs)[GBK][SROW], double* diag_out) {
  constexpr int R = T / 16;             // outputs per thread per dimension
  constexpr int NL = T * GBK / 256;     // elements per thread per operand and K block
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t i0 = (int64_t)tm * T, j0 = (int64_t)tn * T;
  const AT* A = static_cast<const AT*>(pb.A);
  const AT* B = static_cast<const AT*>(pb.B);
  float ra[NL], rb[NL];
  // element e of this thread: op(A)(ii, ll) and op(B)(ll, jj), each read
  // along its contiguous index
  auto a_at = [&](int e, int& ii, int& ll) {
    const int x = tid + 256 * e;
    if (g.ta) { ll = x % GBK; ii = x / GBK; } else { ii = x % T; ll = x / T; }
  };
  auto b_at = [&](int e, int& ll, int& jj) {
    const int x = tid + 256 * e;
    if (!g.tb) { ll = x % GBK; jj = x / GBK; } else { jj = x % T; ll = x / T; }
  };
  auto fetch = [&](int64_t l0) {
#pragma unroll
    for (int e = 0; e < NL; ++e) {
      int ii, ll, jj, lb;
      a_at(e, ii, ll);
      const int64_t gi = i0 + ii, gl = l0 + ll;
      ra[e] = (gi < pb.m && gl < pb.k) ? widen(A[g.ta ? gl + gi * pb.lda : gi + gl * pb.lda]) : 0.f;
      b_at(e, lb, jj);
      const int64_t gj = j0 + jj, gl2 = l0 + lb;
      rb[e] = (gl2 < pb.k && gj < pb.n) ? widen(B[g.tb ? gj + gl2 * pb.ldb : gl2 + gj * pb.ldb]) : 0.f;
    }
  };
  float acc[R][R];
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int c = 0; c < R; ++c) acc[r][c] = 0.f;
  fetch(0);
  for (int64_t l0 = 0; l0 < pb.k; l0 += GBK) {
#pragma unroll
    for (int e = 0; e < NL; ++e) {
      int ii, ll, jj, lb;
      a_at(e, ii, ll);
      As[ll][ii] = ra[e];
      b_at(e, lb, jj);
      Bs[lb][jj] = rb[e];
    }
    __syncthreads();
    if (l0 + GBK < pb.k) fetch(l0 + GBK);
#pragma unroll 8
    for (int l = 0; l < GBK; ++l) {
      float av[R], bv[R];
      ldsR<R>(&As[l][R * tx], av);
      ldsR<R>(&Bs[l][R * ty], bv);
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int c = 0; c < R; ++c) acc[r][c] = fmaf(av[r], bv[c], acc[r][c]);
    }
    __syncthreads();
  }
  // epilogue: D = alpha * acc + beta * C (D is FP32); C read per its type
  double dsum = 0.0;
  const bool has_c = pb.C && g.beta != 0.0;
  float* D = static_cast<float*>(pb.D);
  // the storage type of C is uniform: one branch per tile, not per element
  auto store = [&](auto load_c) {
#pragma unroll
    for (int c = 0; c < R; ++c) {
      const int64_t j = j0 + R * ty + c;
      if (j >= pb.n) continue;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int64_t i = i0 + R * tx + r;
        if (i >= pb.m) continue;
        if (i == j) dsum += (double)acc[r][c];
        float v = g.alpha_f * acc[r][c];
        if (has_c) v = fmaf(g.beta_f, load_c(i + j * pb.ldc), v);
        D[i + j * pb.ldd] = v;
      }
    }
  };
  if (!has_c || g.cdt == ARMA_F32) {
    const float* C = static_cast<const float*>(pb.C);
    store([&](int64_t x) { return C[x]; });
  } else if (g.cdt == ARMA_BF16) {
    const __nv_bfloat16* C = static_cast<const __nv_bfloat16*>(pb.C);
    store([&](int64_t x) { return __bfloat162float(C[x]); });
  } else {
    const double* C = static_cast<const double*>(pb.C);
    store([&](int64_t x) { return (float)C[x]; });
  }
  if (diag_out) {   // diagonal tile: this tile's share of the trace (slot 0 of its kTraceSlots)
    double q = 0.0;
    block_sum2(dsum, q);
    if (threadIdx.x == 0) {
      diag_out[0] = dsum;
      for (int k = 1; k < kTraceSlots; ++k) diag_out[k] = 0.0;
    }
  }
}

// the next tile of the work list for this CTA (thread 0 takes it from the
// shared counter; the list is ordered longest first)
__device__ __forceinline__ int64_t next_tile(const GroupedArgs& g, int* slot) {
  __syncthreads();
  if (threadIdx.x == 0) *slot = (int)atomicAdd(g.next_tile, 1u);
  __syncthreads();
  return *slot;
}

template <typename AT>
__global__ void __launch_bounds__(256, 2) grouped_kernel(const __grid_constant__ GroupedArgs g) {
  __shared__ __align__(16) float As[GBK][SROW];
  __shared__ __align__(16) float Bs[GBK][SROW];
  __shared__ int s_next;
  const GroupedProblem* probs = g.probs;
  for (int64_t i = next_tile(g, &s_next); i < g.tiles; i = next_tile(g, &s_next)) {
    const int64_t t = g.tile_order[i];
    const uint32_t code = g.tile_code[t];
    const int32_t p = g.tile_prob[t];
    const GroupedProblem pb = probs[p];
    const int tm = (int)(code >> 16), tn = (int)(code & 0xFFFFu);
    double* dout = (g.trace_partials && tm == tn) ? g.trace_partials + kTraceSlots * t : nullptr;
    if (pb.tile == 32) grouped_tile<AT, 32>(pb, tm, tn, g, As, Bs, dout);
    else grouped_tile<AT, 64>(pb, tm, tn, g, As, Bs, dout);
  }
}

// t_g = sum over the diagonal tiles of problem g, in tile order
__global__ void grouped_trace_kernel(const __grid_constant__ GroupedArgs g) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= g.count) return;
  const GroupedProblem pb = g.probs[p];
  if (!pb.trace) return;
  const int64_t d = pb.m < pb.n ? pb.m : pb.n;
  const int64_t ntn = (pb.n + pb.tile - 1) / pb.tile;
  double s = 0.0;
  for (int64_t q = 0; q * pb.tile < d; ++q) {
    const double* part = g.trace_partials + kTraceSlots * (pb.first_tile + q * ntn + q);
    double tile = 0.0;
    for (int k = 0; k < kTraceSlots; ++k) tile += part[k];
    s += tile;
  }
  *pb.trace = s;
}

}  // namespace

cudaError_t launch_grouped(const GroupedArgs& g, cudaStream_t s, int* launches) {
  if (g.tiles == 0) return cudaSuccess;
  if (g.tc) {
    cudaError_t e = launch_grouped_tc(g, s, launches);
    if (e != cudaSuccess || !g.trace_partials) return e;
    grouped_trace_kernel<<<(unsigned)((g.count + 255) / 256), 256, 0, s>>>(g);
    if (launches) ++*launches;
    return cudaGetLastError();
  }
  // one resident wave (2 CTAs per SM by the register bound); CTAs take
  // tiles from the shared counter until the list is done
  const int sms = device_sm_count();
  int64_t grid = (int64_t)sms * 2;
  if (grid > g.tiles) grid = g.tiles;
  if (g.abdt == ARMA_BF16) grouped_kernel<__nv_bfloat16><<<(unsigned)grid, 256, 0, s>>>(g);
  else if (g.abdt == ARMA_F32) grouped_kernel<float><<<(unsigned)grid, 256, 0, s>>>(g);
  else return cudaErrorInvalidValue;
  if (launches) ++*launches;
  if (g.trace_partials) {
    grouped_trace_kernel<<<(unsigned)((g.count + 255) / 256), 256, 0, s>>>(g);
    if (launches) ++*launches;
  }
  return cudaGetLastError();
}

}  // namespace arma
