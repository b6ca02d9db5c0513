// Grouped evaluation of many independent small products of uneven sizes in
// one persistent launch: for every problem g,
//     D_g = alpha * op(A_g) * op(B_g) + beta * C_g,   t_g = trace(op(A_g) op(B_g))
// (the batched form of the paper's folded product and diagonal-only trace,
// Sec. II xGEMM paragraph, Sec. III (5)).  A host-built tile list spans all
// problems; each CTA walks it with a fixed stride, so there is one launch for
// the whole batch (plus a small trace finalisation) instead of one or more
// launches per problem, and the pair of launches can be captured in a CUDA
// graph.  Per problem the tile shape is 32 x 32 or 64 x 64, picked on the host
// by a padded-work cost model.  Accumulation is FP32 (BF16 inputs are
// widened exactly); traces are accumulated per diagonal tile in FP64 and
// summed in a fixed order.
#include "common.cuh"
#include "grouped.h"

namespace arma {
namespace {

template <int T>   // tile edge: 32 or 64; 256 threads, (T/16)^2 outputs each
__device__ __forceinline__ void grouped_tile(const GroupedProblem& pb, int tm, int tn, const GroupedArgs& g,
                                             float (&As)[16][65], float (&Bs)[16][65], double* diag_out) {
  constexpr int R = T / 16;   // outputs per thread per dimension
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t i0 = (int64_t)tm * T, j0 = (int64_t)tn * T;
  float acc[R][R];
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int c = 0; c < R; ++c) acc[r][c] = 0.f;
  for (int64_t l0 = 0; l0 < pb.k; l0 += 16) {
    // op(A) tile T x 16 and op(B) tile 16 x T, loaded along the contiguous index
    for (int e = tid; e < T * 16; e += 256) {
      int ii, ll;
      if (!g.ta) { ii = e % T; ll = e / T; } else { ll = e & 15; ii = e >> 4; }
      const int64_t gi = i0 + ii, gl = l0 + ll;
      float v = 0.f;
      if (gi < pb.m && gl < pb.k) v = load_as<float>(pb.A, g.ta ? gl + gi * pb.lda : gi + gl * pb.lda, g.abdt);
      As[ll][ii] = v;
      int jj;
      if (!g.tb) { ll = e & 15; jj = e >> 4; } else { jj = e % T; ll = e / T; }
      const int64_t gj = j0 + jj;
      const int64_t gl2 = l0 + ll;
      float w = 0.f;
      if (gl2 < pb.k && gj < pb.n) w = load_as<float>(pb.B, g.tb ? gj + gl2 * pb.ldb : gl2 + gj * pb.ldb, g.abdt);
      Bs[ll][jj] = w;
    }
    __syncthreads();
#pragma unroll
    for (int l = 0; l < 16; ++l) {
      float av[R], bv[R];
#pragma unroll
      for (int r = 0; r < R; ++r) av[r] = As[l][tx + 16 * r];
#pragma unroll
      for (int c = 0; c < R; ++c) bv[c] = Bs[l][ty + 16 * c];
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int c = 0; c < R; ++c) acc[r][c] = fmaf(av[r], bv[c], acc[r][c]);
    }
    __syncthreads();
  }
  double dsum = 0.0;
#pragma unroll
  for (int c = 0; c < R; ++c) {
    const int64_t j = j0 + ty + 16 * c;
    if (j >= pb.n) continue;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int64_t i = i0 + tx + 16 * r;
      if (i >= pb.m) continue;
      if (i == j) dsum += (double)acc[r][c];
      float v = g.alpha_f * acc[r][c];
      if (pb.C && g.beta != 0.0) v = fmaf(g.beta_f, load_as<float>(pb.C, i + j * pb.ldc, g.cdt), v);
      store_as<float>(pb.D, i + j * pb.ldd, g.ddt, v);
    }
  }
  if (diag_out) {   // diagonal tile: this tile's share of the trace
    double q = 0.0;
    block_sum2(dsum, q);
    if (threadIdx.x == 0) *diag_out = dsum;
  }
}

__global__ void __launch_bounds__(256) grouped_kernel(const __grid_constant__ GroupedArgs g) {
  __shared__ float As[16][65];
  __shared__ float Bs[16][65];
  const GroupedProblem* probs = g.probs;
  for (int64_t t = blockIdx.x; t < g.tiles; t += gridDim.x) {
    const uint32_t code = g.tile_code[t];
    const int32_t p = g.tile_prob[t];
    const GroupedProblem pb = probs[p];
    const int tm = (int)(code >> 16), tn = (int)(code & 0xFFFFu);
    double* dout = (g.trace_partials && tm == tn) ? g.trace_partials + t : nullptr;
    if (pb.tile == 32) grouped_tile<32>(pb, tm, tn, g, As, Bs, dout);
    else grouped_tile<64>(pb, tm, tn, g, As, Bs, dout);
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
  for (int64_t q = 0; q * pb.tile < d; ++q) s += g.trace_partials[pb.first_tile + q * ntn + q];
  *pb.trace = s;
}

}  // namespace

cudaError_t launch_grouped(const GroupedArgs& g, cudaStream_t s, int* launches) {
  if (g.tiles == 0) return cudaSuccess;
  const int sms = device_sm_count();
  int64_t grid = (int64_t)sms * 8;
  if (grid > g.tiles) grid = g.tiles;
  grouped_kernel<<<(unsigned)grid, 256, 0, s>>>(g);
  if (launches) ++*launches;
  if (g.trace_partials) {
    grouped_trace_kernel<<<(unsigned)((g.count + 255) / 256), 256, 0, s>>>(g);
    if (launches) ++*launches;
  }
  return cudaGetLastError();
}

}  // namespace arma
