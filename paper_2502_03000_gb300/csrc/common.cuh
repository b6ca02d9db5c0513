// Device helpers shared by the kernels: typed element access and the
// deterministic two-stage FP64 reduction.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace arma {

template <typename CT>
__device__ __forceinline__ CT load_as(const void* p, int64_t idx, int dt) {
  if (dt == ARMA_F64) return (CT)(static_cast<const double*>(p)[idx]);
  if (dt == ARMA_F32) return (CT)(static_cast<const float*>(p)[idx]);
  return (CT)__bfloat162float(static_cast<const __nv_bfloat16*>(p)[idx]);
}

template <typename CT>
__device__ __forceinline__ void store_as(void* p, int64_t idx, int dt, CT v) {
  if (dt == ARMA_F64) static_cast<double*>(p)[idx] = (double)v;
  else if (dt == ARMA_F32) static_cast<float*>(p)[idx] = (float)v;
  else static_cast<__nv_bfloat16*>(p)[idx] = __float2bfloat16_rn((float)v);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  return v;
}

// Sum (s, q) over the block in a fixed order; result valid in thread 0.
__device__ __forceinline__ void block_sum2(double& s, double& q) {
  __shared__ double sh_s[32], sh_q[32];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  s = warp_sum(s);
  q = warp_sum(q);
  __syncthreads();
  if (lane == 0) { sh_s[wid] = s; sh_q[wid] = q; }
  __syncthreads();
  if (wid == 0) {
    s = lane < nw ? sh_s[lane] : 0.0;
    q = lane < nw ? sh_q[lane] : 0.0;
    s = warp_sum(s);
    q = warp_sum(q);
  }
}

// Stage 1 writes this block's (s, q) to partials[2*block]; the last block
// to arrive (ticket) adds all partials in block order, so the result does
// not depend on scheduling.  Writes alpha*sum to *sum_out and sqrt(sumsq)
// to *norm_out (either may be null), then re-arms the ticket.
__device__ __forceinline__ void reduce_finish(double s, double q, double* partials,
                                              unsigned int* ticket, double* sum_out,
                                              double* norm_out, double alpha) {
  __shared__ unsigned int sh_last;
  block_sum2(s, q);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = s;
    partials[2 * blockIdx.x + 1] = q;
    __threadfence();
    unsigned int t = atomicAdd(ticket, 1u);
    sh_last = (t == gridDim.x - 1) ? 1u : 0u;
  }
  __syncthreads();
  if (!sh_last) return;
  __threadfence();
  double ts = 0.0, tq = 0.0;
  for (unsigned int b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
    ts += __ldcg(partials + 2 * b);
    tq += __ldcg(partials + 2 * b + 1);
  }
  block_sum2(ts, tq);
  if (threadIdx.x == 0) {
    if (sum_out) *sum_out = alpha * ts;
    if (norm_out) *norm_out = sqrt(tq);
    *ticket = 0u;
  }
}

int device_sm_count();

}  // namespace arma
