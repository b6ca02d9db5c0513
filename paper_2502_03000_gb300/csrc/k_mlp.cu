// The learned cost model: a 3-layer perceptron (FP32) that predicts the log
// run time of a candidate plan from its features, with hand-written
// inference, gradient and Adam kernels.  The paper plans with fixed rules
// (Sec. II: compile-time patterns and a greedy chain rule); this network is
// this library's addition for ranking candidate plans, trained on timings
// the library records.
//
// Parameters, packed: W1 (H x F, row-major), b1 (H), W2 (H x H), b2 (H),
// W3 (H), b3 (1).  Loss: mean squared error over the batch.
//
//   forward   one thread per sample, all weights in shared memory
//   grad      pass 1: one thread per sample stores h1, h2 and the backward
//             signals; pass 2: one thread per parameter sums its gradient
//             over the samples in sample order (deterministic, no atomics)
//   adam      one thread per parameter
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace arma {
namespace mlp {

constexpr int MAXH = 128;
constexpr int MAXF = 64;

__host__ __device__ inline int64_t param_count(int F, int H) {
  return (int64_t)H * F + H + (int64_t)H * H + H + H + 1;
}

struct Offs {
  int64_t W1, b1, W2, b2, W3, b3;
};
__host__ __device__ inline Offs offs(int F, int H) {
  Offs o;
  o.W1 = 0;
  o.b1 = o.W1 + (int64_t)H * F;
  o.W2 = o.b1 + H;
  o.b2 = o.W2 + (int64_t)H * H;
  o.W3 = o.b2 + H;
  o.b3 = o.W3 + H;
  return o;
}

// per-sample forward; if act != null also stores z1, z2 (pre-activations)
__global__ void forward_kernel(const float* __restrict__ P, int F, int H, const float* __restrict__ X, int N,
                               float* __restrict__ Y, float* __restrict__ Z1, float* __restrict__ Z2) {
  extern __shared__ float sp[];
  const int64_t np = param_count(F, H);
  for (int64_t i = threadIdx.x; i < np; i += blockDim.x) sp[i] = P[i];
  __syncthreads();
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const Offs o = offs(F, H);
  float x[MAXF];
  for (int f = 0; f < F; ++f) x[f] = X[(int64_t)n * F + f];
  float h1[MAXH];
  for (int i = 0; i < H; ++i) {
    float z = sp[o.b1 + i];
    for (int f = 0; f < F; ++f) z = fmaf(sp[o.W1 + (int64_t)i * F + f], x[f], z);
    if (Z1) Z1[(int64_t)n * H + i] = z;
    h1[i] = z > 0.f ? z : 0.f;
  }
  float y = sp[o.b3];
  for (int i = 0; i < H; ++i) {
    float z = sp[o.b2 + i];
    for (int j = 0; j < H; ++j) z = fmaf(sp[o.W2 + (int64_t)i * H + j], h1[j], z);
    if (Z2) Z2[(int64_t)n * H + i] = z;
    y = fmaf(sp[o.W3 + i], z > 0.f ? z : 0.f, y);
  }
  Y[n] = y;
}

// backward signals per sample: dy, dz2 = dy W3 * relu'(z2), dz1 = W2^T dz2 * relu'(z1)
__global__ void backward_signals_kernel(const float* __restrict__ P, int F, int H, int N,
                                        const float* __restrict__ Y, const float* __restrict__ T,
                                        const float* __restrict__ Z1, const float* __restrict__ Z2,
                                        float* __restrict__ DY, float* __restrict__ DZ1, float* __restrict__ DZ2) {
  extern __shared__ float sp[];
  const int64_t np = param_count(F, H);
  for (int64_t i = threadIdx.x; i < np; i += blockDim.x) sp[i] = P[i];
  __syncthreads();
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const Offs o = offs(F, H);
  const float dy = 2.f * (Y[n] - T[n]) / (float)N;
  DY[n] = dy;
  float dz2[MAXH];
  for (int i = 0; i < H; ++i) {
    const float z = Z2[(int64_t)n * H + i];
    dz2[i] = z > 0.f ? dy * sp[o.W3 + i] : 0.f;
    DZ2[(int64_t)n * H + i] = dz2[i];
  }
  for (int j = 0; j < H; ++j) {
    const float z = Z1[(int64_t)n * H + j];
    float s = 0.f;
    for (int i = 0; i < H; ++i) s = fmaf(sp[o.W2 + (int64_t)i * H + j], dz2[i], s);
    DZ1[(int64_t)n * H + j] = z > 0.f ? s : 0.f;
  }
}

// one thread per parameter: its gradient summed over samples in order
__global__ void param_grad_kernel(int F, int H, int N, const float* __restrict__ X,
                                  const float* __restrict__ Z1, const float* __restrict__ Z2,
                                  const float* __restrict__ DY, const float* __restrict__ DZ1,
                                  const float* __restrict__ DZ2, float* __restrict__ G) {
  const int64_t np = param_count(F, H);
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  const Offs o = offs(F, H);
  float s = 0.f;
  if (p < o.b1) {                       // W1[i][f] = sum_n dz1[n][i] x[n][f]
    const int64_t i = p / F, f = p % F;
    for (int n = 0; n < N; ++n) s = fmaf(DZ1[(int64_t)n * H + i], X[(int64_t)n * F + f], s);
  } else if (p < o.W2) {                // b1[i]
    const int64_t i = p - o.b1;
    for (int n = 0; n < N; ++n) s += DZ1[(int64_t)n * H + i];
  } else if (p < o.b2) {                // W2[i][j] = sum_n dz2[n][i] h1[n][j]
    const int64_t q = p - o.W2, i = q / H, j = q % H;
    for (int n = 0; n < N; ++n) {
      const float z = Z1[(int64_t)n * H + j];
      s = fmaf(DZ2[(int64_t)n * H + i], z > 0.f ? z : 0.f, s);
    }
  } else if (p < o.W3) {                // b2[i]
    const int64_t i = p - o.b2;
    for (int n = 0; n < N; ++n) s += DZ2[(int64_t)n * H + i];
  } else if (p < o.b3) {                // W3[j] = sum_n dy[n] h2[n][j]
    const int64_t j = p - o.W3;
    for (int n = 0; n < N; ++n) {
      const float z = Z2[(int64_t)n * H + j];
      s = fmaf(DY[n], z > 0.f ? z : 0.f, s);
    }
  } else {                              // b3
    for (int n = 0; n < N; ++n) s += DY[n];
  }
  G[p] = s;
}

__global__ void adam_kernel(float* P, const float* G, float* M, float* V, int64_t np, float lr, float b1,
                            float b2, float eps, float c1, float c2) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  const float g = G[p];
  const float m = b1 * M[p] + (1.f - b1) * g;
  const float v = b2 * V[p] + (1.f - b2) * g * g;
  M[p] = m;
  V[p] = v;
  P[p] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
}

}  // namespace mlp
}  // namespace arma

using namespace arma;

extern "C" {

int64_t arma_gpu_mlp_param_count(int32_t features, int32_t hidden) {
  return mlp::param_count(features, hidden);
}

size_t arma_gpu_mlp_workspace(int32_t features, int32_t hidden, int32_t n) {
  (void)features;
  // Y, DY (n each) and Z1, Z2, DZ1, DZ2 (n x hidden each), FP32
  return (size_t)n * 4 * (2 + 4 * (size_t)hidden) + 1024;
}

static bool mlp_dims_ok(int32_t F, int32_t H, int32_t N) {
  return F >= 1 && F <= mlp::MAXF && H >= 1 && H <= mlp::MAXH && N >= 0;
}

static bool mlp_smem(size_t smem) {
  return cudaFuncSetAttribute(mlp::forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) ==
             cudaSuccess &&
         cudaFuncSetAttribute(mlp::backward_signals_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem) == cudaSuccess;
}

arma_status arma_gpu_mlp_forward(const float* params, int32_t features, int32_t hidden, const float* x,
                                 int32_t n, float* y, void* stream) {
  if (!params || (!x && n > 0) || (!y && n > 0) || !mlp_dims_ok(features, hidden, n)) return ARMA_ERR_INVALID;
  if (n == 0) return ARMA_OK;
  const size_t smem = (size_t)mlp::param_count(features, hidden) * 4;
  if (!mlp_smem(smem)) return ARMA_ERR_CUDA;
  mlp::forward_kernel<<<(n + 127) / 128, 128, smem, static_cast<cudaStream_t>(stream)>>>(
      params, features, hidden, x, n, y, nullptr, nullptr);
  return cudaGetLastError() == cudaSuccess ? ARMA_OK : ARMA_ERR_CUDA;
}

arma_status arma_gpu_mlp_grad(const float* params, int32_t features, int32_t hidden, const float* x,
                              const float* target, int32_t n, float* grad, float* y_out, void* workspace,
                              size_t workspace_bytes, void* stream) {
  if (!params || !x || !target || !grad || !mlp_dims_ok(features, hidden, n) || n < 1) return ARMA_ERR_INVALID;
  if (!workspace || workspace_bytes < arma_gpu_mlp_workspace(features, hidden, n)) return ARMA_ERR_WORKSPACE;
  const int F = features, H = hidden;
  float* w = static_cast<float*>(workspace);
  float* Y = y_out ? y_out : w;
  float* DY = w + n;
  float* Z1 = DY + n;
  float* Z2 = Z1 + (size_t)n * H;
  float* DZ1 = Z2 + (size_t)n * H;
  float* DZ2 = DZ1 + (size_t)n * H;
  const size_t smem = (size_t)mlp::param_count(F, H) * 4;
  if (!mlp_smem(smem)) return ARMA_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const unsigned nb = (unsigned)((n + 127) / 128);
  mlp::forward_kernel<<<nb, 128, smem, s>>>(params, F, H, x, n, Y, Z1, Z2);
  mlp::backward_signals_kernel<<<nb, 128, smem, s>>>(params, F, H, n, Y, target, Z1, Z2, DY, DZ1, DZ2);
  const int64_t np = mlp::param_count(F, H);
  mlp::param_grad_kernel<<<(unsigned)((np + 127) / 128), 128, 0, s>>>(F, H, n, x, Z1, Z2, DY, DZ1, DZ2, grad);
  return cudaGetLastError() == cudaSuccess ? ARMA_OK : ARMA_ERR_CUDA;
}

arma_status arma_gpu_mlp_adam(float* params, const float* grad, float* m, float* v, int64_t count,
                              int32_t step, float lr, float beta1, float beta2, float eps, void* stream) {
  if (!params || !grad || !m || !v || count < 1 || step < 1) return ARMA_ERR_INVALID;
  const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
  mlp::adam_kernel<<<(unsigned)((count + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      params, grad, m, v, count, lr, beta1, beta2, eps, c1, c2);
  return cudaGetLastError() == cudaSuccess ? ARMA_OK : ARMA_ERR_CUDA;
}

}  // extern "C"
