// Evaluation of fused elementwise plans without a caller workspace.
//
// Some callers cannot allocate device memory at all: a host application
// that hands a plug-in nothing but raw input and output pointers, code that
// runs inside another framework's memory pool where outside allocations are
// forbidden, or a latency-critical loop that cannot afford cudaMalloc's
// implicit device synchronisation.  For them, plans made only of fused
// elementwise passes (the kernel that keeps its reduction partials and
// ticket counters in scratch memory) can run with the scratch held in a
// fixed-size array in this library's own device memory instead.
//
// The array is a file-scope __device__ variable: every GPU that loads the
// library holds ARMA_STATIC_SCRATCH_BYTES of it until the process exits.
// Host code cannot use the variable's name as a device address, so the
// first call on each device looks the address up with cudaGetSymbolAddress
// (with that device current) and caches it; that first call should come
// before any stream capture.  All calls share the one array and it keeps
// the last call's contents; the evaluation clears the part that must start
// at zero (status word and ticket counters) before it launches.  Calls
// whose kernels overlap on the GPU race on the array.
#include <cuda_runtime.h>

#include <mutex>

#include "internal.h"

namespace {

static __device__ __align__(256) unsigned char g_static_scratch[ARMA_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {nullptr};

arma_status static_scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return ARMA_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p) return ARMA_ERR_CUDA;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return ARMA_OK;
}

}  // namespace

extern "C" arma_status arma_gpu_eval_fused_static(const arma_plan* plan, const void* const* in_ptrs,
                                                  void* const* out_ptrs, void* stream) {
  if (!plan) return ARMA_ERR_INVALID;
  for (const arma::Step& st : plan->steps)
    if (st.kind != arma::ST_EW) return ARMA_ERR_UNSUPPORTED;
  if (plan->ws_bytes > ARMA_STATIC_SCRATCH_BYTES) return ARMA_ERR_WORKSPACE;
  void* scratch = nullptr;
  arma_status s = static_scratch_address(&scratch);
  if (s != ARMA_OK) return s;
  return arma_gpu_eval(plan, in_ptrs, out_ptrs, scratch, ARMA_STATIC_SCRATCH_BYTES, stream);
}
