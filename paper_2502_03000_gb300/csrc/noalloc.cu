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
// Host code cannot use the variable's name as a device address, so each
// call made outside stream capture looks the address up with
// cudaGetSymbolAddress (with the device current) and records it; a call
// under capture uses the recorded address, so the first call on a device
// should come before any stream capture.  All calls share the one array and it keeps
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

// The array's device address on the current device.  Outside stream
// capture it is looked up afresh on every call (cheap, and correct again
// after the device's primary context was reset and recreated); under
// capture, where no runtime call may touch the device, the address recorded
// by the last call outside capture on this device is used.
arma_status static_scratch_address(cudaStream_t stream, void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return ARMA_ERR_CUDA;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(stream, &cap) != cudaSuccess) return ARMA_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  if (cap == cudaStreamCaptureStatusNone) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p) return ARMA_ERR_CUDA;
    g_addr[dev] = p;
  }
  if (!g_addr[dev]) return ARMA_ERR_CUDA;
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
  arma_status s = static_scratch_address(static_cast<cudaStream_t>(stream), &scratch);
  if (s != ARMA_OK) return s;
  return arma_gpu_eval(plan, in_ptrs, out_ptrs, scratch, ARMA_STATIC_SCRATCH_BYTES, stream);
}
