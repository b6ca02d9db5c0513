// tcgen05 GEMM (placeholder until the tensor-core path lands).
#include "common.cuh"

namespace arma {
bool gemm_tc_supported(const GemmArgs&) { return false; }
int64_t gemm_tc_scratch_bytes(int64_t, int64_t, int64_t, int32_t) { return 0; }
cudaError_t launch_gemm_tc(const GemmArgs&, cudaStream_t, int*) { return cudaErrorNotSupported; }
}  // namespace arma
