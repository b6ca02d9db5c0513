// LU solve (placeholder).
#include "common.cuh"

namespace arma {
int64_t solve_scratch_bytes(int64_t, int64_t, int32_t) { return 256; }
cudaError_t launch_solve(const SolveArgs&, cudaStream_t, int*) { return cudaErrorNotSupported; }
}  // namespace arma
