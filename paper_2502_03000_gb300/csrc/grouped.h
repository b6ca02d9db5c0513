// Problem table of the grouped (batched) product kernel.
#pragma once

#include <stdint.h>

namespace arma {

struct GroupedProblem {       // one per problem, in the device table
  int64_t m, n, k;
  const void* A; int64_t lda;
  const void* B; int64_t ldb;
  const void* C; int64_t ldc;   // may be null
  void* D; int64_t ldd;
  double* trace;                // may be null
  int64_t first_tile;           // index of tile (0, 0) in the tile list
  int32_t tile;                 // tile edge: 32 or 64 (SIMT), 128 (tensor cores)
  int32_t pad;
};

struct GroupedArgs {
  int64_t count, tiles;
  const GroupedProblem* probs;
  const int32_t* tile_prob;     // tile -> problem
  const uint32_t* tile_code;    // tile -> (tm << 16) | tn
  const int32_t* tile_order;    // processing order: tiles by decreasing work
  unsigned int* next_tile;      // work counter (zeroed before the launch)
  int32_t ta, tb, abdt, cdt, ddt, pad;
  double alpha, beta;
  float alpha_f, beta_f;
  double* trace_partials;       // [tiles] (diagonal tiles only), null without traces
  int32_t tc;                   // 1: 128 x 128 tiles on the tensor cores
  int32_t* status;              // workspace status word (device-side failures)
};

cudaError_t launch_grouped(const GroupedArgs& g, cudaStream_t s, int* launches);
cudaError_t launch_grouped_tc(const GroupedArgs& g, cudaStream_t s, int* launches);

}  // namespace arma
