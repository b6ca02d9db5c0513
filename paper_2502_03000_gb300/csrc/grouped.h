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

constexpr int kTraceSlots = 8;  // trace partials per diagonal tile (one per writer, summed in order)

// One tensor-core output tile with everything its kernel reads, in the
// order the tiles are processed (longest first): one 64-byte load per tile
// instead of a chain of dependent ones.
struct __align__(16) GroupedTile {
  const void* A;
  const void* B;
  const void* C;                // may be null
  void* D;
  int32_t m, n, k;              // D is contiguous: leading dimension m
  int32_t lda, ldb, ldc;
  uint16_t tm, tn;              // tile row and column
  int32_t t;                    // index in the tile list (trace partial slot)
};
static_assert(sizeof(GroupedTile) == 64, "GroupedTile is one 64-byte record");

struct GroupedArgs {
  int64_t count, tiles;
  const GroupedProblem* probs;
  const int32_t* tile_prob;     // tile -> problem
  const uint32_t* tile_code;    // tile -> (tm << 16) | tn
  const int32_t* tile_order;    // processing order: tiles by decreasing work
  const GroupedTile* recs;      // tensor-core tiles, in processing order
  unsigned int* next_tile;      // work counter (zeroed before the launch)
  int32_t ta, tb, abdt, cdt, ddt, pad;
  double alpha, beta;
  float alpha_f, beta_f;
  double* trace_partials;       // [tiles][kTraceSlots] (diagonal tiles only), null without traces
  int32_t tc;                   // 1: 128 x 128 tiles on the tensor cores
  int32_t* status;              // workspace status word (device-side failures)
};

cudaError_t launch_grouped(const GroupedArgs& g, cudaStream_t s, int* launches);
cudaError_t launch_grouped_tc(const GroupedArgs& g, cudaStream_t s, int* launches);

}  // namespace arma
