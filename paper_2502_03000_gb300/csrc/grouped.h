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
  int64_t pa, pb;               // tensor cores: first packed row of op(A) and of op(B)^T
};

constexpr int kTraceSlots = 8;  // trace partials per diagonal tile (one per writer, summed in order)

// One tensor-core output tile with everything its kernel reads, in the
// order the tiles are processed (longest first): one 64-byte load per tile
// instead of a chain of dependent ones.  The operands are read from the
// packed arrays: K block kb of the tile's op(A) rows starts at packed row
// ya + kb * sa (sa = m), of its op(B)^T rows at yb + kb * sb (sb = n).
struct __align__(16) GroupedTile {
  const void* C;                // may be null
  void* D;                      // contiguous: leading dimension m
  int32_t ya, yb;               // packed row of (tile row 0, K block 0)
  int32_t sa, sb;               // packed rows per K block
  int32_t m, n, k, ldc;
  uint16_t tm, tn;              // tile row and column
  int32_t t;                    // index in the tile list (trace partial slot)
  uint16_t ha, hb;              // rows each operand box loads (16, 32, 64 or 128)
  int32_t pad;
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
  // tensor cores: the packed operands in the workspace, K-block-major BF16
  // rows of 64 (slice s of op(A) row p at pack_a + (s * rows_a + p) * 64)
  void* pack_a;
  void* pack_b;
  int64_t rows_a, rows_b;       // packed rows per slice
  int32_t slices;               // 1 (BF16 operands) or 3 (FP32 operands, exact BF16 slices)
  int32_t pad2;
  const int32_t* pack_items;    // pack work items: (2 problem + operand, first row, rows) triplets
  int64_t n_items;
};

// packed rows per pack work item (about: whole rows with all their K blocks)
constexpr int kPackRun = 64;

// K elements per packed row (one K block)
constexpr int kPackK = 64;

cudaError_t launch_grouped(const GroupedArgs& g, cudaStream_t s, int* launches);
cudaError_t launch_grouped_tc(const GroupedArgs& g, cudaStream_t s, int* launches);

}  // namespace arma
