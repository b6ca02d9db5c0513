// Grouped products on the tensor cores (tcgen05, sm_103a): the batched form
// of the folded product D_g = alpha * op(A_g) op(B_g) + beta * C_g with the
// diagonal-only trace t_g = trace(op(A_g) op(B_g)) (Sec. II xGEMM paragraph,
// Sec. III (5)), for thousands of problems of uneven sizes in one persistent
// launch.
//
// One CTA per SM walks its share of the host-built list of 128 x 128 output
// tiles (ordered by decreasing work; CTA c takes positions c, 2G-1-c, 2G+c,
// ... so that the long tiles spread evenly).  Every role walks the same
// sequence, so they need no tile queue:
//   warps 0..15  producers, two groups of eight warps taking alternate K
//                blocks: per K block of 64 a group loads the two operand
//                tiles from global memory (both operands
//                K-contiguous: op(A) = A^T, op(B) = B; leading dimensions of
//                any value, so no tensor map fits them), convert to BF16
//                (S = 1) or split FP32 exactly into three BF16 slices (S = 3,
//                Henry et al. 2019, the BF16 work the paper cites), and store
//                them 128-byte-swizzled into a ring of shared-memory stages;
//                the next block is prefetched into L2 meanwhile
//   warp 16      TMEM owner (two 128-column FP32 accumulators) and MMA issuer:
//                one tcgen05.mma per 16 of K and slice product (6 products of
//                order <= 2 for S = 3, smallest first)
//   warps 17..20 epilogue: tcgen05.ld of a finished accumulator while the next
//                tile's MMAs run into the other; alpha, beta*C, D, and the
//                diagonal of diagonal tiles for the traces
// Every mbarrier wait is bounded: on timeout the CTA records ARMA_ERR_TIMEOUT
// in the status word, waits (bounded) for its issued MMAs, frees TMEM and
// returns.
#include <cuda_bf16.h>

#include <atomic>

#include "common.cuh"
#include "grouped.h"
#include "tc_ops.cuh"

namespace arma {
namespace {

using namespace tc;

constexpr int GM = 128, GN = 128, GK = 64;   // output tile and K block
constexpr int NPROD = 256;                   // producer threads of one group (8 warps)
constexpr int NGROUP = 2;                    // producer groups, alternate K blocks
constexpr int MMA_WARP = 8 * NGROUP;         // warp 16
constexpr int NEPI = 256;                    // warps 17..24: lane quarters 1, 2, 3, 0, twice
constexpr int GTHREADS = (8 * NGROUP + 9) * 32;
constexpr int GSLICE = GM * GK * 2;          // one BF16 operand slice (GN == GM): 16 KiB
constexpr int GTMEM = 256;                   // two 128 x 128 FP32 accumulators

template <int S>
__host__ __device__ constexpr int gstages() { return S == 1 ? 4 : 2; }
template <int S>
__host__ __device__ constexpr int stage_bytes() { return 2 * S * GSLICE; }   // A slices, then B slices
template <int S>
__host__ __device__ constexpr int smem_bytes() { return gstages<S>() * stage_bytes<S>() + 1024 + 256; }

// byte offset of (row r, K index c) in a 128-byte-swizzled K-major tile
// (rows of 64 BF16; the 16-byte chunk index is XORed with r mod 8)
__device__ __forceinline__ uint32_t sw_off(int r, int c) {
  return (uint32_t)(r * 128 + ((((c >> 3) ^ (r & 7)) << 4)) + ((c & 7) << 1));
}

// position of CTA c's walk over the ordered tile list (G CTAs) in round
// `round`: rounds of G tiles, alternate rounds reversed
__device__ __forceinline__ int64_t walk(int64_t round, int c, int G) {
  return round * G + ((round & 1) ? (G - 1 - c) : c);
}

// this thread's 16 rows (pw + 8 i) x 2 K columns (2 lane, 2 lane + 1) of a
// K-contiguous operand tile: rows [row0, row0 + 128) of op(X), K [l0, l0 + 64)
__device__ __forceinline__ void load_pairs(uint32_t (&v)[16], const __nv_bfloat16* X, int64_t ld, int64_t rows,
                                           int64_t row0, int64_t k, int64_t l0, int pw, int lane) {
  const int l = (int)l0 + 2 * lane;
  const unsigned short* p = reinterpret_cast<const unsigned short*>(X) + (row0 + pw) * ld + l;
  const int nr = (int)(rows - row0), kk = (int)k, step = 8 * (int)ld;
  // an even leading dimension and an aligned base make each pair one
  // aligned 32-bit word (l is even)
  const bool words = ((ld & 1) == 0) && ((reinterpret_cast<uintptr_t>(X) & 3u) == 0);
#pragma unroll
  for (int i = 0; i < 16; ++i, p += step) {
    const int r = pw + 8 * i;
    uint32_t w = 0u;
    if (r < nr && l < kk) {
      if (words && l + 1 < kk) w = *reinterpret_cast<const uint32_t*>(p);
      else w = (uint32_t)p[0] | ((l + 1 < kk) ? (uint32_t)p[1] << 16 : 0u);
    }
    v[i] = w;
  }
}

__device__ __forceinline__ void load_pairs(float2 (&v)[16], const float* X, int64_t ld, int64_t rows, int64_t row0,
                                           int64_t k, int64_t l0, int pw, int lane) {
  const int l = (int)l0 + 2 * lane;
  const float* p = X + (row0 + pw) * ld + l;
  const int nr = (int)(rows - row0), kk = (int)k, step = 8 * (int)ld;
  const bool pairs = ((ld & 1) == 0) && ((reinterpret_cast<uintptr_t>(X) & 7u) == 0);
#pragma unroll
  for (int i = 0; i < 16; ++i, p += step) {
    const int r = pw + 8 * i;
    float2 w = make_float2(0.f, 0.f);
    if (r < nr && l < kk) {
      if (pairs && l + 1 < kk) w = *reinterpret_cast<const float2*>(p);
      else { w.x = p[0]; w.y = (l + 1 < kk) ? p[1] : 0.f; }
    }
    v[i] = w;
  }
}

// x = s0 + s1 + s2 exactly, each a BF16: s0 = RN(x), s1 = RN(x - s0), s2 =
// x - s0 - s1 (each difference is exact in FP32; s2 has at most 8
// significant bits); FP32 conversions and subtractions only
__device__ __forceinline__ void split3_rn(float x, uint16_t (&sl)[3]) {
  const __nv_bfloat16 b0 = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(b0);
  const __nv_bfloat16 b1 = __float2bfloat16_rn(r1);
  const float r2 = r1 - __bfloat162float(b1);
  sl[0] = __bfloat16_as_ushort(b0);
  sl[1] = __bfloat16_as_ushort(b1);
  sl[2] = __bfloat16_as_ushort(__float2bfloat16_rn(r2));
}

// the row lines of the next K block into L2 (lanes 0..15: the 16 rows of this warp)
__device__ __forceinline__ void prefetch_rows(const void* X, int64_t ld, int64_t es, int64_t rows, int64_t row0,
                                              int64_t k, int64_t l0, int pw, int lane) {
  if (lane >= 16 || l0 >= k) return;
  const int r = pw + 8 * lane;
  if (r >= rows - row0) return;
  const char* a = static_cast<const char*>(X) + ((row0 + r) * ld + l0) * es;
  asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
}

template <typename AT, int S>
__global__ void __launch_bounds__(GTHREADS, 1) grouped_tc_kernel(const __grid_constant__ GroupedArgs g) {
  constexpr int STAGES = gstages<S>();
  constexpr int SB = stage_bytes<S>();
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * SB);
  // bars: full[STAGES], empty[STAGES], tfull[2], tempty[2], done
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + STAGES);
  const uint32_t tfull0 = smem_u32(bars + 2 * STAGES), tempty0 = smem_u32(bars + 2 * STAGES + 2);
  const uint32_t done_bar = smem_u32(bars + 2 * STAGES + 4);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 5);
  volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int G = gridDim.x, c = blockIdx.x;
  const int64_t rounds = (g.tiles + G - 1) / G;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full0 + 8 * s, NPROD);
      mbar_init(empty0 + 8 * s, 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(tfull0 + 8 * a, 1);
      mbar_init(tempty0 + 8 * a, NEPI);
    }
    mbar_init(done_bar, 1);
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == MMA_WARP) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(GTMEM)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp < MMA_WARP) {
    // ------------------------------------------------------------ producers
    // group grp takes the K blocks q = grp, grp + NGROUP, ... of this CTA's
    // sequence; block q uses stage q % STAGES in its (q / STAGES)-th round
    const int pw = warp & 7, grp = warp >> 3;
    int64_t q = 0;
    bool ok = true;
    for (int64_t rd = 0; rd < rounds && ok; ++rd) {
      const int64_t pos = walk(rd, c, G);
      if (pos >= g.tiles) continue;
      const GroupedTile pb = g.recs[pos];
      const int64_t i0 = (int64_t)pb.tm * GM, j0 = (int64_t)pb.tn * GN;
      const AT* A = static_cast<const AT*>(pb.A);
      const AT* B = static_cast<const AT*>(pb.B);
      const int64_t nkb = (pb.k + GK - 1) / GK;
      for (int64_t kb = 0; kb < nkb; ++kb, ++q) {
        if ((int)(q % NGROUP) != grp) continue;
        if (kb + NGROUP < nkb) {
          prefetch_rows(A, pb.lda, (int64_t)sizeof(AT), pb.m, i0, pb.k, (kb + NGROUP) * GK, pw, lane);
          prefetch_rows(B, pb.ldb, (int64_t)sizeof(AT), pb.n, j0, pb.k, (kb + NGROUP) * GK, pw, lane);
        }
        const int stage = (int)(q % STAGES);
        const uint32_t phase = (uint32_t)((q / STAGES) & 1);
        // the stage's previous MMAs have finished reading it
        ok = __all_sync(0xffffffffu, mbar_wait(empty0 + 8 * stage, phase ^ 1u, abort));
        if (!ok) break;
        unsigned char* sA = smem + stage * SB;
        unsigned char* sB = sA + S * GSLICE;
        if constexpr (S == 1) {
          uint32_t va[16], vb[16];
          load_pairs(va, A, pb.lda, pb.m, i0, pb.k, kb * GK, pw, lane);
          load_pairs(vb, B, pb.ldb, pb.n, j0, pb.k, kb * GK, pw, lane);
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            *reinterpret_cast<uint32_t*>(sA + sw_off(pw + 8 * i, 2 * lane)) = va[i];
            *reinterpret_cast<uint32_t*>(sB + sw_off(pw + 8 * i, 2 * lane)) = vb[i];
          }
        } else {
          // FP32: exact three-slice split
#pragma unroll
          for (int op = 0; op < 2; ++op) {
            float2 v[16];
            if (op == 0) load_pairs(v, reinterpret_cast<const float*>(A), pb.lda, pb.m, i0, pb.k, kb * GK, pw, lane);
            else load_pairs(v, reinterpret_cast<const float*>(B), pb.ldb, pb.n, j0, pb.k, kb * GK, pw, lane);
            unsigned char* dst = op == 0 ? sA : sB;
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              uint16_t x0[3], x1[3];
              split3_rn(v[i].x, x0);
              split3_rn(v[i].y, x1);
              const uint32_t off = sw_off(pw + 8 * i, 2 * lane);
#pragma unroll
              for (int sl = 0; sl < 3; ++sl)
                *reinterpret_cast<uint32_t*>(dst + sl * GSLICE + off) = (uint32_t)x0[sl] | ((uint32_t)x1[sl] << 16);
            }
          }
        }
        // generic-proxy stores become visible to the tensor core, then arrive
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(full0 + 8 * stage);
      }
    }
  } else if (warp == MMA_WARP) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(GM, GN);
      int stage = 0;
      uint32_t phase = 0;
      int acc = 0;
      uint32_t aphase = 0;
      bool ok = true, issued = false;
      for (int64_t rd = 0; rd < rounds && ok; ++rd) {
        const int64_t pos = walk(rd, c, G);
        if (pos >= g.tiles) continue;
        const int64_t nkb = (g.recs[pos].k + GK - 1) / GK;
        if (!mbar_wait(tempty0 + 8 * acc, aphase ^ 1u, abort)) { ok = false; break; }
        fence_after();
        const uint32_t dcol = tmem_base + (uint32_t)(acc * GN);
        for (int64_t kb = 0; kb < nkb; ++kb) {
          if (!mbar_wait(full0 + 8 * stage, phase, abort)) { ok = false; break; }
          fence_after();
          const uint64_t ad = sw128_desc(smem_u32(smem + stage * SB));
          const uint64_t bd = sw128_desc(smem_u32(smem + stage * SB + S * GSLICE));
          constexpr int NT = S == 1 ? 1 : 6;
#pragma unroll
          for (int term = 0; term < NT; ++term) {
            // split products smallest first: (2,0) (1,1) (0,2) (1,0) (0,1) (0,0)
            const int sa = S == 1 ? 0 : (term == 0 ? 2 : term == 1 ? 1 : term == 2 ? 0 : term == 3 ? 1 : 0);
            const int sb = S == 1 ? 0 : (term == 0 ? 0 : term == 1 ? 1 : term == 2 ? 2 : term == 3 ? 0 : term == 4 ? 1 : 0);
            const uint64_t a0 = ad + (uint64_t)((sa * GSLICE) >> 4), b0 = bd + (uint64_t)((sb * GSLICE) >> 4);
#pragma unroll
            for (int kk = 0; kk < GK / 16; ++kk)
              mma_bf16(dcol, a0 + (uint64_t)(2 * kk), b0 + (uint64_t)(2 * kk), idesc,
                       (kb > 0 || term > 0 || kk > 0) ? 1u : 0u);
          }
          mma_commit(empty0 + 8 * stage);    // frees the stage when these MMAs finish
          issued = true;
          if (++stage == STAGES) { stage = 0; phase ^= 1u; }
        }
        if (!ok) break;
        mma_commit(tfull0 + 8 * acc);         // the tile's accumulator is complete
        if (++acc == 2) { acc = 0; aphase ^= 1u; }
      }
      if (issued) {
        mma_commit(done_bar);
        for (uint32_t i = 0; i < WAIT_LIMIT && !mbar_try(done_bar, 0); ++i) {
        }
      }
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ epilogue
    // warp w: TMEM lane quarter w % 4 (tile rows 32 (w % 4) ..) and column
    // half (w - 17) / 4; each thread owns one row and 64 columns
    const int q = warp & 3;
    const int half = (warp - (MMA_WARP + 1)) >> 2;
    const uint32_t lane_base = (uint32_t)(q * 32) << 16;
    int acc = 0;
    uint32_t aphase = 0;
    bool ok = true;
    for (int64_t rd = 0; rd < rounds && ok; ++rd) {
      const int64_t pos = walk(rd, c, G);
      if (pos >= g.tiles) continue;
      const GroupedTile pb = g.recs[pos];
      const int64_t t = pb.t;
      const int tm = pb.tm, tn = pb.tn;
      const int64_t i0 = (int64_t)tm * GM, j0 = (int64_t)tn * GN + 64 * half;
      const int64_t row = i0 + 32 * q + lane;
      const bool row_ok = row < pb.m;
      const bool has_c = pb.C && g.beta != 0.0;
      const int ncol = (int)(pb.n - j0 < 64 ? pb.n - j0 : 64);   // may be <= 0
      // this warp's block of C into L2 while the tile's MMAs run: lane j,
      // columns j and j + 32
      if (has_c && i0 + 32 * q < pb.m) {
        const int64_t es = g.cdt == ARMA_F64 ? 8 : g.cdt == ARMA_F32 ? 4 : 2;
#pragma unroll
        for (int u = 0; u < 2; ++u)
          if (lane + 32 * u < ncol)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(static_cast<const char*>(pb.C) +
                                                          ((i0 + 32 * q) + (j0 + lane + 32 * u) * pb.ldc) * es));
      }
      ok = __all_sync(0xffffffffu, mbar_wait(tfull0 + 8 * acc, aphase, abort));
      if (!ok) break;
      fence_after();
      const bool any_k = pb.k > 0;
      float* Dr = static_cast<float*>(pb.D) + row + j0 * (int64_t)pb.m;
      const int ldc = pb.ldc, ldd = pb.m;
      const int diag = (int)(row - j0);
      double dsum = 0.0;
      // 16 columns at a time: the TMEM load, then all 16 C loads, then D
      // (D may be C itself, so C is read before D is written)
#pragma unroll 1
      for (int c0 = 0; c0 < 64 && c0 < ncol; c0 += 16) {
        float v[16];
        if (any_k) {
          tmem_ld16(tmem_base + lane_base + (uint32_t)(acc * GN + 64 * half + c0), v);
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j) v[j] = 0.f;
        }
        if (!row_ok) continue;
        float cv[16];
        if (has_c && g.cdt == ARMA_F32) {
          const float* Cr = static_cast<const float*>(pb.C) + row + (j0 + c0) * pb.ldc;
#pragma unroll
          for (int j = 0; j < 16; ++j) cv[j] = c0 + j < ncol ? Cr[j * ldc] : 0.f;
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j)
            cv[j] = (has_c && c0 + j < ncol) ? load_as<float>(pb.C, row + (j0 + c0 + j) * pb.ldc, g.cdt) : 0.f;
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          if (c0 + j >= ncol) continue;
          if (c0 + j == diag) dsum += (double)v[j];
          Dr[(c0 + j) * ldd] = fmaf(g.beta_f, cv[j], g.alpha_f * v[j]);
        }
      }
      // the accumulator is free for the MMA issuer again
      fence_before();
      mbar_arrive(tempty0 + 8 * acc);
      if (++acc == 2) { acc = 0; aphase ^= 1u; }
      if (g.trace_partials && tm == tn) {     // diagonal tile: each warp's share of the trace
        dsum = warp_sum(dsum);
        if (lane == 0) g.trace_partials[kTraceSlots * t + 4 * half + q] = dsum;
      }
    }
  }

  fence_before();
  __syncthreads();
  if (threadIdx.x == 0 && *abort && g.status) atomicCAS(g.status, 0, (int32_t)ARMA_ERR_TIMEOUT);
  if (warp == MMA_WARP) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(GTMEM) : "memory");
  }
}

// ---------------------------------------------------------------------------
// BF16 operands: every warp of the CTA loads, one thread issues the MMAs and
// every warp drains the accumulator; two CTAs per SM, each with two stages
// so that the loads of K block k + 1 overlap the MMAs of block k.  CTAs take
// tiles from a shared counter over the ordered list (longest first); the
// next tile's position and record are fetched while the current tile runs.
// ---------------------------------------------------------------------------
constexpr int STHREADS = 256;
constexpr int SCTAS = 2;                       // CTAs per SM (<= 128 registers per thread)
constexpr int STMEM = 128;                     // one 128 x 128 FP32 accumulator
constexpr int SSTAGE = 2 * GSLICE;             // A tile, then B tile
constexpr int SSMEM = 2 * SSTAGE + 1024 + 256;

__global__ void __launch_bounds__(STHREADS, SCTAS) grouped_tc_serial_kernel(const __grid_constant__ GroupedArgs g) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + 2 * SSTAGE);   // MMA done, per stage
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2);
  volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
  int* s_pos = reinterpret_cast<int*>(tmem_slot + 2);                // the current tile's position
  uint4* s_rec = reinterpret_cast<uint4*>(bars + 4);                 // and its record
  const uint32_t done0 = smem_u32(bars);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint4* recs = reinterpret_cast<const uint4*>(g.recs);
  if (threadIdx.x == 0) {
    mbar_init(done0, 1);
    mbar_init(done0 + 8, 1);
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    int p0 = 0;
    if (lane == 0) p0 = (int)atomicAdd(g.next_tile, 1u);
    p0 = __shfl_sync(0xffffffffu, p0, 0);
    if (lane == 0) *s_pos = p0;
    if (lane < 4 && p0 < g.tiles) s_rec[lane] = recs[4 * (int64_t)p0 + lane];
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(STMEM)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const uint32_t idesc = idesc_bf16(GM, GN);
  int64_t issued = 0;   // K blocks issued by this CTA: stage = issued & 1
  bool ok = true;
  while (ok) {
    const int64_t pos = *s_pos;
    if (pos >= g.tiles) break;
    GroupedTile pb;
    *reinterpret_cast<uint4*>(&pb) = s_rec[0];
    reinterpret_cast<uint4*>(&pb)[1] = s_rec[1];
    reinterpret_cast<uint4*>(&pb)[2] = s_rec[2];
    reinterpret_cast<uint4*>(&pb)[3] = s_rec[3];
    const int64_t i0 = (int64_t)pb.tm * GM, j0 = (int64_t)pb.tn * GN;
    const __nv_bfloat16* A = static_cast<const __nv_bfloat16*>(pb.A);
    const __nv_bfloat16* B = static_cast<const __nv_bfloat16*>(pb.B);
    const int64_t nkb = (pb.k + GK - 1) / GK;
    uint32_t ra[16], rb[16];
    if (nkb > 0) {
      load_pairs(ra, A, pb.lda, pb.m, i0, pb.k, 0, warp, lane);
      load_pairs(rb, B, pb.ldb, pb.n, j0, pb.k, 0, warp, lane);
    }
    // the next tile's position and record, in flight during this tile
    // (after this warp's first loads, so that they overlap)
    int npos = 0;
    uint4 nrec = make_uint4(0u, 0u, 0u, 0u);
    if (warp == 0) {
      if (lane == 0) npos = (int)atomicAdd(g.next_tile, 1u);
      npos = __shfl_sync(0xffffffffu, npos, 0);
      if (lane < 4 && npos < g.tiles) nrec = recs[4 * (int64_t)npos + lane];
    }
    for (int64_t kb = 0; kb < nkb; ++kb, ++issued) {
      const int st = (int)(issued & 1);
      unsigned char* sA = smem + st * SSTAGE;
      unsigned char* sB = sA + GSLICE;
      // the stage's previous MMAs (two K blocks ago) must have finished
      if (issued >= 2 && !mbar_wait(done0 + 8 * st, (uint32_t)(((issued >> 1) - 1) & 1), abort)) *abort = 1;
      if (!*abort) {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          *reinterpret_cast<uint32_t*>(sA + sw_off(warp + 8 * i, 2 * lane)) = ra[i];
          *reinterpret_cast<uint32_t*>(sB + sw_off(warp + 8 * i, 2 * lane)) = rb[i];
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic stores -> tensor core
      if (__syncthreads_or(*abort != 0)) { ok = false; break; }
      if (threadIdx.x == 0) {
        fence_after();
        const uint64_t ad = sw128_desc(smem_u32(sA)), bd = sw128_desc(smem_u32(sB));
#pragma unroll
        for (int kk = 0; kk < GK / 16; ++kk)
          mma_bf16(tmem_base, ad + (uint64_t)(2 * kk), bd + (uint64_t)(2 * kk), idesc, (kb > 0 || kk > 0) ? 1u : 0u);
        mma_commit(done0 + 8 * st);
      }
      // the next block's loads overlap these MMAs
      if (kb + 1 < nkb) {
        load_pairs(ra, A, pb.lda, pb.m, i0, pb.k, (kb + 1) * GK, warp, lane);
        load_pairs(rb, B, pb.ldb, pb.n, j0, pb.k, (kb + 1) * GK, warp, lane);
      }
    }
    if (!ok) break;
    // while the last MMAs run: this warp's block of C (32 rows x 64 columns)
    // into L2
    const bool has_c = pb.C && g.beta != 0.0;
    {
      const int q = warp & 3, h = warp >> 2;
      if (has_c && i0 + 32 * q < pb.m) {
        const int64_t es = g.cdt == ARMA_F64 ? 8 : g.cdt == ARMA_F32 ? 4 : 2;
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int64_t col = j0 + 64 * h + 32 * u + lane;
          if (col < pb.n)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(static_cast<const char*>(pb.C) +
                                                          ((i0 + 32 * q) + col * pb.ldc) * es));
        }
      }
    }
    // accumulator complete: the last commit covers every earlier MMA
    if (nkb > 0) {
      const int64_t last = issued - 1;
      if (!mbar_wait(done0 + 8 * (int)(last & 1), (uint32_t)((last >> 1) & 1), abort)) *abort = 1;
      if (__syncthreads_or(*abort != 0)) { ok = false; break; }
      fence_after();
    }
    // epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31 (tile rows) and
    // columns 64 (w / 4) .. +63
    const int q = warp & 3, h = warp >> 2;
    const int64_t row = i0 + 32 * q + lane;
    const bool row_ok = row < pb.m;
    float* Dr = static_cast<float*>(pb.D) + row + (j0 + 64 * h) * (int64_t)pb.m;
    const int ncol = (int)(pb.n - (j0 + 64 * h));
    const int diag = (int)(row - (j0 + 64 * h));
    double dsum = 0.0;
#pragma unroll 1
    for (int c0 = 0; c0 < 64 && c0 < ncol; c0 += 16) {
      float v[16];
      if (nkb > 0) {
        tmem_ld16(tmem_base + ((uint32_t)(32 * q) << 16) + (uint32_t)(64 * h + c0), v);
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = 0.f;
      }
      if (!row_ok) continue;
      // all 16 C values before any D (D may be C itself)
      float cv[16];
      if (has_c && g.cdt == ARMA_F32) {
        const float* Cr = static_cast<const float*>(pb.C) + row + (j0 + 64 * h + c0) * (int64_t)pb.ldc;
#pragma unroll
        for (int j = 0; j < 16; ++j) cv[j] = c0 + j < ncol ? Cr[j * pb.ldc] : 0.f;
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j)
          cv[j] = (has_c && c0 + j < ncol) ? load_as<float>(pb.C, row + (j0 + 64 * h + c0 + j) * pb.ldc, g.cdt) : 0.f;
      }
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        if (c0 + j >= ncol) continue;
        if (c0 + j == diag) dsum += (double)v[j];
        Dr[(c0 + j) * pb.m] = fmaf(g.beta_f, cv[j], g.alpha_f * v[j]);
      }
    }
    if (g.trace_partials && pb.tm == pb.tn) {   // diagonal tile: its share of the trace
      double qq = 0.0;
      block_sum2(dsum, qq);
      if (threadIdx.x == 0) {
        g.trace_partials[(int64_t)kTraceSlots * pb.t] = dsum;
        for (int k = 1; k < kTraceSlots; ++k) g.trace_partials[(int64_t)kTraceSlots * pb.t + k] = 0.0;
      }
    }
    // TMEM reads finish before the next tile's MMAs overwrite the
    // accumulator; the next record replaces the current one
    fence_before();
    __syncthreads();
    if (threadIdx.x < 4) s_rec[threadIdx.x] = nrec;
    if (threadIdx.x == 0) *s_pos = npos;
    __syncthreads();
    fence_after();
  }
  // every issued MMA completes before TMEM is released
  if (issued > 0 && threadIdx.x == 0) {
    const int64_t last = issued - 1;
    for (uint32_t i = 0; i < WAIT_LIMIT && !mbar_try(done0 + 8 * (int)(last & 1), (uint32_t)((last >> 1) & 1)); ++i) {
    }
  }
  fence_before();
  __syncthreads();
  if (threadIdx.x == 0 && *abort && g.status) atomicCAS(g.status, 0, (int32_t)ARMA_ERR_TIMEOUT);
  if (warp == 0) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(STMEM) : "memory");
  }
}

cudaError_t launch_tc_serial(const GroupedArgs& g, cudaStream_t s, int* launches) {
  static std::atomic<bool> attr[64];
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (!attr[dev].load(std::memory_order_acquire)) {
    cudaError_t e = cudaFuncSetAttribute(grouped_tc_serial_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SSMEM);
    if (e != cudaSuccess) return e;
    attr[dev].store(true, std::memory_order_release);
  }
  int64_t grid = (int64_t)device_sm_count() * SCTAS;
  if (grid > g.tiles) grid = g.tiles;
  grouped_tc_serial_kernel<<<(unsigned)grid, STHREADS, SSMEM, s>>>(g);
  if (launches) ++*launches;
  return cudaGetLastError();
}

template <typename AT, int S>
cudaError_t launch_tc(const GroupedArgs& g, cudaStream_t s, int* launches) {
  constexpr int smem = smem_bytes<S>();
  static std::atomic<bool> attr[64];
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (!attr[dev].load(std::memory_order_acquire)) {
    cudaError_t e = cudaFuncSetAttribute(grouped_tc_kernel<AT, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    attr[dev].store(true, std::memory_order_release);
  }
  // one CTA per SM, each walking its share of the tile list
  int64_t grid = (int64_t)device_sm_count();
  if (grid > g.tiles) grid = g.tiles;
  grouped_tc_kernel<AT, S><<<(unsigned)grid, GTHREADS, smem, s>>>(g);
  if (launches) ++*launches;
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_grouped_tc(const GroupedArgs& g, cudaStream_t s, int* launches) {
  if (g.tiles == 0) return cudaSuccess;
  if (!g.recs) return cudaErrorInvalidValue;
  if (g.abdt == ARMA_BF16) return launch_tc_serial(g, s, launches);
  if (g.abdt == ARMA_F32) return launch_tc<float, 3>(g, s, launches);
  return cudaErrorInvalidValue;
}

}  // namespace arma
