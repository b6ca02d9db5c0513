// Grouped products on the tensor cores (tcgen05, sm_103a): the batched form
// of the folded product D_g = alpha * op(A_g) op(B_g) + beta * C_g with the
// diagonal-only trace t_g = trace(op(A_g) op(B_g)) (Sec. II xGEMM paragraph,
// Sec. III (5)), for thousands of problems of uneven sizes in one persistent
// launch.
//
// The CTAs (three per SM) take 128 x 128 output tiles from a shared counter
// over the host-built list, longest first.  Per K block
// of 64 every thread loads its share of the two operand tiles from global
// memory (both operands K-contiguous: op(A) = A^T, op(B) = B), converts them
// to BF16 and stores them in the 128-byte-swizzled K-major layout that the
// tcgen05 shared-memory descriptors describe; one thread then issues the
// MMAs into a 128 x 128 FP32 accumulator in TMEM.  Two shared-memory stages:
// the loads of block k+1 overlap the MMAs of block k.  The epilogue reads
// the accumulator with tcgen05.ld, applies alpha and beta*C, stores D and
// adds the tile's diagonal to the trace partials.
//
// Element type: BF16 operands, which go in as they are (one MMA per 16 of
// K; the kernel keeps a slice parameter S for split operands).  FP32
// operands take the SIMT tiles: their exact three-slice split measured
// slower than SIMT for the benchmark's size mix.
//
// Waits on the MMA-completion barriers are bounded: on timeout the CTA
// records ARMA_ERR_TIMEOUT in the status word, waits (bounded) for its issued
// MMAs, frees TMEM and returns.
#include <cuda_bf16.h>

#include <atomic>

#include "common.cuh"
#include "grouped.h"
#include "tc_ops.cuh"

namespace arma {
namespace {

using namespace tc;

constexpr int GM = 128, GN = 128, GK = 64;   // output tile and K block
constexpr int GTHREADS = 256;
constexpr int GSLICE = GM * GK * 2;          // one BF16 operand slice (GN == GM): 16 KiB
constexpr int GTMEM = 128;                   // TMEM columns: one 128 x 128 FP32 accumulator

template <int S>
__host__ __device__ constexpr int stage_bytes() { return 2 * S * GSLICE; }   // A slices, then B slices
template <int S>
__host__ __device__ constexpr int smem_bytes() { return 2 * stage_bytes<S>() + 1024 + 64; }

// byte offset of (row r, K index c) in a 128-byte-swizzled K-major tile
// (rows of 64 BF16; the 16-byte chunk index is XORed with r mod 8)
__device__ __forceinline__ uint32_t sw_off(int r, int c) {
  return (uint32_t)(r * 128 + ((((c >> 3) ^ (r & 7)) << 4)) + ((c & 7) << 1));
}

// this thread's 16 rows (warp + 8 i) x 2 K columns (2 lane, 2 lane + 1) of a
// K-contiguous operand tile: rows [row0, row0 + 128) of op(X), K [l0, l0 + 64).
// BF16 pairs are packed into one register as loaded; offsets are 32-bit
// (each problem's operand is far below 2^31 elements).
template <typename AT>
struct TileRegs;
template <>
struct TileRegs<__nv_bfloat16> {
  uint32_t v[16];
};

__device__ __forceinline__ void tile_load(TileRegs<__nv_bfloat16>& t, const __nv_bfloat16* X, int64_t ld,
                                          int64_t rows, int64_t row0, int64_t k, int64_t l0, int warp, int lane) {
  const int l = (int)l0 + 2 * lane;
  const unsigned short* p = reinterpret_cast<const unsigned short*>(X) + (row0 + warp) * ld + l;
  const int nr = (int)(rows - row0), kk = (int)k, step = 8 * (int)ld;
  // an even leading dimension and an aligned base make every pair a 4-byte
  // aligned word (l is even): one load per pair instead of two
  const bool words = ((ld & 1) == 0) && ((reinterpret_cast<uintptr_t>(X) & 3u) == 0);
  if (words) {
#pragma unroll
    for (int i = 0; i < 16; ++i, p += step) {
      const int r = warp + 8 * i;
      uint32_t w = 0u;
      if (r < nr && l + 1 < kk) w = *reinterpret_cast<const uint32_t*>(p);
      else if (r < nr && l < kk) w = p[0];
      t.v[i] = w;
    }
    return;
  }
#pragma unroll
  for (int i = 0; i < 16; ++i, p += step) {
    const int r = warp + 8 * i;
    const uint32_t a = (r < nr && l < kk) ? p[0] : 0u;
    const uint32_t b = (r < nr && l + 1 < kk) ? p[1] : 0u;
    t.v[i] = a | (b << 16);
  }
}

template <int S>
__device__ __forceinline__ void tile_store(const TileRegs<__nv_bfloat16>& t, unsigned char* dst, int warp, int lane) {
#pragma unroll
  for (int i = 0; i < 16; ++i) *reinterpret_cast<uint32_t*>(dst + sw_off(warp + 8 * i, 2 * lane)) = t.v[i];
}

constexpr int GCTAS = 3;   // CTAs per SM: 3 x 64 KiB of stages, 3 x 128 TMEM columns

template <typename AT, int S>
__global__ void __launch_bounds__(GTHREADS, S == 1 ? GCTAS : 1) grouped_tc_kernel(const __grid_constant__ GroupedArgs g) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + 2 * stage_bytes<S>());   // MMA done, per stage
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2);
  volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const uint32_t done0 = smem_u32(bars);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    mbar_init(done0, 1);
    mbar_init(done0 + 8, 1);
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(GTMEM)
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
  TileRegs<AT> ra, rb;
  __shared__ int s_next;
  if (threadIdx.x == 0) s_next = (int)atomicAdd(g.next_tile, 1u);
  __syncthreads();
  for (int64_t i = s_next; i < g.tiles && ok;) {
    const int64_t t = g.tile_order[i];
    const uint32_t code = g.tile_code[t];
    const GroupedProblem pb = g.probs[g.tile_prob[t]];
    const int tm = (int)(code >> 16), tn = (int)(code & 0xFFFFu);
    const int64_t i0 = (int64_t)tm * GM, j0 = (int64_t)tn * GN;
    const AT* A = static_cast<const AT*>(pb.A);
    const AT* B = static_cast<const AT*>(pb.B);
    const int64_t nkb = (pb.k + GK - 1) / GK;
    if (nkb > 0) {
      tile_load(ra, A, pb.lda, pb.m, i0, pb.k, 0, warp, lane);
      tile_load(rb, B, pb.ldb, pb.n, j0, pb.k, 0, warp, lane);
    }
    for (int64_t kb = 0; kb < nkb; ++kb, ++issued) {
      const int st = (int)(issued & 1);
      unsigned char* sA = smem + st * stage_bytes<S>();
      unsigned char* sB = sA + S * GSLICE;
      // the stage's previous MMAs (two K blocks ago) must have finished
      if (issued >= 2 && !mbar_wait(done0 + 8 * st, (uint32_t)(((issued >> 1) - 1) & 1), abort)) *abort = 1;
      if (!*abort) {
        tile_store<S>(ra, sA, warp, lane);
        tile_store<S>(rb, sB, warp, lane);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic stores -> tensor core
      if (__syncthreads_or(*abort != 0)) { ok = false; break; }
      if (threadIdx.x == 0) {
        fence_after();
        const uint64_t ad = sw128_desc(smem_u32(sA)), bd = sw128_desc(smem_u32(sB));
        constexpr int NT = S == 1 ? 1 : 6;
#pragma unroll
        for (int term = 0; term < NT; ++term) {
          // split products smallest first: (2,0) (1,1) (0,2) (1,0) (0,1) (0,0)
          const int sa = S == 1 ? 0 : (term == 0 ? 2 : term == 1 ? 1 : term == 2 ? 0 : term == 3 ? 1 : 0);
          const int sb = S == 1 ? 0 : (term == 0 ? 0 : term == 1 ? 1 : term == 2 ? 2 : term == 3 ? 0 : term == 4 ? 1 : 0);
          const uint64_t a0 = ad + (uint64_t)((sa * GSLICE) >> 4), b0 = bd + (uint64_t)((sb * GSLICE) >> 4);
#pragma unroll
          for (int kk = 0; kk < GK / 16; ++kk)
            mma_bf16(tmem_base, a0 + (uint64_t)(2 * kk), b0 + (uint64_t)(2 * kk), idesc,
                     (kb > 0 || term > 0 || kk > 0) ? 1u : 0u);
        }
        mma_commit(done0 + 8 * st);
      }
      // the next block's loads overlap these MMAs
      if (kb + 1 < nkb) {
        tile_load(ra, A, pb.lda, pb.m, i0, pb.k, (kb + 1) * GK, warp, lane);
        tile_load(rb, B, pb.ldb, pb.n, j0, pb.k, (kb + 1) * GK, warp, lane);
      }
    }
    if (!ok) break;
    // while the last MMAs run: this warp's block of C (32 rows x 64 columns)
    // into L2
    const int q = warp & 3, h = warp >> 2;
    const bool has_c = pb.C && g.beta != 0.0;
    if (has_c && i0 + 32 * q < pb.m) {
      const size_t es = g.cdt == ARMA_F64 ? 8 : g.cdt == ARMA_F32 ? 4 : 2;
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int64_t col = j0 + 64 * h + 32 * u + lane;
        if (col < pb.n) {
          const char* a = static_cast<const char*>(pb.C) + (size_t)((i0 + 32 * q) + col * pb.ldc) * es;
          asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
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
    const int64_t row = i0 + 32 * q + lane;
    const bool row_ok = row < pb.m;
    float* D = static_cast<float*>(pb.D);
    double dsum = 0.0;
    // 32-bit offsets from this thread's row (each problem is far below 2^31
    // elements); columns beyond n are skipped, rows beyond m store nothing
    const int ncol = (int)(pb.n - (j0 + 64 * h));
    const int ldc = (int)pb.ldc, ldd = (int)pb.ldd;
    float* Dr = D + row + (j0 + 64 * h) * pb.ldd;
    const int diag = (int)(row - (j0 + 64 * h));   // column index of the diagonal element
#pragma unroll 1
    for (int c0 = 0; c0 < 64; c0 += 16) {
      float v[16];
      if (nkb > 0) {
        tmem_ld16(tmem_base + ((uint32_t)(32 * q) << 16) + (uint32_t)(64 * h + c0), v);
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = 0.f;
      }
      if (!row_ok) continue;
      // C is read as each D element is formed (few live registers: three
      // CTAs share the SM's register file); the storage type is uniform
      if (has_c && g.cdt == ARMA_F32) {
        const float* Cr = static_cast<const float*>(pb.C) + row + (j0 + 64 * h + c0) * pb.ldc;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          if (c0 + j >= ncol) continue;
          if (c0 + j == diag) dsum += (double)v[j];
          Dr[(c0 + j) * ldd] = fmaf(g.beta_f, Cr[j * ldc], g.alpha_f * v[j]);
        }
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          if (c0 + j >= ncol) continue;
          if (c0 + j == diag) dsum += (double)v[j];
          const float cv = has_c ? load_as<float>(pb.C, row + (j0 + 64 * h + c0 + j) * pb.ldc, g.cdt) : 0.f;
          Dr[(c0 + j) * ldd] = fmaf(g.beta_f, cv, g.alpha_f * v[j]);
        }
      }
    }
    if (g.trace_partials && tm == tn) {   // diagonal tile: its share of the trace
      double qq = 0.0;
      block_sum2(dsum, qq);
      if (threadIdx.x == 0) g.trace_partials[t] = dsum;
    }
    // TMEM reads finish before the next tile's MMAs overwrite the accumulator;
    // the next tile comes from the shared counter (longest first)
    fence_before();
    if (threadIdx.x == 0) s_next = (int)atomicAdd(g.next_tile, 1u);
    __syncthreads();
    fence_after();
    i = s_next;
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
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(GTMEM) : "memory");
  }
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
    // the whole unified cache as shared memory, so that several CTAs fit
    e = cudaFuncSetAttribute(grouped_tc_kernel<AT, S>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    attr[dev].store(true, std::memory_order_release);
  }
  // one wave of GCTAS CTAs per SM (the register bound of the launch and
  // the shared-memory carveout allow it; TMEM holds 4 x 128 columns); the
  // CTAs take tiles from the shared counter
  int64_t grid = (int64_t)device_sm_count() * (S == 1 ? GCTAS : 1);
  if (grid > g.tiles) grid = g.tiles;
  grouped_tc_kernel<AT, S><<<(unsigned)grid, GTHREADS, smem, s>>>(g);
  if (launches) ++*launches;
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_grouped_tc(const GroupedArgs& g, cudaStream_t s, int* launches) {
  if (g.tiles == 0) return cudaSuccess;
  if (g.abdt == ARMA_BF16) return launch_tc<__nv_bfloat16, 1>(g, s, launches);
  return cudaErrorInvalidValue;   // FP32 operands take the SIMT tiles
}

}  // namespace arma
