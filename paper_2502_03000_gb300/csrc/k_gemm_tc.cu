// Tensor-core products on sm_103a: tcgen05.mma (kind::f16, BF16 operands,
// FP32 accumulation in TMEM) fed by TMA into 128-byte-swizzled shared
// memory, with the paper's folded scalars, transposes and diagonal scalings
// (Sec. II, glue_times carrying alpha and the transpose flags, Fig. 3)
// applied in the operand preparation and in the epilogue.
//
// Pipeline (one CTA per SM, persistent over output tiles):
//   warp 0      TMA producer: A and B tiles into a 4-stage smem ring
//   warp 1      owns TMEM (512 columns = two 128 x 256 FP32 accumulators)
//               and issues tcgen05.mma from one elected lane
//   warps 2..9  epilogue: drain each finished TMEM accumulator chunk into
//               FP32 register sums, then scale and store (overlaps the MMA
//               through the second accumulator)
//
// Precision tiers.  BF16: one product of BF16-rounded operands.  Split-BF16:
// each operand is split exactly into three BF16 slices x = x0 + x1 + x2
// (its leading 24 significand bits) and the six slice products whose order
// is at most 2 (x0y0, x0y1, x1y0, x0y2, x1y1, x2y0) are accumulated, which
// gives about FP32 accuracy from BF16 tensor cores (Henry et al. 2019, the
// BF16 work the paper cites for future element types).  Slice products run
// smallest first.  The tensor core's own FP32 accumulation loses accuracy
// over long K, so the split tier accumulates in TMEM for 256 of K at a time
// and the epilogue adds each chunk into correctly rounded FP32 registers;
// split-K over CTAs (FP32 partials, combined in FP64) is used only to fill
// the GPU when the output has few tiles.
//
// Every mbarrier wait is bounded: on timeout the kernel records an error in
// the workspace status word, drains its own copies and MMAs (again with
// bounded waits), frees TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <atomic>
#include <mutex>

#include "common.cuh"
#include "ff.cuh"
#include "tc_ops.cuh"

namespace arma {

namespace tc {

constexpr int BM = 128, BN = 256, BK = 64, STAGES = 4;
constexpr int A_TILE = BM * BK * 2;           // 16 KiB
constexpr int B_TILE = BN * BK * 2;           // 32 KiB
constexpr int STAGE_BYTES = A_TILE + B_TILE;  // 48 KiB
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/;
constexpr int TMEM_COLS = 512;
constexpr int THREADS = 320;          // producer, MMA, 8 epilogue warps
constexpr int EPI_THREADS = 256;

// slice pairs (a, b) of the split tier, smallest contribution first
__constant__ int kTermA[6] = {2, 1, 0, 1, 0, 0};
__constant__ int kTermB[6] = {0, 1, 2, 0, 1, 0};

struct Params {
  int64_t m, n, k;          // logical problem
  int64_t mpad, npad, kp;   // padded slice extents (rows per slice, row stride in elements)
  int32_t terms;            // 1 (BF16) or 6 (split-BF16)
  int32_t splits;           // K chunks
  int32_t kb_per_split;     // k-blocks of BK per work item
  int32_t chunk_kb;         // k-blocks per TMEM accumulation chunk
  int32_t nchunks;          // chunks per work item
  int32_t tiles_m, tiles_n;
  // epilogue
  int32_t partial;          // 1: write FP32 partial P[split] (ld = m); 0: final D
  float* P;
  void* D; int64_t ldd; int32_t ddt;
  const void* C; int64_t ldc; int32_t cdt;
  double alpha, beta;
  float alpha_f, beta_f;    // alpha and beta rounded to float
  int32_t has_c;            // beta != 0
  float beta_h, beta_l;     // beta as an exact float pair (FP64 epilogue)
  const void* rs; int64_t rs_inc; int32_t rsdt;
  const void* cs; int64_t cs_inc; int32_t csdt;
  int32_t* status;          // workspace status word (0 = ok)
  int32_t sym;              // 1, 2: X X^T / X^T X, lower-triangle tiles only (tiles_m == 2 tiles_n)
  const int* skip;          // optional: return at once when *skip != 0
};

struct WorkItem {
  int32_t tm, tn, split;
};

// Symmetric products keep the tiles that reach the lower triangle: tile row
// tm (rows 128 tm ..) meets tile column tn (columns 256 tn ..) there iff
// tn <= tm / 2, so row tm holds tm / 2 + 1 tiles and the first x rows hold
// tri_rows(x) of them.
__device__ __forceinline__ int32_t tri_rows(int32_t x) {
  const int32_t y = x >> 1;
  return (x & 1) ? (y + 1) * (y + 1) : y * (y + 1);
}

__device__ __forceinline__ WorkItem work_item_sym(const Params& p, int32_t w) {
  // the same grouping as below, over the lower-triangle tiles: groups of 16
  // tile rows; inside a group, tile columns in order, each over the group's
  // rows that reach it
  const int32_t per_split = tri_rows(p.tiles_m);
  WorkItem it;
  it.split = w / per_split;
  const int32_t r = w - it.split * per_split;
  const int32_t G = 16;
  int32_t a = 0;
  while (a + G < p.tiles_m && tri_rows(a + G) <= r) a += G;
  const int32_t b = min(a + G, p.tiles_m), gsize = b - a;
  int32_t q = r - tri_rows(a);
  const int32_t full = a / 2 + 1;           // columns every row of the group reaches
  if (q < full * gsize) {
    it.tn = q / gsize;
    it.tm = a + q % gsize;
    return it;
  }
  q -= full * gsize;
  int32_t tn = full;
  while (q >= b - 2 * tn) { q -= b - 2 * tn; ++tn; }
  it.tn = tn;
  it.tm = 2 * tn + q;
  return it;
}

__device__ __forceinline__ WorkItem work_item(const Params& p, int32_t w) {
  if (p.sym) return work_item_sym(p, w);
  // split outermost; inside a split, groups of 16 tile rows sweep the tile
  // columns so that concurrently running CTAs share A and B panels in L2
  const int32_t per_split = p.tiles_m * p.tiles_n;
  WorkItem it;
  it.split = w / per_split;
  int32_t r = w - it.split * per_split;
  const int32_t G = 16;
  int32_t group = r / (G * p.tiles_n);
  int32_t first = group * G;
  int32_t gsize = min(G, p.tiles_m - first);
  int32_t q = r - group * G * p.tiles_n;
  it.tm = first + q % gsize;
  it.tn = q / gsize;
  return it;
}

__global__ void __launch_bounds__(THREADS, 1)
    gemm_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const __grid_constant__ Params p) {
  if (p.skip && *p.skip) return;            // uniform: before any barrier or TMEM allocation
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
  // bars: full[STAGES], empty[STAGES], tfull[2], tempty[2], done
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + STAGES);
  const uint32_t tfull0 = smem_u32(bars + 2 * STAGES), tempty0 = smem_u32(bars + 2 * STAGES + 2);
  const uint32_t done_bar = smem_u32(bars + 2 * STAGES + 4);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 5);
  volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int32_t kb_total = p.kb_per_split;
  const int32_t total_work = (p.sym ? tri_rows(p.tiles_m) : p.tiles_m * p.tiles_n) * p.splits;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(tfull0 + 8 * a, 1);
      mbar_init(tempty0 + 8 * a, EPI_THREADS);
    }
    mbar_init(done_bar, 1);
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      int32_t inflight[STAGES];
      for (int s = 0; s < STAGES; ++s) inflight[s] = -1;
      for (int32_t w = blockIdx.x; w < total_work && ok; w += gridDim.x) {
        WorkItem it = work_item(p, w);
        const int32_t kb0 = it.split * kb_total;
        for (int32_t c = 0; c < p.nchunks && ok; ++c) {
          const int32_t cb = c * p.chunk_kb;
          const int32_t ce = min(cb + p.chunk_kb, kb_total);
          for (int t = 0; t < p.terms && ok; ++t) {
            const int sa = p.terms == 1 ? 0 : kTermA[t], sb = p.terms == 1 ? 0 : kTermB[t];
            for (int32_t kb = cb; kb < ce; ++kb) {
              if (!mbar_wait(empty0 + 8 * stage, phase ^ 1u, abort)) { ok = false; break; }
              const uint32_t fb = full0 + 8 * stage;
              mbar_expect_tx(fb, STAGE_BYTES);
              const uint32_t sA = smem_u32(smem + stage * STAGE_BYTES);
              const int32_t x = (kb0 + kb) * BK;
              tma_load_2d(sA, &tmA, fb, x, (int32_t)(sa * p.mpad + (int64_t)it.tm * BM));
              tma_load_2d(sA + A_TILE, &tmB, fb, x, (int32_t)(sb * p.npad + (int64_t)it.tn * BN));
              inflight[stage] = (int32_t)phase;
              if (++stage == STAGES) { stage = 0; phase ^= 1u; }
            }
          }
        }
      }
      if (!ok) {
        // drain copies already issued (bounded) before the CTA can exit
        for (int s = 0; s < STAGES; ++s) {
          if (inflight[s] < 0) continue;
          for (uint32_t i = 0; i < WAIT_LIMIT && !mbar_try(full0 + 8 * s, (uint32_t)inflight[s]); ++i) {
          }
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(BM, BN);
      int stage = 0;
      uint32_t phase = 0;
      int acc = 0;
      uint32_t aphase = 0;
      bool ok = true;
      bool issued = false;
      for (int32_t w = blockIdx.x; w < total_work && ok; w += gridDim.x) {
        for (int32_t c = 0; c < p.nchunks && ok; ++c) {
          if (!mbar_wait(tempty0 + 8 * acc, aphase ^ 1u, abort)) { ok = false; break; }
          fence_after();
          const uint32_t dcol = tmem_base + (uint32_t)(acc * BN);
          uint32_t accumulate = 0;
          const int32_t cb = c * p.chunk_kb;
          const int32_t nkb = p.terms * (min(cb + p.chunk_kb, kb_total) - cb);
          for (int32_t j = 0; j < nkb; ++j) {
            if (!mbar_wait(full0 + 8 * stage, phase, abort)) { ok = false; break; }
            fence_after();
            const uint32_t sA = smem_u32(smem + stage * STAGE_BYTES);
            const uint32_t sB = sA + A_TILE;
            const uint64_t ad = sw128_desc(sA), bd = sw128_desc(sB);
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk) {
              // advance 16 BF16 (32 bytes) along K inside the swizzle atom
              mma_bf16(dcol, ad + (uint64_t)(2 * kk), bd + (uint64_t)(2 * kk), idesc, accumulate);
              accumulate = 1;
            }
            mma_commit(empty0 + 8 * stage);  // frees the smem stage when these MMAs finish
            issued = true;
            if (++stage == STAGES) { stage = 0; phase ^= 1u; }
          }
          if (!ok) break;
          mma_commit(tfull0 + 8 * acc);      // chunk accumulator ready for the epilogue
          if (++acc == 2) { acc = 0; aphase ^= 1u; }
        }
      }
      if (issued) {
        // all MMAs of this CTA complete before TMEM is released
        mma_commit(done_bar);
        for (uint32_t i = 0; i < WAIT_LIMIT && !mbar_try(done_bar, 0); ++i) {
        }
      }
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ epilogue
    // warp w: TMEM lane quarter w % 4, column half (w - 2) / 4; each thread
    // owns one output row and 128 consecutive columns of the tile
    const int quarter = warp & 3;
    const int half = (warp - 2) >> 2;
    const bool f64_out = p.ddt == ARMA_F64;
    const bool d_bf16 = p.ddt == ARMA_BF16;
    const bool has_c = p.C != nullptr && p.has_c;
    const float alpha_f = p.alpha_f, beta_f = has_c ? p.beta_f : 0.f;
    int acc = 0;
    uint32_t aphase = 0;
    for (int32_t w = blockIdx.x; w < total_work; w += gridDim.x) {
      WorkItem it = work_item(p, w);
      const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
      bool ok = true;
      if (p.nchunks > 1) {
        // chunks 0..n-2 are added into FP32 registers and released at once;
        // the last chunk is added too and the sums are written back into
        // its TMEM buffer, which the store loop below then reads
        float sum[BN / 2];
#pragma unroll
        for (int j = 0; j < BN / 2; ++j) sum[j] = 0.f;
        for (int32_t c = 0; c < p.nchunks; ++c) {
          ok = __all_sync(0xffffffffu, mbar_wait(tfull0 + 8 * acc, aphase, abort));
          if (!ok) break;
          fence_after();
          const uint32_t tb = tmem_base + lane_base + (uint32_t)(acc * BN + half * (BN / 2));
#pragma unroll
          for (int c0 = 0; c0 < BN / 2; c0 += 16) {
            float v[16];
            tmem_ld16(tb + (uint32_t)c0, v);
#pragma unroll
            for (int j = 0; j < 16; ++j) sum[c0 + j] += v[j];
          }
          if (c + 1 < p.nchunks) {
            fence_before();
            mbar_arrive(tempty0 + 8 * acc);
            if (++acc == 2) { acc = 0; aphase ^= 1u; }
          } else {
#pragma unroll
            for (int c0 = 0; c0 < BN / 2; c0 += 16) {
              float v[16];
#pragma unroll
              for (int j = 0; j < 16; ++j) v[j] = sum[c0 + j];
              tmem_st16(tb + (uint32_t)c0, v);
            }
            tmem_st_wait();
          }
        }
      } else {
        ok = __all_sync(0xffffffffu, mbar_wait(tfull0 + 8 * acc, aphase, abort));
        if (ok) fence_after();
      }
      if (!ok) break;
      // store loop: 16 columns at a time from TMEM (compact code)
      const int64_t row = (int64_t)it.tm * BM + quarter * 32 + lane;
      const bool row_ok = row < p.m;
      const int64_t colh = (int64_t)it.tn * BN + half * (BN / 2);
      const uint32_t tb = tmem_base + lane_base + (uint32_t)(acc * BN + half * (BN / 2));
      float rsf = 1.f;
      if (!p.partial && p.rs && row_ok) rsf = load_as<float>(p.rs, row * p.rs_inc, p.rsdt);
#pragma unroll 1
      for (int c0 = 0; c0 < BN / 2; c0 += 16) {
        float v[16];
        tmem_ld16(tb + (uint32_t)c0, v);
        const int64_t col0 = colh + c0;
        if (p.partial) {                  // uniform: the warp skips the rest together
          float* dst = p.P + (int64_t)it.split * p.m * p.n + row;
          if (row_ok)
#pragma unroll
            for (int j = 0; j < 16; ++j)
              if (col0 + j < p.n) dst[(col0 + j) * p.m] = v[j];
          continue;
        }
        // The product of these tiers is FP32-accurate, so beta*C is added in
        // FP32: C is read as a float with integer operations (an FP64 C
        // rounded to nearest, error <= 2^-24 |C|); FP64 results are widened
        // exactly by integer operations, so the epilogue issues no FP64
        // instruction.  An FP64 C outside float range is finished in FP64
        // behind a warp vote; its D element is stored only then, after C was
        // read again (C may alias D).
        // loads first (one uniform branch per storage type), then arithmetic
        float cf[16];
        uint32_t bad = 0u;
        if (has_c && p.cdt == ARMA_F64) {
          const double* Cd = static_cast<const double*>(p.C);
          double cd[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) cd[j] = (row_ok && col0 + j < p.n) ? Cd[row + (col0 + j) * p.ldc] : 0.0;
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            float f;
            if (!ff::d2f_rn(cd[j], f)) {
              bad |= 1u << j;
              f = 0.f;
            }
            cf[j] = f;
          }
        } else if (has_c && p.cdt == ARMA_F32) {
          const float* Cf = static_cast<const float*>(p.C);
#pragma unroll
          for (int j = 0; j < 16; ++j) cf[j] = (row_ok && col0 + j < p.n) ? Cf[row + (col0 + j) * p.ldc] : 0.f;
        } else if (has_c) {
          const unsigned short* Cb = static_cast<const unsigned short*>(p.C);
#pragma unroll
          for (int j = 0; j < 16; ++j)
            cf[j] = (row_ok && col0 + j < p.n) ? __uint_as_float((uint32_t)Cb[row + (col0 + j) * p.ldc] << 16) : 0.f;
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j) cf[j] = 0.f;
        }
        float rr[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          float r = alpha_f * v[j] * rsf;
          if (p.cs && col0 + j < p.n) r *= load_as<float>(p.cs, (col0 + j) * p.cs_inc, p.csdt);
          rr[j] = fmaf(beta_f, cf[j], r);
        }
        if (row_ok) {
          const int64_t at0 = row + col0 * p.ldd;
          if (f64_out) {
            double* D = static_cast<double*>(p.D) + at0;
#pragma unroll
            for (int j = 0; j < 16; ++j)
              if (col0 + j < p.n && !(bad & (1u << j))) D[j * p.ldd] = ff::f2d_exact(rr[j]);
          } else if (d_bf16) {
            __nv_bfloat16* D = static_cast<__nv_bfloat16*>(p.D) + at0;
#pragma unroll
            for (int j = 0; j < 16; ++j)
              if (col0 + j < p.n) D[j * p.ldd] = __float2bfloat16_rn(rr[j]);
          } else {
            float* D = static_cast<float*>(p.D) + at0;
#pragma unroll
            for (int j = 0; j < 16; ++j)
              if (col0 + j < p.n) D[j * p.ldd] = rr[j];
          }
        }
        if (__any_sync(0xffffffffu, bad != 0u)) {   // every lane of the warp gets here
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            if (!(bad & (1u << j))) continue;
            const int64_t col = col0 + j;
            float r = alpha_f * v[j] * rsf;
            if (p.cs) r *= load_as<float>(p.cs, col * p.cs_inc, p.csdt);
            const double t = (double)r + p.beta * static_cast<const double*>(p.C)[row + col * p.ldc];
            store_as<double>(p.D, row + col * p.ldd, p.ddt, t);
          }
        }
      }
      fence_before();
      mbar_arrive(tempty0 + 8 * acc);
      if (++acc == 2) { acc = 0; aphase ^= 1u; }
    }
  }

  fence_before();
  __syncthreads();
  if (threadIdx.x == 0 && *abort && p.status) atomicCAS(p.status, 0, (int32_t)ARMA_ERR_TIMEOUT);
  if (warp == 1) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS)
                 : "memory");
  }
}

// ---------------------------------------------------------------------------
// operand preparation: op(X) (R x K, any storage type, either orientation)
// -> T BF16 slices, K-major, rows padded to rpad, row stride kp (>= K, zero fill)
// ---------------------------------------------------------------------------
// (32-bit halves throughout: 64-bit integer operations issue to the FP64
// pipe on this GPU)
__device__ __forceinline__ void split3_f64(double x, uint16_t (&s)[3]) {
  const uint32_t uh = (uint32_t)__double2hiint(x), ul = (uint32_t)__double2loint(x);
  const uint32_t sign = uh & 0x80000000u;
  const int32_t e = (int32_t)((uh >> 20) & 0x7FF);
  if (e == 0 || e == 0x7FF) { s[0] = s[1] = s[2] = 0; return; }
  const uint32_t mh = (uh & 0xFFFFFu) | 0x100000u;   // significand bits 52..32
  const int32_t E = e - 1023;   // value = m * 2^(E - 52)
  s[0] = bf16_bits_of_window(sign, E - 7, (mh >> 13) & 0xFFu);
  s[1] = bf16_bits_of_window(sign, E - 15, (mh >> 5) & 0xFFu);
  s[2] = bf16_bits_of_window(sign, E - 23, ((mh << 3) | (ul >> 29)) & 0xFFu);
}


// double -> BF16, round to nearest even, integer operations only (32-bit
// halves)
__device__ __forceinline__ uint16_t d2bf16_rn(double x) {
  const uint32_t uh = (uint32_t)__double2hiint(x), ul = (uint32_t)__double2loint(x);
  const uint16_t sign = (uint16_t)((uh >> 16) & 0x8000u);
  const int32_t e = (int32_t)((uh >> 20) & 0x7FF);
  if (e == 0x7FF) return (uint16_t)(sign | 0x7F80u | (((uh & 0xFFFFFu) | ul) ? 0x40u : 0u));
  int32_t be = e - 1023 + 127;
  if (e == 0 || be <= 0) return sign;                 // zero / below BF16 normal range
  uint32_t keep = (uh & 0xFFFFFu) >> 13;              // 7 fraction bits
  const uint32_t rh = uh & 0x1FFFu;                   // remainder: rh:ul, half = 0x1000:0
  const bool above = rh > 0x1000u || (rh == 0x1000u && ul != 0u);
  const bool tie = rh == 0x1000u && ul == 0u;
  if (above || (tie && (keep & 1u))) ++keep;
  if (keep == 128u) { keep = 0u; ++be; }
  if (be >= 255) return (uint16_t)(sign | 0x7F80u);
  return (uint16_t)(sign | ((uint32_t)be << 7) | keep);
}

struct PrepArgs {
  const void* X; int64_t ldx; int32_t xdt, trans;  // op(X)(r, l) = trans ? X[l + r*ldx] : X[r + l*ldx]
  int64_t R, K, rpad, kp;
  int32_t slices;        // 1 or 3
  __nv_bfloat16* out;    // [slices][rpad][kp]
  const int* skip;       // optional: return at once when *skip != 0
};

// 32 x 32 tiles through shared memory: read along X's contiguous index,
// write along K.  The storage-type branch sits outside the row loop, so a
// thread's four loads are in flight together.
template <typename XT>
__device__ __forceinline__ void prep_tile_load(const PrepArgs& a, int64_t r0, int64_t l0, int tx, int ty,
                                               uint16_t (&t)[3][32][33]) {
  XT x[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int q = ty + 8 * k;
    int64_t r, l;
    if (a.trans) { l = l0 + tx; r = r0 + q; } else { r = r0 + tx; l = l0 + q; }
    x[k] = (r < a.R && l < a.K) ? static_cast<const XT*>(a.X)[a.trans ? l + r * a.ldx : r + l * a.ldx] : XT(0);
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int q = ty + 8 * k;
    uint16_t sl[3] = {0, 0, 0};
    if constexpr (sizeof(XT) == 8) {
      if (a.slices == 1) sl[0] = d2bf16_rn(x[k]);
      else split3_f64(x[k], sl);
    } else if constexpr (sizeof(XT) == 4) {
      if (a.slices == 1) sl[0] = __bfloat16_as_ushort(__float2bfloat16_rn(x[k]));
      else split3_f32(x[k], sl);
    } else {
      sl[0] = x[k];                      // BF16 is its own first slice
    }
    const int rr = a.trans ? q : tx, ll = a.trans ? tx : q;
#pragma unroll
    for (int u = 0; u < 3; ++u)
      if (u < a.slices) t[u][rr][ll] = sl[u];
  }
}

__global__ void __launch_bounds__(256) prep_kernel(const __grid_constant__ PrepArgs a) {
  __shared__ uint16_t t[3][32][33];
  if (a.skip && *a.skip) return;
  if (a.slices != 1 && a.slices != 3) return;   // the tile above holds at most 3 slices
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t r0 = (int64_t)blockIdx.x * 32, l0 = (int64_t)blockIdx.y * 32;
  if (a.xdt == ARMA_F64) prep_tile_load<double>(a, r0, l0, tx, ty, t);
  else if (a.xdt == ARMA_F32) prep_tile_load<float>(a, r0, l0, tx, ty, t);
  else prep_tile_load<uint16_t>(a, r0, l0, tx, ty, t);
  __syncthreads();
  for (int q = ty; q < 32; q += 8) {
    const int64_t r = r0 + q, l = l0 + tx;
    if (r < a.rpad && l < a.kp) {
      for (int u = 0; u < a.slices; ++u) {
        uint16_t v = (r < a.R && l < a.K) ? t[u][q][tx] : (uint16_t)0;
        reinterpret_cast<uint16_t*>(a.out)[((int64_t)u * a.rpad + r) * a.kp + l] = v;
      }
    }
  }
}

// op(X) contiguous along K (the common case): each thread converts 8
// consecutive K elements of one row and writes one 16-byte vector per slice.
// The storage-type branch sits outside the element loop, so the eight loads
// of a thread are in flight together.
template <typename XT>
__device__ __forceinline__ void prep_group(const PrepArgs& a, int64_t r, int64_t l0, uint16_t (&s0)[8],
                                           uint16_t (&s1)[8], uint16_t (&s2)[8]) {
  const XT* X = static_cast<const XT*>(a.X) + r * a.ldx;
  XT x[8];
  // a whole aligned group inside the matrix: 16-byte loads (the same values)
  const bool whole = r < a.R && l0 + 8 <= a.K && (reinterpret_cast<uintptr_t>(X + l0) & 15u) == 0;
  bool done = false;
  if constexpr (sizeof(XT) == 8) {
    if (whole) {
      const double2* p = reinterpret_cast<const double2*>(X + l0);
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        const double2 v = __ldg(p + h);
        x[2 * h] = v.x;
        x[2 * h + 1] = v.y;
      }
      done = true;
    }
  } else if constexpr (sizeof(XT) == 4) {
    if (whole) {
      const float4* p = reinterpret_cast<const float4*>(X + l0);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const float4 v = __ldg(p + h);
        x[4 * h] = v.x;
        x[4 * h + 1] = v.y;
        x[4 * h + 2] = v.z;
        x[4 * h + 3] = v.w;
      }
      done = true;
    }
  }
  if (!done) {
#pragma unroll
    for (int e = 0; e < 8; ++e) x[e] = (r < a.R && l0 + e < a.K) ? X[l0 + e] : XT(0);
  }
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    uint16_t sl[3] = {0, 0, 0};
    if constexpr (sizeof(XT) == 8) {
      if (a.slices == 1) sl[0] = d2bf16_rn(x[e]);
      else split3_f64(x[e], sl);
    } else if constexpr (sizeof(XT) == 4) {
      if (a.slices == 1) sl[0] = __bfloat16_as_ushort(__float2bfloat16_rn(x[e]));
      else split3_f32(x[e], sl);
    } else {
      sl[0] = x[e];                      // BF16 is its own first slice
    }
    s0[e] = sl[0]; s1[e] = sl[1]; s2[e] = sl[2];
  }
}

__global__ void __launch_bounds__(256) prep_kcontig_kernel(const __grid_constant__ PrepArgs a) {
  if (a.slices != 1 && a.slices != 3) return;
  if (a.skip && *a.skip) return;
  // 32-bit index arithmetic (the host keeps rpad * kp / 8 below 2^31): a
  // 64-bit division per group costs more than the conversion itself
  const uint32_t groups = (uint32_t)(a.kp / 8);
  const uint32_t total = (uint32_t)(a.rpad * (a.kp / 8));
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    const uint32_t rr = t / groups;
    const int64_t r = rr, l0 = (int64_t)(t - rr * groups) * 8;
    __align__(16) uint16_t s0[8];
    __align__(16) uint16_t s1[8];
    __align__(16) uint16_t s2[8];
    if (a.xdt == ARMA_F64) prep_group<double>(a, r, l0, s0, s1, s2);
    else if (a.xdt == ARMA_F32) prep_group<float>(a, r, l0, s0, s1, s2);
    else prep_group<uint16_t>(a, r, l0, s0, s1, s2);
    uint4* o0 = reinterpret_cast<uint4*>(reinterpret_cast<uint16_t*>(a.out) + r * a.kp + l0);
    *o0 = *reinterpret_cast<const uint4*>(s0);
    if (a.slices == 3) {
      uint4* o1 = reinterpret_cast<uint4*>(reinterpret_cast<uint16_t*>(a.out) + (a.rpad + r) * a.kp + l0);
      uint4* o2 = reinterpret_cast<uint4*>(reinterpret_cast<uint16_t*>(a.out) + (2 * a.rpad + r) * a.kp + l0);
      *o1 = *reinterpret_cast<const uint4*>(s1);
      *o2 = *reinterpret_cast<const uint4*>(s2);
    }
  }
}

// D = alpha * diag(r) * (sum_s P_s) * diag(c) + beta * C, partials summed in FP64
struct CombineArgs {
  int64_t m, n;
  int32_t splits;
  const float* P;
  void* D; int64_t ldd; int32_t ddt;
  const void* C; int64_t ldc; int32_t cdt;
  double alpha, beta;
  const void* rs; int64_t rs_inc; int32_t rsdt;
  const void* cs; int64_t cs_inc; int32_t csdt;
  int32_t sym;   // partials hold the lower-triangle tiles only
  const int* skip;
};

__global__ void __launch_bounds__(256) combine_kernel(const __grid_constant__ CombineArgs a) {
  if (a.skip && *a.skip) return;
  const int64_t total = a.m * a.n;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t col = t / a.m, row = t - col * a.m;
    if (a.sym && row < col) continue;   // mirrored afterwards
    double s = 0.0;
    for (int k = 0; k < a.splits; ++k) s += (double)a.P[(int64_t)k * total + t];
    double r = a.alpha * s;
    if (a.rs) r *= load_as<double>(a.rs, row * a.rs_inc, a.rsdt);
    if (a.cs) r *= load_as<double>(a.cs, col * a.cs_inc, a.csdt);
    if (a.C && a.beta != 0.0) r += a.beta * load_as<double>(a.C, row + col * a.ldc, a.cdt);
    store_as<double>(a.D, row + col * a.ldd, a.ddt, r);
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct Geometry {
  int32_t terms;    // slice products accumulated (1 or 6)
  int32_t slices;   // BF16 slices stored per operand (1 or 3)
  int32_t splits, kb_per_split, chunk_kb, nchunks, tiles_m, tiles_n;
  int64_t mpad, npad, kp;
  int64_t a_bytes, b_bytes, p_bytes;
};

// sym: op(B)^T is op(A), so one prepared operand serves both TMA maps; its
// rows are padded to a multiple of both tile heights
Geometry geometry(int64_t m, int64_t n, int64_t k, int32_t tier, bool sym = false, bool nosplit = false,
                  int32_t req = 0) {
  Geometry g;
  g.terms = tier == ARMA_TIER_SPLIT_BF16 ? 6 : 1;
  g.slices = tier == ARMA_TIER_SPLIT_BF16 ? 3 : 1;
  g.kp = (k + 7) / 8 * 8;
  g.mpad = sym ? (m + BN - 1) / BN * BN : (m + BM - 1) / BM * BM;
  g.npad = sym ? g.mpad : (n + BN - 1) / BN * BN;
  g.tiles_m = (int32_t)(g.mpad / BM);
  g.tiles_n = (int32_t)(g.npad / BN);
  const int64_t kb = (k + BK - 1) / BK;
  // split K over CTAs only when the output has too few tiles to fill the GPU
  // (or as many splits as asked for)
  int64_t splits = 1;
  const int64_t tiles = (int64_t)g.tiles_m * g.tiles_n;
  if (!nosplit && req > 0) splits = req;
  else
    while (!nosplit && tiles * splits < 148 && kb / (splits * 2) >= 4) splits *= 2;
  if (splits > kb) splits = kb > 0 ? kb : 1;
  g.splits = (int32_t)(splits < 1 ? 1 : splits);
  g.kb_per_split = (int32_t)((kb + g.splits - 1) / g.splits);
  // accumulate at most 256 of K per TMEM chunk for the split tier
  g.chunk_kb = g.terms > 1 ? 256 / BK : g.kb_per_split;
  if (g.chunk_kb < 1) g.chunk_kb = 1;
  g.nchunks = (g.kb_per_split + g.chunk_kb - 1) / g.chunk_kb;
  g.a_bytes = (int64_t)g.slices * g.mpad * g.kp * 2;
  g.b_bytes = sym ? 0 : (int64_t)g.slices * g.npad * g.kp * 2;
  g.p_bytes = g.splits > 1 ? (int64_t)g.splits * m * n * 4 : 0;
  return g;
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

bool make_map(CUtensorMap* map, const void* base, int64_t kp, int64_t rows, int box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)kp, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(kp * 2)};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// A map straight over the caller's BF16 operand when it is already K-major
// (element (row r, k) at base[k + r * ld]): no preparation pass.  Rows past
// `rows` and K past `kdim` are outside the tensor and read as zero.
bool make_map_direct(CUtensorMap* map, const void* base, int64_t kdim, int64_t rows, int64_t ld, int box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)kdim, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// a BF16 operand the kernel can read in place: one slice (BF16 tier), K-major,
// 16-byte aligned base and a leading dimension of a multiple of 8 elements
// (TMA strides are multiples of 16 bytes)
bool direct_operand(const void* X, int32_t dt, int64_t ld, bool kmajor, int32_t slices) {
  return slices == 1 && dt == ARMA_BF16 && kmajor && ld % 8 == 0 && ld >= 8 &&
         (reinterpret_cast<uintptr_t>(X) & 15u) == 0;
}

}  // namespace tc

bool gemm_tc_supported(const GemmArgs& a) {
  if (a.tier != ARMA_TIER_SPLIT_BF16 && a.tier != ARMA_TIER_BF16) return false;
  if (a.m < 1 || a.n < 1 || a.k < 1) return false;
  if (a.m > (1ll << 30) || a.n > (1ll << 30) || a.k > (1ll << 30)) return false;
  if (!a.scratch) return false;
  tc::Geometry g = tc::geometry(a.m, a.n, a.k, a.tier, a.sym != 0, a.nosplit != 0, a.split_req);
  return a.scratch_bytes >= g.a_bytes + g.b_bytes + g.p_bytes + 1024;
}

int gemm_tc_splits(int64_t m, int64_t n, int64_t k, int32_t tier, bool sym, bool nosplit, int32_t split_req) {
  if (m < 1 || n < 1 || k < 1) return 1;
  return tc::geometry(m, n, k, tier, sym, nosplit, split_req).splits;
}

int64_t gemm_tc_scratch_bytes(int64_t m, int64_t n, int64_t k, int32_t tier, int32_t split_req) {
  if (tier != ARMA_TIER_SPLIT_BF16 && tier != ARMA_TIER_BF16) return 0;
  if (m < 1 || n < 1 || k < 1) return 0;
  tc::Geometry g = tc::geometry(m, n, k, tier, false, false, split_req);
  return g.a_bytes + g.b_bytes + g.p_bytes + 1024;
}

cudaError_t launch_gemm_tc(const GemmArgs& a, cudaStream_t s, int* launches) {
  using namespace tc;
  const bool sym = a.sym != 0;
  Geometry g = geometry(a.m, a.n, a.k, a.tier, sym, a.nosplit != 0, a.split_req);
  char* base = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(a.scratch) + 255) & ~uintptr_t(255));
  __nv_bfloat16* As = reinterpret_cast<__nv_bfloat16*>(base);
  __nv_bfloat16* Bs = reinterpret_cast<__nv_bfloat16*>(base + ((g.a_bytes + 255) / 256) * 256);
  float* P = reinterpret_cast<float*>(base + ((g.a_bytes + 255) / 256) * 256 + ((g.b_bytes + 255) / 256) * 256);
  if (g.slices != 1 && g.slices != 3) return cudaErrorInvalidValue;
  // operand preparation: op(A) rows = m, op(B)^T rows = n, both K-major
  PrepArgs pa;
  pa.X = a.A; pa.ldx = a.lda; pa.xdt = a.adt; pa.trans = a.ta;
  pa.R = a.m; pa.K = a.k; pa.rpad = g.mpad; pa.kp = g.kp; pa.slices = g.slices; pa.out = As;
  pa.skip = a.skip;
  const int sms0 = device_sm_count();
  auto prep = [&](const PrepArgs& pp) {
    if (pp.trans && pp.rpad * (pp.kp / 8) < (1ll << 31)) {
      const int64_t total = pp.rpad * (pp.kp / 8);
      int64_t blocks = (total + 255) / 256, cap = (int64_t)sms0 * 8;
      prep_kcontig_kernel<<<(unsigned)(blocks < cap ? blocks : cap), 256, 0, s>>>(pp);
    } else {
      dim3 gg((unsigned)((pp.rpad + 31) / 32), (unsigned)((pp.kp + 31) / 32));
      prep_kernel<<<gg, 256, 0, s>>>(pp);
    }
  };
  // BF16 operands that are already K-major (op(A) = A^T, op(B) = B) feed
  // TMA in place: no preparation pass over them
  const bool directA = !sym && direct_operand(a.A, a.adt, a.lda, a.ta != 0, g.slices);
  const bool directB = !sym && direct_operand(a.B, a.bdt, a.ldb, a.tb == 0, g.slices);
  if (!directA) {
    prep(pa);
    if (launches) ++*launches;
  }
  // op(B)^T (n x k): element (j, l) = op(B)(l, j) = tb ? B[j + l*ldb] : B[l + j*ldb]
  PrepArgs pb;
  pb.X = a.B; pb.ldx = a.ldb; pb.xdt = a.bdt; pb.trans = a.tb ? 0 : 1;
  pb.R = a.n; pb.K = a.k; pb.rpad = g.npad; pb.kp = g.kp; pb.slices = g.slices; pb.out = Bs;
  pb.skip = a.skip;
  if (!sym && !directB) {
    prep(pb);
    if (launches) ++*launches;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;

  CUtensorMap mapA, mapB;
  if (directA ? !make_map_direct(&mapA, a.A, a.k, a.m, a.lda, BM)
              : !make_map(&mapA, As, g.kp, (int64_t)g.slices * g.mpad, BM))
    return cudaErrorInvalidValue;
  if (directB ? !make_map_direct(&mapB, a.B, a.k, a.n, a.ldb, BN)
              : !make_map(&mapB, sym ? As : Bs, g.kp, (int64_t)g.slices * g.npad, BN))
    return cudaErrorInvalidValue;

  Params p;
  memset(&p, 0, sizeof p);
  p.m = a.m; p.n = a.n; p.k = a.k;
  p.mpad = g.mpad; p.npad = g.npad; p.kp = g.kp;
  p.terms = g.terms; p.splits = g.splits; p.kb_per_split = g.kb_per_split;
  p.chunk_kb = g.chunk_kb; p.nchunks = g.nchunks;
  p.tiles_m = g.tiles_m; p.tiles_n = g.tiles_n;
  p.partial = g.splits > 1 ? 1 : 0;
  p.P = P;
  p.D = a.D; p.ldd = a.ldd; p.ddt = a.ddt;
  p.C = a.C; p.ldc = a.ldc; p.cdt = a.cdt;
  p.alpha = a.alpha; p.beta = a.beta;
  p.alpha_f = (float)a.alpha; p.beta_f = (float)a.beta;
  p.has_c = a.C != nullptr && a.beta != 0.0;
  p.beta_h = (float)a.beta;
  p.beta_l = (float)(a.beta - (double)p.beta_h);
  p.rs = a.rs; p.rs_inc = a.rs_inc; p.rsdt = a.rsdt;
  p.cs = a.cs; p.cs_inc = a.cs_inc; p.csdt = a.csdt;
  p.status = a.status;
  p.sym = sym ? 1 : 0;
  p.skip = a.skip;

  static std::atomic<bool> attr_set[64];
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (!attr_set[dev].load(std::memory_order_acquire)) {
    e = cudaFuncSetAttribute(gemm_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    if (e != cudaSuccess) return e;
    attr_set[dev].store(true, std::memory_order_release);
  }
  const int64_t per_split = sym ? (g.tiles_m / 2) * (int64_t)(g.tiles_m / 2 + 1) : (int64_t)g.tiles_m * g.tiles_n;
  const int64_t work = per_split * g.splits;
  const int sms = device_sm_count();
  int ctas = sms;
  if (a.max_ctas > 0 && a.max_ctas < ctas) ctas = a.max_ctas;
  const int grid = (int)(work < ctas ? work : ctas);
  gemm_tc_kernel<<<grid, THREADS, SMEM_BYTES, s>>>(mapA, mapB, p);
  if (launches) ++*launches;
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (g.splits == 1) return a.sym == 1 ? launch_mirror_lower(a.D, a.n, a.ldd, a.ddt, s, launches) : e;

  CombineArgs c;
  c.m = a.m; c.n = a.n; c.splits = g.splits; c.P = P;
  c.D = a.D; c.ldd = a.ldd; c.ddt = a.ddt;
  c.C = a.C; c.ldc = a.ldc; c.cdt = a.cdt;
  c.alpha = a.alpha; c.beta = a.beta;
  c.rs = a.rs; c.rs_inc = a.rs_inc; c.rsdt = a.rsdt;
  c.cs = a.cs; c.cs_inc = a.cs_inc; c.csdt = a.csdt;
  c.sym = sym ? 1 : 0;
  c.skip = a.skip;
  const int64_t total = a.m * a.n;
  int64_t blocks = (total + 255) / 256, cap = (int64_t)sms * 8;
  combine_kernel<<<(unsigned)(blocks < cap ? blocks : cap), 256, 0, s>>>(c);
  if (launches) ++*launches;
  e = cudaGetLastError();
  if (e != cudaSuccess || a.sym != 1) return e;
  return launch_mirror_lower(a.D, a.n, a.ldd, a.ddt, s, launches);
}

}  // namespace arma
