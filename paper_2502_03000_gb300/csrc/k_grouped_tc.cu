// Grouped products on the tensor cores (tcgen05, sm_103a): the batched form
// of the folded product D_g = alpha * op(A_g) op(B_g) + beta * C_g with the
// diagonal-only trace t_g = trace(op(A_g) op(B_g)) (Sec. II xGEMM paragraph,
// Sec. III (5)), for thousands of problems of uneven sizes in two launches.
//
// 1. pack   one CTA per (problem, operand) copies op(A_g) and op(B_g)^T (both
//           K-contiguous, leading dimensions of any value) into one packed
//           array per operand: K-block-major BF16 rows of 64 (K block kb of a
//           problem's R rows at rows p_g + kb R .. + R - 1, K past k_g zero).
//           FP32 operands are split exactly into three BF16 slices (Henry et
//           al. 2019, the BF16 work the paper cites), one array per slice.
//           Every row of 64 is one 128-byte line, so the product kernel
//           reads the operands with TMA whatever the caller's strides.
// 2. product  one persistent CTA per SM walks its share of the host-built
//           list of 128 x 128 output tiles (ordered by decreasing work; CTA c
//           takes positions c, 2G-1-c, 2G+c, ... so that the long tiles
//           spread evenly).  Every role walks the same sequence:
//   warp 0     TMA producer: per K block one box of op(A) rows and one of
//              op(B)^T rows per slice into a ring of shared-memory stages
//              (128-byte swizzle); the box is the smallest of 16, 32, 64 and
//              128 rows that covers the tile's rows
//   warp 1     TMEM owner (four 128-column FP32 accumulators, all of TMEM)
//              and MMA issuer: tile i of the CTA's sequence into accumulator
//              i % 4; one tcgen05.mma per 16 of K and slice product (6
//              products of order <= 2 for three slices, smallest first)
//   warps 2..17 four epilogue groups of four warps (one per TMEM lane
//              quarter); group e drains the tiles i = e (mod 4), so four
//              tiles' epilogues are in flight: the tile's C lines into L2
//              while its MMAs run, then per 16 columns tcgen05.ld, C, alpha,
//              beta*C, D, and the diagonal of diagonal tiles for the traces
// Rows of a box past the problem's rows (and stale shared memory past a
// short box) only reach output rows and columns that are never stored: each
// output element depends on its own row of op(A) and column of op(B) alone.
// Every mbarrier wait is bounded: on timeout the CTA records
// ARMA_ERR_TIMEOUT in the status word, waits (bounded) for its issued copies
// and MMAs, frees TMEM and returns.
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <atomic>

#include "common.cuh"
#include "grouped.h"
#include "tc_ops.cuh"

namespace arma {
namespace tc {
PFN_cuTensorMapEncodeTiled_v12000 encode_fn();   // k_gemm_tc.cu
}

namespace {

using namespace tc;

constexpr int GM = 128, GN = 128, GK = kPackK;   // output tile and K block
constexpr int GBOX = GM * GK * 2;               // one 128-row BF16 operand box: 16 KiB
constexpr int NACC = 4;                         // accumulators = epilogue groups
constexpr int NEPI = 128;                       // threads of one epilogue group (4 warps)
constexpr int GTHREADS = 64 + NACC * NEPI;      // 18 warps
constexpr int GTMEM = NACC * GN;                // four 128 x 128 FP32 accumulators: all 512 columns

template <int S>
__host__ __device__ constexpr int gstages() { return S == 1 ? 6 : 2; }
template <int S>
__host__ __device__ constexpr int stage_bytes() { return 2 * S * GBOX; }   // A slices, then B slices
template <int S>
__host__ __device__ constexpr int smem_bytes() { return gstages<S>() * stage_bytes<S>() + 1024 + 256; }

// box heights and the tensor map of each
constexpr int kBoxes = 4;
__host__ __device__ constexpr int box_index(int rows) { return rows <= 16 ? 0 : rows <= 32 ? 1 : rows <= 64 ? 2 : 3; }

struct PackedMaps {
  CUtensorMap a[kBoxes];
  CUtensorMap b[kBoxes];
};

// position of CTA c's walk over the ordered tile list (G CTAs) in round
// `round`: rounds of G tiles, alternate rounds reversed
__device__ __forceinline__ int64_t walk(int64_t round, int c, int G) {
  return round * G + ((round & 1) ? (G - 1 - c) : c);
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

// ---------------------------------------------------------------------------
// pack: the work is the host-built list of runs of whole rows of one operand
// (0: op(A), 1: op(B)^T) of one problem, with all their K blocks; warp w of
// the grid takes runs w, w + W, ...  Pair t of a run is (row t / nkb, K
// block t % nkb), K block fastest, so a warp reads consecutive source
// memory.  Packed row (kb, r) of a problem lies at p_g + kb R + r.  Elements
// past K are zero.  All loads of a step are issued before their data is used.
//   BF16: a group of 8 lanes copies one pair per step, 16 bytes a lane, from
//         aligned 16-byte loads of the source row, each lane joining its
//         chunk with the next lane's (rows may start at any element).  Only
//         chunks that hold an element of the row are loaded.
//   FP32: a warp per pair, a float pair per lane (one 8-byte load when the
//         row starts are even), then the exact three-way split; pairs taken
//         K block by K block, so consecutive pairs write consecutive rows of
//         the three slice arrays.
// ---------------------------------------------------------------------------
constexpr int PU = 2;     // BF16: pairs per lane group and step
constexpr int PU32 = 16;  // FP32: pairs per warp and step

// bytes sh .. sh + 15 of the 32 bytes c (sh even): shift by 2 words, by one
// word, then by 16 bits
__device__ __forceinline__ uint4 window16(const uint32_t (&c)[8], uint32_t sh) {
  uint32_t d[6], e[5];
#pragma unroll
  for (int i = 0; i < 6; ++i) d[i] = (sh & 8u) ? c[i + 2] : c[i];
#pragma unroll
  for (int i = 0; i < 5; ++i) e[i] = (sh & 4u) ? d[i + 1] : d[i];
  const uint32_t fs = (sh & 2u) * 8u;
  return make_uint4(__funnelshift_r(e[0], e[1], fs), __funnelshift_r(e[1], e[2], fs),
                    __funnelshift_r(e[2], e[3], fs), __funnelshift_r(e[3], e[4], fs));
}

// one run of BF16 pairs
__device__ __forceinline__ void pack_run_bf16(const char* X, int64_t ld, int64_t R, int64_t K, int64_t p0,
                                              int32_t r0, int64_t T, uint32_t nkb, uint4* out, int lane) {
  const int gsub = lane >> 3, j = lane & 7;
  for (int64_t t0 = 0; t0 < T; t0 += 4 * PU) {
    uint4 q[PU], qx[PU];
    int64_t dst[PU];
    uint32_t shv[PU];
    int nvv[PU];
#pragma unroll
    for (int u = 0; u < PU; ++u) {
      const int64_t t = t0 + 4 * u + gsub;
      const bool rv = t < T;
      const uint32_t tu = (uint32_t)(rv ? t : 0);
      const uint32_t rl = tu / nkb, kb = tu - rl * nkb;
      const int64_t r = r0 + rl;
      dst[u] = rv ? p0 + (int64_t)kb * R + r : -1;
      const int nv = rv ? (int)min((int64_t)GK, K - (int64_t)GK * kb) : 0;   // elements of this pair
      nvv[u] = nv;
      const char* A = X + 2 * (r * ld + (int64_t)GK * kb);
      const uint32_t sh = (uint32_t)(reinterpret_cast<uintptr_t>(A) & 15u);
      shv[u] = sh;
      const char* a0 = A - sh;
      const char* last = A + 2 * nv - 1;
      q[u] = make_uint4(0u, 0u, 0u, 0u);
      qx[u] = q[u];
      if (nv > 0 && a0 + 16 * j <= last) q[u] = __ldg(reinterpret_cast<const uint4*>(a0 + 16 * j));
      if (nv > 0 && j == 7 && a0 + 128 <= last) qx[u] = __ldg(reinterpret_cast<const uint4*>(a0 + 128));
    }
#pragma unroll
    for (int u = 0; u < PU; ++u) {
      uint4 nx;
      nx.x = __shfl_down_sync(0xffffffffu, q[u].x, 1, 8);
      nx.y = __shfl_down_sync(0xffffffffu, q[u].y, 1, 8);
      nx.z = __shfl_down_sync(0xffffffffu, q[u].z, 1, 8);
      nx.w = __shfl_down_sync(0xffffffffu, q[u].w, 1, 8);
      if (j == 7) nx = qx[u];
      const uint32_t c[8] = {q[u].x, q[u].y, q[u].z, q[u].w, nx.x, nx.y, nx.z, nx.w};
      uint4 w = window16(c, shv[u]);
      if (8 * j + 8 > nvv[u]) {   // past the pair's valid elements: zero
        uint32_t ww[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int tt = 0; tt < 4; ++tt) {
          const int e = 8 * j + 2 * tt;
          if (e >= nvv[u]) ww[tt] = 0u;
          else if (e + 1 >= nvv[u]) ww[tt] &= 0xFFFFu;
        }
        w = make_uint4(ww[0], ww[1], ww[2], ww[3]);
      }
      if (dst[u] >= 0) out[dst[u] * 8 + j] = w;
    }
  }
}

// one run of FP32 pairs, split into S slices: K block by K block, rows r0 ..
// r0 + nr - 1 within each, a source pointer walked from pair to pair
template <int S>
__device__ __forceinline__ void pack_run_f32(const float* X, int64_t ld, int64_t R, int64_t K, int64_t p0,
                                             int32_t r0, int32_t nr, int64_t T, int64_t rows, uint32_t* out,
                                             int lane) {
  const bool pairs = (ld & 1) == 0 && (reinterpret_cast<uintptr_t>(X) & 7u) == 0;
  int32_t rl = 0;
  int64_t c = 2 * lane, base = p0 + r0;   // base: packed row of (this K block, row r0)
  const float* src = X + (int64_t)r0 * ld + c;
  for (int64_t t0 = 0; t0 < T; t0 += PU32) {
    float x0[PU32], x1[PU32];
    const int32_t rl0 = rl;        // the walk's state at the step's first pair,
    const int64_t base0 = base;    // replayed for the stores
#pragma unroll
    for (int u = 0; u < PU32; ++u) {
      x0[u] = x1[u] = 0.f;
      if (t0 + u < T && c < K) {
        if (pairs && c + 1 < K) {
          const float2 f = __ldg(reinterpret_cast<const float2*>(src));
          x0[u] = f.x;
          x1[u] = f.y;
        } else {
          x0[u] = __ldg(src);
          x1[u] = c + 1 < K ? __ldg(src + 1) : 0.f;
        }
      }
      // the next pair: the next row of this K block, or row r0 of the next
      src += ld;
      if (++rl == nr) {
        rl = 0;
        c += GK;
        base += R;
        src = X + (int64_t)r0 * ld + c;
      }
    }
    int32_t rs = rl0;
    int64_t bs = base0;
#pragma unroll
    for (int u = 0; u < PU32; ++u) {
      if (t0 + u >= T) break;
      uint16_t a0[3], a1[3];
      split3_rn(x0[u], a0);
      split3_rn(x1[u], a1);
      const int64_t dst = bs + rs;
#pragma unroll
      for (int sl = 0; sl < S; ++sl)
        out[((int64_t)sl * rows + dst) * (GK / 2) + lane] = (uint32_t)a0[sl] | ((uint32_t)a1[sl] << 16);
      if (++rs == nr) {
        rs = 0;
        bs += R;
      }
    }
  }
}

template <typename AT, int S>
__global__ void __launch_bounds__(256, sizeof(AT) == 2 ? 4 : 3) grouped_pack_kernel(const __grid_constant__ GroupedArgs g) {
  const int lane = threadIdx.x & 31;
  const int64_t W = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t it = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; it < g.n_items; it += W) {
    const int32_t code = g.pack_items[3 * it], r0 = g.pack_items[3 * it + 1], nr = g.pack_items[3 * it + 2];
    const int64_t pi = code >> 1;
    const int op = code & 1;
    const GroupedProblem& P = g.probs[pi];
    const int64_t R = op ? P.n : P.m, K = P.k;
    const void* X = op ? P.B : P.A;
    const int64_t ld = op ? P.ldb : P.lda;
    const int64_t p0 = op ? P.pb : P.pa;
    const uint32_t nkb = (uint32_t)((K + GK - 1) / GK);
    const int64_t T = (int64_t)nr * nkb;
    if constexpr (sizeof(AT) == 2)
      pack_run_bf16(static_cast<const char*>(X), ld, R, K, p0, r0, T, nkb,
                    static_cast<uint4*>(op ? g.pack_b : g.pack_a), lane);
    else
      pack_run_f32<S>(static_cast<const float*>(X), ld, R, K, p0, r0, nr, T, op ? g.rows_b : g.rows_a,
                      static_cast<uint32_t*>(op ? g.pack_b : g.pack_a), lane);
  }
}

// 16 FP32 values of C along a row: x[j] = C[j * ldc] for j < n (0 past n
// or when !ok); no predicates when all 16 are wanted
__device__ __forceinline__ void load_c16(float (&x)[16], const float* C, int64_t ldc, bool ok, int n) {
  if (ok && n >= 16) {
#pragma unroll
    for (int j = 0; j < 16; ++j) x[j] = __ldg(C + j * ldc);
  } else {
#pragma unroll
    for (int j = 0; j < 16; ++j) x[j] = (ok && j < n) ? __ldg(C + j * ldc) : 0.f;
  }
}

template <int S>
__global__ void __launch_bounds__(GTHREADS, 1)
    grouped_packed_kernel(const __grid_constant__ GroupedArgs g, const __grid_constant__ PackedMaps maps) {
  constexpr int STAGES = gstages<S>();
  constexpr int SB = stage_bytes<S>();
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * SB);
  // bars: full[STAGES], empty[STAGES], tfull[NACC], tempty[NACC], done
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + STAGES);
  const uint32_t tfull0 = smem_u32(bars + 2 * STAGES), tempty0 = smem_u32(bars + 2 * STAGES + NACC);
  const uint32_t done_bar = smem_u32(bars + 2 * STAGES + 2 * NACC);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 2 * NACC + 1);
  volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int G = gridDim.x, c = blockIdx.x;
  const int64_t rounds = (g.tiles + G - 1) / G;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    for (int a = 0; a < NACC; ++a) {
      mbar_init(tfull0 + 8 * a, 1);
      mbar_init(tempty0 + 8 * a, NEPI);
    }
    mbar_init(done_bar, 1);
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(GTMEM)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      for (int i = 0; i < kBoxes; ++i) {
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&maps.a[i])) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&maps.b[i])) : "memory");
      }
      int64_t q = 0;   // K blocks issued: stage q % STAGES in round q / STAGES
      bool ok = true;
      for (int64_t rd = 0; rd < rounds && ok; ++rd) {
        const int64_t pos = walk(rd, c, G);
        if (pos >= g.tiles) continue;
        const GroupedTile& pb = g.recs[pos];
        const int32_t ya = pb.ya, yb = pb.yb, sa = pb.sa, sb = pb.sb, kk = pb.k;
        const int ha = pb.ha, hb = pb.hb;
        const int ia = box_index(ha), ib = box_index(hb);
        const uint32_t bytes = (uint32_t)(S * (ha + hb) * GK * 2);
        const int64_t nkb = (kk + GK - 1) / GK;
        for (int64_t kb = 0; kb < nkb; ++kb, ++q) {
          const int stage = (int)(q % STAGES);
          const uint32_t phase = (uint32_t)((q / STAGES) & 1);
          if (!mbar_wait(empty0 + 8 * stage, phase ^ 1u, abort)) { ok = false; break; }
          const uint32_t sA = smem_u32(smem + stage * SB), sBb = sA + S * GBOX;
          mbar_expect_tx(full0 + 8 * stage, bytes);
#pragma unroll
          for (int sl = 0; sl < S; ++sl) {
            tma_load_2d(sA + sl * GBOX, &maps.a[ia], full0 + 8 * stage, 0,
                        (int32_t)(ya + kb * sa + (int64_t)sl * g.rows_a));
            tma_load_2d(sBb + sl * GBOX, &maps.b[ib], full0 + 8 * stage, 0,
                        (int32_t)(yb + kb * sb + (int64_t)sl * g.rows_b));
          }
        }
      }
      // copies still in flight land before the CTA leaves: the last use of
      // each stage has completed (bounded)
      for (int64_t u = q - 1; u >= 0 && u >= q - STAGES; --u) {
        const int stage = (int)(u % STAGES);
        const uint32_t phase = (uint32_t)((u / STAGES) & 1);
        for (uint32_t i = 0; i < WAIT_LIMIT && !mbar_try(full0 + 8 * stage, phase); ++i) {
        }
      }
    }
    __syncwarp();
  } else if (warp == 1) {
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
          const uint64_t bd = sw128_desc(smem_u32(smem + stage * SB + S * GBOX));
          constexpr int NT = S == 1 ? 1 : 6;
#pragma unroll
          for (int term = 0; term < NT; ++term) {
            // split products smallest first: (2,0) (1,1) (0,2) (1,0) (0,1) (0,0)
            const int sa = S == 1 ? 0 : (term == 0 ? 2 : term == 1 ? 1 : term == 2 ? 0 : term == 3 ? 1 : 0);
            const int sb = S == 1 ? 0 : (term == 0 ? 0 : term == 1 ? 1 : term == 2 ? 2 : term == 3 ? 0 : term == 4 ? 1 : 0);
            const uint64_t a0 = ad + (uint64_t)((sa * GBOX) >> 4), b0 = bd + (uint64_t)((sb * GBOX) >> 4);
#pragma unroll
            for (int k16 = 0; k16 < GK / 16; ++k16)
              mma_bf16(dcol, a0 + (uint64_t)(2 * k16), b0 + (uint64_t)(2 * k16), idesc,
                       (kb > 0 || term > 0 || k16 > 0) ? 1u : 0u);
          }
          mma_commit(empty0 + 8 * stage);    // frees the stage when these MMAs finish
          issued = true;
          if (++stage == STAGES) { stage = 0; phase ^= 1u; }
        }
        if (!ok) break;
        mma_commit(tfull0 + 8 * acc);         // the tile's accumulator is complete
        if (++acc == NACC) { acc = 0; aphase ^= 1u; }
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
    // group e = (w - 2) / 4 drains accumulator e, i.e. the tiles i = e
    // (mod NACC) of this CTA's sequence; warp w reads TMEM lane quarter
    // w % 4 (tile rows 32 (w % 4) ..): each thread owns one row, 128 columns
    const int q = warp & 3;
    const int e = (warp - 2) >> 2;
    const uint32_t lane_base = (uint32_t)(q * 32) << 16;
    const uint32_t acc_col = (uint32_t)(e * GN);
    uint32_t aphase = 0;
    int64_t i = -1;   // index of the tile in this CTA's sequence
    for (int64_t rd = 0; rd < rounds; ++rd) {
      const int64_t pos = walk(rd, c, G);
      if (pos >= g.tiles) continue;
      if ((++i) % NACC != e) continue;
      const GroupedTile pb = g.recs[pos];
      const int64_t t = pb.t;
      const int tm = pb.tm, tn = pb.tn;
      const int64_t i0 = (int64_t)tm * GM, j0 = (int64_t)tn * GN;
      const int64_t row = i0 + 32 * q + lane;
      const bool row_ok = row < pb.m;
      const bool has_c = pb.C && g.beta != 0.0;
      const int ncol = (int)(pb.n - j0 < GN ? pb.n - j0 : GN);
      // the C lines of this warp's 32 rows into L2 while the tile's MMAs run
      // (lane l: columns l, l + 32, l + 64, l + 96)
      if (has_c && i0 + 32 * q < pb.m) {
        const int64_t es = g.cdt == ARMA_F64 ? 8 : g.cdt == ARMA_F32 ? 4 : 2;
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (lane + 32 * u < ncol)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(static_cast<const char*>(pb.C) +
                                                          ((i0 + 32 * q) + (j0 + lane + 32 * u) * (int64_t)pb.ldc) * es));
      }
      // FP32 C: the first 16 columns are loaded before the accumulator is
      // complete, and then the loads of the next 16 columns are in flight
      // while a chunk's D is written (all of a chunk's C is read before its
      // D, and D columns are written in order, so D may be C itself)
      const bool c32 = has_c && g.cdt == ARMA_F32;
      const int64_t ldc = pb.ldc, ldd = pb.m;
      const float* Cr = c32 ? static_cast<const float*>(pb.C) + row + j0 * ldc : nullptr;
      float cn[16];
      load_c16(cn, Cr, ldc, c32 && row_ok, ncol);
      if (!__all_sync(0xffffffffu, mbar_wait(tfull0 + 8 * e, aphase, abort))) break;
      aphase ^= 1u;
      fence_after();
      double dsum = 0.0;
      float* Dr = static_cast<float*>(pb.D) + row + j0 * ldd;
      // this row's diagonal column, if the trace runs through it (i < min(m, n))
      const int diag = (tm == tn && row - j0 < ncol) ? (int)(row - j0) : -1;
#pragma unroll 1
      for (int c0 = 0; c0 < ncol; c0 += 16) {
        float cv[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) cv[j] = cn[j];
        load_c16(cn, Cr + (int64_t)(c0 + 16) * ldc, ldc, c32 && row_ok, ncol - (c0 + 16));
        float v[16];
        if (pb.k > 0) {
          tmem_ld16(tmem_base + lane_base + acc_col + (uint32_t)c0, v);
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j) v[j] = 0.f;
        }
        if (!row_ok) continue;
        float* dp = Dr + (int64_t)c0 * ldd;
        if (diag >= c0 && diag < c0 + 16) {
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (c0 + j == diag) dsum += (double)v[j];
        }
        if (c32 || !has_c) {
          if (c0 + 16 <= ncol) {
#pragma unroll
            for (int j = 0; j < 16; ++j) dp[j * ldd] = fmaf(g.beta_f, cv[j], g.alpha_f * v[j]);
          } else {
#pragma unroll
            for (int j = 0; j < 16; ++j)
              if (c0 + j < ncol) dp[j * ldd] = fmaf(g.beta_f, cv[j], g.alpha_f * v[j]);
          }
        } else {
          // C of another type, element by element (D is FP32, so it is
          // never C itself here)
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (c0 + j < ncol)
              dp[j * ldd] = fmaf(g.beta_f, load_as<float>(pb.C, row + (j0 + c0 + j) * ldc, g.cdt), g.alpha_f * v[j]);
        }
      }
      // the accumulator is free for the MMA issuer again
      fence_before();
      mbar_arrive(tempty0 + 8 * e);
      if (g.trace_partials && tm == tn) {     // diagonal tile: each warp's share of the trace
        dsum = warp_sum(dsum);
        if (lane == 0) {
          g.trace_partials[kTraceSlots * t + q] = dsum;
          g.trace_partials[kTraceSlots * t + 4 + q] = 0.0;
        }
      }
    }
  }

  fence_before();
  __syncthreads();
  if (threadIdx.x == 0 && *abort && g.status) atomicCAS(g.status, 0, (int32_t)ARMA_ERR_TIMEOUT);
  if (warp == 1) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(GTMEM) : "memory");
  }
}

// a packed array as a 2-D BF16 tensor of `rows` rows of 64, read in boxes of
// box_rows x 64 with the 128-byte swizzle the MMA descriptors expect
bool make_packed_map(CUtensorMap* map, const void* base, int64_t rows, int box_rows) {
  auto fn = encode_fn();
  if (!fn || rows < 1) return false;
  cuuint64_t dims[2] = {(cuuint64_t)GK, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(GK * 2)};
  cuuint32_t box[2] = {(cuuint32_t)GK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <typename AT, int S>
cudaError_t launch_packed(const GroupedArgs& g, cudaStream_t s, int* launches) {
  if (g.slices != S) return cudaErrorInvalidValue;
  const bool any = g.rows_a > 0 && g.rows_b > 0;   // some problem has K > 0
  if (any && (!g.pack_a || !g.pack_b)) return cudaErrorInvalidValue;
  // 1. pack
  if (any && g.n_items > 0) {
    if (!g.pack_items) return cudaErrorInvalidValue;
    // a persistent grid: as many CTAs of 8 warps as fit on the GPU at once,
    // or fewer for a short list
    static std::atomic<int> per_sm{0};
    int fit = per_sm.load(std::memory_order_relaxed);
    if (fit <= 0) {
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, grouped_pack_kernel<AT, S>, 256, 0) != cudaSuccess ||
          fit < 1)
        fit = 1;
      per_sm.store(fit, std::memory_order_relaxed);
    }
    int64_t blocks = (g.n_items + 7) / 8, cap = (int64_t)device_sm_count() * fit;
    grouped_pack_kernel<AT, S><<<(unsigned)(blocks < cap ? blocks : cap), 256, 0, s>>>(g);
    if (launches) ++*launches;
  }
  // 2. the products (with no K anywhere no box is ever loaded)
  PackedMaps maps;
  memset(&maps, 0, sizeof maps);
  if (any) {
    for (int i = 0; i < kBoxes; ++i) {
      if (!make_packed_map(&maps.a[i], g.pack_a, (int64_t)S * g.rows_a, 16 << i)) return cudaErrorInvalidValue;
      if (!make_packed_map(&maps.b[i], g.pack_b, (int64_t)S * g.rows_b, 16 << i)) return cudaErrorInvalidValue;
    }
  }
  constexpr int smem = smem_bytes<S>();
  static std::atomic<bool> attr[64];
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (!attr[dev].load(std::memory_order_acquire)) {
    cudaError_t e = cudaFuncSetAttribute(grouped_packed_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    attr[dev].store(true, std::memory_order_release);
  }
  // one CTA per SM, each walking its share of the tile list
  int64_t grid = (int64_t)device_sm_count();
  if (grid > g.tiles) grid = g.tiles;
  grouped_packed_kernel<S><<<(unsigned)grid, GTHREADS, smem, s>>>(g, maps);
  if (launches) ++*launches;
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_grouped_tc(const GroupedArgs& g, cudaStream_t s, int* launches) {
  if (g.tiles == 0) return cudaSuccess;
  if (!g.recs) return cudaErrorInvalidValue;
  if (g.abdt == ARMA_BF16) return launch_packed<__nv_bfloat16, 1>(g, s, launches);
  if (g.abdt == ARMA_F32) return launch_packed<float, 3>(g, s, launches);
  return cudaErrorInvalidValue;
}

}  // namespace arma
