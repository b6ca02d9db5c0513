// FP64-accurate products on the tensor cores by exact slicing (the error-free
// splitting of Ozaki, Ogita, Oishi & Rump, "Error-free transformations of
// matrix multiplication by using fast routines of matrix multiplication and
// its applications", Numer. Algorithms 2012), for the products the paper maps
// onto xGEMM (Sec. II, the xGEMM paragraph; Fig. 3) when FP64 accuracy is
// asked for, and for the FP64 residual of iterative refinement (Sec. I and
// Sec. III (9): inv(A)*b as a solve).
//
// Scaling.  Row i of op(A) is scaled by 2^-e_i, with e_i the smallest
// exponent such that every |op(A)_il| < 2^e_i; likewise column j of op(B) by
// 2^-f_j.  Both scalings are exact.
//
// Slicing.  A scaled value r in (-1, 1) is written exactly as
//     r = sum_{s<8} q_s 2^(-7(s+1)) + rest,   |rest| <= 2^-57,
// with integers |q_0| <= 128, |q_s| <= 64 (balanced base-128 digits of the
// 56-bit fixed-point value of r): every q_s is exact in BF16.
//
// Products.  op(A) op(B) = 2^(e_i + f_j) sum_{s,t} 2^(-7(s+t+2)) Q_s P_t
// keeps the 36 slice products with s + t <= 7; the dropped ones are below
// 2^-53 of the row and column maxima per term, the size of one FP64 rounding.
// Each Q_s P_t is a BF16 x BF16 product on tcgen05.  K is taken 1024 at a time,
// so every partial sum is an integer of magnitude <= 1024 * 2^14 = 2^24: the
// tensor core's FP32 accumulation is exact (checked on this GPU against
// int64 products, sums of exactly 2^24 included).  The epilogue converts
// each chunk to int32, adds the products of equal weight (s + t = d, at most
// 8 of them, < 2^27) in int32, and accumulates the weighted groups in FP64.
//
// Pipeline (one CTA per SM, persistent over (tile, K split) work items):
//   warp 0      TMA producer: slice tiles of op(A) (128 x 64) and op(B)^T
//               (64 x 64) into a 6-stage ring
//   warp 1      TMEM owner (two 128 x 64 FP32 accumulators) and MMA issuer
//   warps 2..9  epilogue: one row and 32 columns of the tile per thread
// Each work item writes its FP64 partial, scaled by 2^(e_i + f_j), to
// scratch; a combine pass adds the K splits and applies alpha, the diagonal
// scalings and beta * C in FP64.  Rows or columns holding a non-finite value
// give NaN.  Every mbarrier wait is bounded.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <atomic>
#include <mutex>

#include "common.cuh"
#include "tc_ops.cuh"

namespace arma {

namespace oz {

using namespace tc;

constexpr int S = 8;                 // slices per operand
constexpr int NPAIR = 36;            // slice pairs with s + t <= 7
constexpr int BM = 128, BN = 64, BK = 64, STAGES = 6;
constexpr int A_TILE = BM * BK * 2;  // 16 KiB
constexpr int B_TILE = BN * BK * 2;  // 8 KiB
constexpr int STAGE_BYTES = A_TILE + B_TILE;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;
constexpr int KB_CHUNK = 16;         // 16 K blocks of 64: 1024 of K per accumulation
constexpr int THREADS = 320;
constexpr int EPI_THREADS = 256;
constexpr int TMEM_COLS = 128;       // two 64-column accumulators
constexpr int32_t NONFINITE = 0x7fffffff;

// pair p -> (s, t), ordered by d = s + t; group d holds pairs [first(d), first(d) + d + 1)
__host__ __device__ constexpr int pair_s(int p) {
  int d = 0;
  while ((d + 1) * (d + 2) / 2 <= p) ++d;
  return p - d * (d + 1) / 2;
}
__host__ __device__ constexpr int pair_d(int p) {
  int d = 0;
  while ((d + 1) * (d + 2) / 2 <= p) ++d;
  return d;
}

struct Params {
  int64_t m, n, k;
  int64_t mpad, npad, kp;     // slice rows (padded) and row stride
  int32_t tiles_m, tiles_n, splits, chunks_per_split, chunks;
  double* P;                  // [splits][m * n] FP64 partials, column-major (ld = m)
  const int32_t* ea;          // row exponents of op(A)
  const int32_t* eb;          // column exponents of op(B)
  int32_t* status;
  const int* skip;
};

struct WorkItem {
  int32_t tm, tn, split;
};

__device__ __forceinline__ WorkItem work_item(const Params& p, int32_t w) {
  const int32_t per_split = p.tiles_m * p.tiles_n;
  WorkItem it;
  it.split = w / per_split;
  const int32_t r = w - it.split * per_split;
  it.tm = r % p.tiles_m;      // consecutive CTAs share the B tile column in L2
  it.tn = r / p.tiles_m;
  return it;
}

// 2^e for -1022 <= e <= 1023 (clamped), built from its bits; scale2 applies
// 2^e in two exact steps, so e may reach +-2044
__device__ __forceinline__ double pow2_half(int e) {
  e = e < -1022 ? -1022 : e > 1023 ? 1023 : e;
  return __longlong_as_double((long long)(e + 1023) << 52);
}
__device__ __forceinline__ double scale2(double v, int e) {
  const int e1 = e / 2, e2 = e - e1;
  return v * pow2_half(e1) * pow2_half(e2);
}

__global__ void __launch_bounds__(THREADS, 1)
    ozaki_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                 const __grid_constant__ Params p) {
  if (p.skip && *p.skip) return;            // uniform, before any barrier or TMEM allocation
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
  const int32_t total_work = p.tiles_m * p.tiles_n * p.splits;
  const int32_t kb_total = (int32_t)((p.k + BK - 1) / BK);

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
        const WorkItem it = work_item(p, w);
        const int32_t c0 = it.split * p.chunks_per_split;
        const int32_t c1 = min(c0 + p.chunks_per_split, p.chunks);
        for (int32_t c = c0; c < c1 && ok; ++c) {
          const int32_t kb0 = c * KB_CHUNK, kb1 = min(kb0 + KB_CHUNK, kb_total);
          for (int pr = 0; pr < NPAIR && ok; ++pr) {
            const int sa = pair_s(pr), sb = pair_d(pr) - sa;
            for (int32_t kb = kb0; kb < kb1; ++kb) {
              if (!mbar_wait(empty0 + 8 * stage, phase ^ 1u, abort)) { ok = false; break; }
              const uint32_t fb = full0 + 8 * stage;
              mbar_expect_tx(fb, STAGE_BYTES);
              const uint32_t sA = smem_u32(smem + stage * STAGE_BYTES);
              tma_load_2d(sA, &tmA, fb, kb * BK, (int32_t)(sa * p.mpad + (int64_t)it.tm * BM));
              tma_load_2d(sA + A_TILE, &tmB, fb, kb * BK, (int32_t)(sb * p.npad + (int64_t)it.tn * BN));
              inflight[stage] = (int32_t)phase;
              if (++stage == STAGES) { stage = 0; phase ^= 1u; }
            }
          }
        }
      }
      if (!ok) {
        // copies already issued land before the CTA can exit (bounded)
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
      bool ok = true, issued = false;
      for (int32_t w = blockIdx.x; w < total_work && ok; w += gridDim.x) {
        const WorkItem it = work_item(p, w);
        const int32_t c0 = it.split * p.chunks_per_split;
        const int32_t c1 = min(c0 + p.chunks_per_split, p.chunks);
        for (int32_t c = c0; c < c1 && ok; ++c) {
          const int32_t kb0 = c * KB_CHUNK, kb1 = min(kb0 + KB_CHUNK, kb_total);
          for (int pr = 0; pr < NPAIR && ok; ++pr) {
            if (!mbar_wait(tempty0 + 8 * acc, aphase ^ 1u, abort)) { ok = false; break; }
            fence_after();
            const uint32_t dcol = tmem_base + (uint32_t)(acc * BN);
            uint32_t accumulate = 0;
            for (int32_t kb = kb0; kb < kb1; ++kb) {
              if (!mbar_wait(full0 + 8 * stage, phase, abort)) { ok = false; break; }
              fence_after();
              const uint32_t sA = smem_u32(smem + stage * STAGE_BYTES);
              const uint64_t ad = sw128_desc(sA), bd = sw128_desc(sA + A_TILE);
#pragma unroll
              for (int kk = 0; kk < BK / 16; ++kk) {
                mma_bf16(dcol, ad + (uint64_t)(2 * kk), bd + (uint64_t)(2 * kk), idesc, accumulate);
                accumulate = 1;
              }
              mma_commit(empty0 + 8 * stage);
              issued = true;
              if (++stage == STAGES) { stage = 0; phase ^= 1u; }
            }
            if (!ok) break;
            mma_commit(tfull0 + 8 * acc);     // this pair's chunk sum is ready
            if (++acc == 2) { acc = 0; aphase ^= 1u; }
          }
        }
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
    const int quarter = warp & 3;
    const int half = (warp - 2) >> 2;
    const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
    int acc = 0;
    uint32_t aphase = 0;
    bool ok = true;
    for (int32_t w = blockIdx.x; w < total_work && ok; w += gridDim.x) {
      const WorkItem it = work_item(p, w);
      const int32_t c0 = it.split * p.chunks_per_split;
      const int32_t c1 = min(c0 + p.chunks_per_split, p.chunks);
      double sum[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) sum[j] = 0.0;
      for (int32_t c = c0; c < c1 && ok; ++c) {
        int pr = 0;
        for (int d = 0; d < 8 && ok; ++d) {
          int32_t part[32];
#pragma unroll
          for (int j = 0; j < 32; ++j) part[j] = 0;
          for (int q = 0; q <= d; ++q, ++pr) {
            ok = __all_sync(0xffffffffu, mbar_wait(tfull0 + 8 * acc, aphase, abort));
            if (!ok) break;
            fence_after();
            const uint32_t tb = tmem_base + lane_base + (uint32_t)(acc * BN + half * 32);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              float v[16];
              tmem_ld16(tb + (uint32_t)(16 * h), v);
#pragma unroll
              for (int j = 0; j < 16; ++j) part[16 * h + j] += __float2int_rn(v[j]);   // exact integers
            }
            fence_before();
            mbar_arrive(tempty0 + 8 * acc);
            if (++acc == 2) { acc = 0; aphase ^= 1u; }
          }
          if (!ok) break;
          const double wgt = pow2_half(-7 * (d + 2));
#pragma unroll
          for (int j = 0; j < 32; ++j) sum[j] = fma((double)part[j], wgt, sum[j]);
        }
      }
      if (!ok) break;
      // the partial of this K split, scaled back by 2^(e_i + f_j)
      const int64_t row = (int64_t)it.tm * BM + quarter * 32 + lane;
      if (row < p.m) {
        const int32_t ei = p.ea[row];
        double* dst = p.P + (int64_t)it.split * p.m * p.n + row;
        const int64_t col0 = (int64_t)it.tn * BN + half * 32;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int64_t col = col0 + j;
          if (col >= p.n) continue;
          const int32_t fj = p.eb[col];
          const double v = (ei == NONFINITE || fj == NONFINITE) ? __longlong_as_double(0x7ff8000000000000ll)
                                                                 : scale2(sum[j], ei + fj);
          dst[col * p.m] = v;
        }
      }
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
// Scaling and slicing of op(X) (R x K): element (r, l) at X[r * rs + l * ks]
// ---------------------------------------------------------------------------
struct SliceArgs {
  const double* X;
  int64_t rs, ks;             // strides of op(X); one of them is 1
  int64_t R, K, rpad, kp;
  int32_t* e;                 // [R] row exponents (NONFINITE: the row holds an Inf or NaN)
  __nv_bfloat16* out;         // [S][rpad][kp], K-major
  const int* skip;
};

// exponent field of |x| as an upper bound: |x| < 2^(E - 1022) (E the biased
// exponent; subnormals and zero give the bound of the smallest normal)
__device__ __forceinline__ int32_t exp_bound(double x) {
  const int32_t E = (int32_t)((__double_as_longlong(x) >> 52) & 0x7FF);
  if (E == 0x7FF) return NONFINITE;
  return E == 0 ? -1021 : E - 1022;
}

__device__ __forceinline__ int32_t emax(int32_t a, int32_t b) {
  if (a == NONFINITE || b == NONFINITE) return NONFINITE;
  return a > b ? a : b;
}

// rows contiguous along K (ks == 1): one warp per row
__global__ void __launch_bounds__(256) row_exp_kcontig_kernel(SliceArgs a) {
  if (a.skip && *a.skip) return;
  const int64_t r = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (r >= a.R) return;
  const double* x = a.X + r * a.rs;
  int32_t m = -1021;
  for (int64_t l = lane; l < a.K; l += 32) m = emax(m, exp_bound(x[l]));
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) m = emax(m, __shfl_xor_sync(0xffffffffu, m, off));
  if (lane == 0) a.e[r] = m;
}

// rows adjacent in memory (rs == 1): a thread per row and per 64 of K
// (coalesced across the warp), combined with an integer atomic maximum into
// e, which starts below every bound (NONFINITE is the largest int32, so a
// non-finite value wins the maximum)
__global__ void __launch_bounds__(256) row_exp_rcontig_kernel(SliceArgs a) {
  if (a.skip && *a.skip) return;
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= a.R) return;
  const int64_t l0 = (int64_t)blockIdx.y * 64, l1 = min(l0 + 64, a.K);
  int32_t m = -1021;
  for (int64_t l = l0; l < l1; ++l) m = emax(m, exp_bound(a.X[r + l * a.ks]));
  atomicMax(a.e + r, m);
}

// Slices of one value x of a row with exponent bound e (|x| < 2^e): the
// fixed-point integer M = rint(x 2^(56 - e)), |M| <= 2^56 (the rounding is
// the rest, <= 2^-57 of 2^e), written in balanced base-128 digits
//     M = sum_{s<8} q_s 128^(7 - s),  q_7 .. q_1 in [-64, 63],  |q_0| <= 128,
// taken from the least significant end: q = M mod 128 in [-64, 63], then
// M = (M - q) / 128 exactly.  The scaling is two exact power-of-two products;
// the digits use 32-bit integer operations on the two halves of M (64-bit
// integer operations would run on the FP64 pipe).
__device__ __forceinline__ void slice8(double x, int e, uint16_t (&q)[S]) {
  const int sh = 56 - e, a = sh / 2, b = sh - a;
  const long long M = __double2ll_rn(x * pow2_half(a) * pow2_half(b));
  uint32_t lo = (uint32_t)(unsigned long long)M;
  uint32_t hi = (uint32_t)((unsigned long long)M >> 32);
  int d[S];
#pragma unroll
  for (int s = S - 1; s >= 1; --s) {
    int v = (int)(lo & 127u);
    v -= (v & 64) << 1;                                // balanced digit in [-64, 63]
    const uint32_t vl = (uint32_t)v, vh = (uint32_t)(v >> 31);
    asm("sub.cc.u32 %0, %0, %2;\n\tsubc.u32 %1, %1, %3;" : "+r"(lo), "+r"(hi) : "r"(vl), "r"(vh));
    lo = __funnelshift_r(lo, hi, 7);                   // (hi:lo) >>= 7, arithmetic
    hi = (uint32_t)((int32_t)hi >> 7);
    d[s] = v;
  }
  d[0] = (int)lo;                                      // |q_0| <= 128
#pragma unroll
  for (int s = 0; s < S; ++s) q[s] = __bfloat16_as_ushort(__float2bfloat16_rn((float)d[s]));   // exact
}

// A 32-row x 64-K tile per block through shared memory (so that the global
// reads are coalesced for either orientation); each thread then slices 8
// consecutive K values of one row and writes 16 bytes per slice.
__global__ void __launch_bounds__(256) slice_kernel(SliceArgs a) {
  if (a.skip && *a.skip) return;
  __shared__ double tile[32][65];
  const int64_t r0 = (int64_t)blockIdx.x * 32, l0 = (int64_t)blockIdx.y * 64;
  const int tid = threadIdx.x;
  if (a.ks == 1) {
    for (int t = tid; t < 32 * 64; t += 256) {
      const int rr = t >> 6, ll = t & 63;
      const int64_t r = r0 + rr, l = l0 + ll;
      tile[rr][ll] = (r < a.R && l < a.K) ? a.X[r * a.rs + l] : 0.0;
    }
  } else {
    for (int t = tid; t < 32 * 64; t += 256) {
      const int rr = t & 31, ll = t >> 5;
      const int64_t r = r0 + rr, l = l0 + ll;
      tile[rr][ll] = (r < a.R && l < a.K) ? a.X[r + l * a.ks] : 0.0;
    }
  }
  __syncthreads();
  const int rr = tid >> 3, g = tid & 7;          // row of the tile, group of 8 K values
  const int64_t r = r0 + rr, l = l0 + 8 * g;
  if (r >= a.rpad || l >= a.kp) return;
  const int32_t e = r < a.R ? a.e[r] : 0;
  __align__(16) uint16_t q[S][8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    uint16_t qs[S];
    slice8(e == NONFINITE ? 0.0 : tile[rr][8 * g + j], e == NONFINITE ? 0 : e, qs);
#pragma unroll
    for (int s = 0; s < S; ++s) q[s][j] = qs[s];
  }
#pragma unroll
  for (int s = 0; s < S; ++s)
    *reinterpret_cast<uint4*>(a.out + ((int64_t)s * a.rpad + r) * a.kp + l) = *reinterpret_cast<const uint4*>(q[s]);
}

// D = alpha * diag(rs) * (sum over splits of P) * diag(cs) + beta * C, in FP64
struct CombineArgs {
  int64_t m, n;
  int32_t splits;
  const double* P;
  void* D; int64_t ldd; int32_t ddt;
  const void* C; int64_t ldc; int32_t cdt;
  double alpha, beta;
  const void* rsv; int64_t rs_inc; int32_t rsdt;
  const void* csv; int64_t cs_inc; int32_t csdt;
  const int* skip;
};

__global__ void __launch_bounds__(256) combine_kernel(const __grid_constant__ CombineArgs a) {
  if (a.skip && *a.skip) return;
  const int64_t total = a.m * a.n;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t col = t / a.m, row = t - col * a.m;
    double s = 0.0;
    for (int z = 0; z < a.splits; ++z) s += a.P[(int64_t)z * total + t];
    double v = a.alpha * s;
    if (a.rsv) v *= load_as<double>(a.rsv, row * a.rs_inc, a.rsdt);
    if (a.csv) v *= load_as<double>(a.csv, col * a.cs_inc, a.csdt);
    if (a.C && a.beta != 0.0) v = fma(a.beta, load_as<double>(a.C, row + col * a.ldc, a.cdt), v);
    store_as<double>(a.D, row + col * a.ldd, a.ddt, v);
  }
}

struct Geometry {
  int64_t mpad, npad, kp;
  int32_t tiles_m, tiles_n, chunks, splits, chunks_per_split;
  int64_t a_bytes, b_bytes, ea_bytes, eb_bytes, p_bytes;
};

Geometry geometry(int64_t m, int64_t n, int64_t k, bool nosplit) {
  Geometry g;
  g.mpad = (m + BM - 1) / BM * BM;
  g.npad = (n + BN - 1) / BN * BN;
  g.kp = (k + BK - 1) / BK * BK;     // whole K blocks: the slicing pass writes the zero tail
  g.tiles_m = (int32_t)(g.mpad / BM);
  g.tiles_n = (int32_t)(g.npad / BN);
  g.chunks = (int32_t)((g.kp / BK + KB_CHUNK - 1) / KB_CHUNK);
  // split K (whole chunks) only to fill the GPU when the output has few tiles
  const int64_t tiles = (int64_t)g.tiles_m * g.tiles_n;
  int64_t splits = 1;
  while (!nosplit && tiles * splits * 2 <= 152 && splits * 2 <= g.chunks) splits *= 2;
  g.splits = (int32_t)splits;
  g.chunks_per_split = (int32_t)((g.chunks + splits - 1) / splits);
  g.splits = (g.chunks + g.chunks_per_split - 1) / g.chunks_per_split;
  g.a_bytes = (int64_t)S * g.mpad * g.kp * 2;
  g.b_bytes = (int64_t)S * g.npad * g.kp * 2;
  g.ea_bytes = (m * 4 + 255) / 256 * 256;
  g.eb_bytes = (n * 4 + 255) / 256 * 256;
  g.p_bytes = (int64_t)g.splits * m * n * 8;
  return g;
}

int64_t align256(int64_t b) { return (b + 255) / 256 * 256; }

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

}  // namespace oz

int64_t gemm_ozaki_scratch_bytes(int64_t m, int64_t n, int64_t k) {
  if (m < 1 || n < 1 || k < 1) return 0;
  const oz::Geometry g = oz::geometry(m, n, k, false);
  return oz::align256(g.a_bytes) + oz::align256(g.b_bytes) + g.ea_bytes + g.eb_bytes + oz::align256(g.p_bytes) +
         1024;
}

bool gemm_ozaki_supported(const GemmArgs& a) {
  if (a.m < 2 || a.n < 2 || a.k < 1) return false;
  if (a.adt != ARMA_F64 || a.bdt != ARMA_F64) return false;
  if (a.m > (1ll << 30) || a.n > (1ll << 30) || a.k > (1ll << 30)) return false;
  if (!a.scratch) return false;
  const oz::Geometry g = oz::geometry(a.m, a.n, a.k, a.nosplit != 0);
  if (g.mpad * oz::S > INT32_MAX || g.npad * oz::S > INT32_MAX) return false;
  return a.scratch_bytes >= gemm_ozaki_scratch_bytes(a.m, a.n, a.k);
}

cudaError_t launch_gemm_ozaki(const GemmArgs& a, cudaStream_t s, int* launches) {
  using namespace oz;
  const Geometry g = geometry(a.m, a.n, a.k, a.nosplit != 0);
  char* base = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(a.scratch) + 255) & ~uintptr_t(255));
  __nv_bfloat16* As = reinterpret_cast<__nv_bfloat16*>(base);
  __nv_bfloat16* Bs = reinterpret_cast<__nv_bfloat16*>(base + align256(g.a_bytes));
  int32_t* ea = reinterpret_cast<int32_t*>(base + align256(g.a_bytes) + align256(g.b_bytes));
  int32_t* eb = reinterpret_cast<int32_t*>(reinterpret_cast<char*>(ea) + g.ea_bytes);
  double* P = reinterpret_cast<double*>(reinterpret_cast<char*>(eb) + g.eb_bytes);
  const int sms = device_sm_count();

  // op(A) (m x k): element (i, l) = ta ? A[l + i lda] : A[i + l lda];
  // op(B)^T (n x k): element (j, l) = tb ? B[j + l ldb] : B[l + j ldb]
  SliceArgs sa;
  sa.X = static_cast<const double*>(a.A);
  sa.rs = a.ta ? a.lda : 1; sa.ks = a.ta ? 1 : a.lda;
  sa.R = a.m; sa.K = a.k; sa.rpad = g.mpad; sa.kp = g.kp;
  sa.e = ea; sa.out = As; sa.skip = a.skip;
  SliceArgs sb;
  sb.X = static_cast<const double*>(a.B);
  sb.rs = a.tb ? 1 : a.ldb; sb.ks = a.tb ? a.ldb : 1;
  sb.R = a.n; sb.K = a.k; sb.rpad = g.npad; sb.kp = g.kp;
  sb.e = eb; sb.out = Bs; sb.skip = a.skip;
  auto slice = [&](const SliceArgs& x) -> cudaError_t {
    const int64_t gy = x.kp / 64;
    if (gy > 65535) return cudaErrorInvalidConfiguration;
    if (x.ks == 1) {
      row_exp_kcontig_kernel<<<(unsigned)((x.R + 7) / 8), 256, 0, s>>>(x);
    } else {
      // 0x80808080 as int32 is below every exponent bound
      cudaError_t e0 = cudaMemsetAsync(x.e, 0x80, (size_t)x.R * sizeof(int32_t), s);
      if (e0 != cudaSuccess) return e0;
      row_exp_rcontig_kernel<<<dim3((unsigned)((x.R + 255) / 256), (unsigned)gy), 256, 0, s>>>(x);
    }
    slice_kernel<<<dim3((unsigned)(x.rpad / 32), (unsigned)gy), 256, 0, s>>>(x);
    if (launches) *launches += 2;
    return cudaGetLastError();
  };
  cudaError_t e;
  if (!a.reuse_a && (e = slice(sa)) != cudaSuccess) return e;
  if ((e = slice(sb)) != cudaSuccess) return e;

  CUtensorMap mapA, mapB;
  if (!make_map(&mapA, As, g.kp, (int64_t)S * g.mpad, BM)) return cudaErrorInvalidValue;
  if (!make_map(&mapB, Bs, g.kp, (int64_t)S * g.npad, BN)) return cudaErrorInvalidValue;
  Params p;
  memset(&p, 0, sizeof p);
  p.m = a.m; p.n = a.n; p.k = a.k;
  p.mpad = g.mpad; p.npad = g.npad; p.kp = g.kp;
  p.tiles_m = g.tiles_m; p.tiles_n = g.tiles_n; p.splits = g.splits;
  p.chunks_per_split = g.chunks_per_split; p.chunks = g.chunks;
  p.P = P; p.ea = ea; p.eb = eb;
  p.status = a.status; p.skip = a.skip;
  static std::atomic<bool> attr_set[64];
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (!attr_set[dev].load(std::memory_order_acquire)) {
    e = cudaFuncSetAttribute(ozaki_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    if (e != cudaSuccess) return e;
    attr_set[dev].store(true, std::memory_order_release);
  }
  const int64_t work = (int64_t)g.tiles_m * g.tiles_n * g.splits;
  const int grid = (int)(work < sms ? work : sms);
  ozaki_kernel<<<grid, THREADS, SMEM_BYTES, s>>>(mapA, mapB, p);
  if (launches) ++*launches;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  CombineArgs c;
  c.m = a.m; c.n = a.n; c.splits = g.splits; c.P = P;
  c.D = a.D; c.ldd = a.ldd; c.ddt = a.ddt;
  c.C = a.C; c.ldc = a.ldc; c.cdt = a.cdt;
  c.alpha = a.alpha; c.beta = a.beta;
  c.rsv = a.rs; c.rs_inc = a.rs_inc; c.rsdt = a.rsdt;
  c.csv = a.cs; c.cs_inc = a.cs_inc; c.csdt = a.csdt;
  c.skip = a.skip;
  const int64_t total = a.m * a.n;
  int64_t blocks = (total + 255) / 256, cap = (int64_t)sms * 8;
  combine_kernel<<<(unsigned)(blocks < cap ? blocks : cap), 256, 0, s>>>(c);
  if (launches) ++*launches;
  return cudaGetLastError();
}

}  // namespace arma
