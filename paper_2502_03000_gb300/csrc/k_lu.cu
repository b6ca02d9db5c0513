// X = inv(A) * B as a solve: the paper's rewrite of inv(A)*b (Sec. I;
// Sec. II, the Glue<Op<Mat,op_inv>,Vec,glue_times> pattern mapped to xGESV;
// Sec. III (9)).  Blocked right-looking LU with partial pivoting (ties go to
// the smallest row index), then forward and back substitution, and for the
// mixed-precision tiers FP64 iterative refinement.
//
//   panel      one launch per 64-column panel: each CTA keeps its block of
//              panel rows in shared memory; per column the CTAs publish
//              their local pivot candidate and meet at one barrier, then all
//              pick the same pivot, swap and update locally.  The CTAs form
//              one thread-block cluster (distributed shared memory, hardware
//              barrier) when the panel fits, else a cooperative grid with a
//              bounded-spin barrier in global memory
//   laswp      the panel's row swaps applied to the other columns
//   trsm       U12 = L11^-1 A12, one warp per column
//   update     A22 -= L21 U12 through the product kernels: DFMA for the FP64
//              tier, split-BF16 tcgen05 (FP32-accurate) or BF16 tcgen05
//   trsv       blocked substitution over all right-hand sides in one
//              cooperative launch: a CTA per (64-row block, 64 right-hand
//              sides) subtracts the blocks its rows depend on as their flags
//              are released, then solves its diagonal block (fallback: one
//              launch per diagonal block)
//   refine     r = B - A x in FP64 (DFMA), correction solved with the FP32
//              factors, x += d in FP64, until the normwise backward error
//              |r| / (|A||x| + |B|) <= 1e-14 or the step limit
//
// Numerical failures never trap: a zero pivot records ARMA_ERR_SINGULAR and
// its 1-based column in the workspace status; refinement that does not reach
// its tolerance records ARMA_ERR_NOCONVERGE.
#include <algorithm>
#include <cooperative_groups.h>
#include <type_traits>
#include <utility>

#include <atomic>

#include "common.cuh"

namespace arma {

namespace lu {

constexpr int NB = 64;          // panel width
constexpr int PT = 256;         // panel threads per CTA
constexpr int MAX_CTAS = 64;
constexpr int MAX_IR = 10;        // default refinement step limit
constexpr int MAX_IR_LIMIT = 15;  // largest limit a plan may ask for
constexpr double IR_TOL = 1e-14;
constexpr unsigned int SPIN_LIMIT = 1u << 26;
constexpr int FLAG_STRIDE = 32;                 // substitution flags, one per 128 bytes

struct Ctl {                    // device control block in the solve scratch
  unsigned int bar_count, bar_gen;
  int err;                      // barrier timeout
  int done;                     // refinement converged
  int steps;                    // refinement steps taken
  int chol_fail;                // Cholesky met a pivot <= 0: 1 + its column
  double nrmA, nrmB, nrmR, nrmX;
};

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier in global memory for a cooperative launch.  The wait is
// bounded by wait_ns (and an iteration count); a wait that runs out, or
// finds that another CTA already gave up, records ARMA_ERR_TIMEOUT and
// returns false, and every CTA then leaves its loop.
__device__ __forceinline__ bool grid_barrier(Ctl* c, unsigned int nblocks, int32_t* status, uint64_t wait_ns) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned int* gen = &c->bar_gen;
    const unsigned int g = *gen;
    __threadfence();
    const unsigned int arrived = atomicAdd(&c->bar_count, 1u) + 1u;
    if (arrived == nblocks) {
      c->bar_count = 0u;
      __threadfence();
      atomicAdd(&c->bar_gen, 1u);
    } else {
      const uint64_t t0 = global_ns();
      unsigned int i = 0;
      while (*gen == g) {
        if (wait_ns == 0 || ++i > SPIN_LIMIT || *(volatile int*)&c->err ||
            ((i & 255u) == 0u && global_ns() - t0 > wait_ns)) {
          atomicExch(&c->err, 1);
          atomicCAS(status, 0, (int32_t)ARMA_ERR_TIMEOUT);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

template <typename T>
struct PanelArgs {
  T* A; int64_t ld, n;
  int64_t j;              // first panel column (and row)
  int32_t w;              // panel width
  int64_t rows_per_cta;
  int32_t* piv;
  double* cand_val;       // [2][MAX_CTAS]
  int64_t* cand_row;      // [2][MAX_CTAS]
  T* cand_data;           // [2][MAX_CTAS][NB]
  T* drow;                // [2][NB]
  Ctl* ctl;
  int32_t* status; int64_t* info;
  uint64_t wait_ns;       // bound on one grid-barrier wait
};

// the CTA's panel rows into shared memory, eight loads in flight per thread
template <int NT, typename T>
__device__ __forceinline__ void load_panel(T* sm, const T* A, int64_t ld, int64_t r0, int64_t j, int64_t nown,
                                           int w, int64_t R) {
  const int64_t total = nown * w;
  for (int64_t t0 = 0; t0 < total; t0 += (int64_t)NT * 8) {
    T v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int64_t t = t0 + threadIdx.x + (int64_t)NT * k;
      const int64_t c = t / nown, r = t - c * nown;
      v[k] = t < total ? A[(r0 + r) + (j + c) * ld] : (T)0;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int64_t t = t0 + threadIdx.x + (int64_t)NT * k;
      const int64_t c = t / nown, r = t - c * nown;
      if (t < total) sm[c * R + r] = v[k];
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(PT) panel_kernel(const __grid_constant__ PanelArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sm = reinterpret_cast<T*>(smraw);   // [w][R] column-major
  __shared__ double red_v[PT / 32];
  __shared__ int64_t red_r[PT / 32];
  __shared__ int64_t s_p;
  __shared__ int s_win;
  __shared__ T s_u[NB];
  const int64_t R = a.rows_per_cta;
  const int64_t r0 = a.j + (int64_t)blockIdx.x * R;             // first owned row
  const int64_t r1 = min(r0 + R, a.n);                          // one past last
  const int64_t nown = r1 > r0 ? r1 - r0 : 0;
  const int w = a.w;
  load_panel<PT>(sm, a.A, a.ld, r0, a.j, nown, w, R);
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int c = 0; c < w; ++c) {
    const int64_t d = a.j + c;                 // global row of the diagonal
    const int ph = c & 1;
    // 1. local pivot candidate among owned rows >= d
    double bv = -1.0;
    int64_t br = INT64_MAX;
    for (int64_t r = threadIdx.x; r < nown; r += PT) {
      const int64_t g = r0 + r;
      if (g < d) continue;
      const double v = fabs((double)sm[c * R + r]);
      if (v > bv || (v == bv && g < br)) { bv = v; br = g; }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const double ov = __shfl_down_sync(0xffffffffu, bv, off);
      const int64_t orr = __shfl_down_sync(0xffffffffu, br, off);
      if (ov > bv || (ov == bv && orr < br)) { bv = ov; br = orr; }
    }
    if (lane == 0) { red_v[wid] = bv; red_r[wid] = br; }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int q = 1; q < PT / 32; ++q)
        if (red_v[q] > bv || (red_v[q] == bv && red_r[q] < br)) { bv = red_v[q]; br = red_r[q]; }
      a.cand_val[ph * MAX_CTAS + blockIdx.x] = bv;
      a.cand_row[ph * MAX_CTAS + blockIdx.x] = br;
      s_p = br;
    }
    __syncthreads();
    // publish the candidate row and, if owned here, row d (panel columns only)
    if (s_p >= r0 && s_p < r1)
      for (int q = threadIdx.x; q < w; q += PT)
        a.cand_data[((int64_t)ph * MAX_CTAS + blockIdx.x) * NB + q] = sm[q * R + (s_p - r0)];
    if (d >= r0 && d < r1)
      for (int q = threadIdx.x; q < w; q += PT) a.drow[ph * NB + q] = sm[q * R + (d - r0)];
    // 2. all CTAs meet (the barrier orders this block's writes before its
    //    arrival: bar.sync, then a device fence by the arriving thread)
    if (!grid_barrier(a.ctl, gridDim.x, a.status, a.wait_ns)) return;
    // 3. every CTA picks the same pivot: warp 0 reads the candidates in
    //    parallel and reduces them (ties to the smallest row index)
    if (wid == 0) {
      double v = -1.0;
      int64_t p = INT64_MAX;
      int win = -1;
      for (unsigned int b = lane; b < gridDim.x; b += 32) {
        const double cv = __ldcg(a.cand_val + ph * MAX_CTAS + b);
        const int64_t cr = __ldcg(reinterpret_cast<const long long*>(a.cand_row) + ph * MAX_CTAS + b);
        if (cv > v || (cv == v && cr < p)) { v = cv; p = cr; win = (int)b; }
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const double ov = __shfl_down_sync(0xffffffffu, v, off);
        const int64_t op = __shfl_down_sync(0xffffffffu, p, off);
        const int ow = __shfl_down_sync(0xffffffffu, win, off);
        if (ov > v || (ov == v && op < p)) { v = ov; p = op; win = ow; }
      }
      if (lane == 0) {
        if (v <= 0.0) {             // exact zero column: singular, keep going
          if (atomicCAS(a.status, 0, (int32_t)ARMA_ERR_SINGULAR) == 0) *a.info = d + 1;
          p = d;
          win = -1;
        }
        s_p = p;
        s_win = win;
        if (blockIdx.x == 0) a.piv[d] = (int32_t)p;
      }
    }
    __syncthreads();
    const int64_t p = s_p;
    const int win = s_win;
    // pivot row values (panel columns)
    for (int q = threadIdx.x; q < w; q += PT) {
      T u;
      if (win >= 0) u = __ldcg(a.cand_data + ((int64_t)ph * MAX_CTAS + win) * NB + q);
      else u = __ldcg(a.drow + ph * NB + q);
      s_u[q] = u;
    }
    __syncthreads();
    // 4. swap rows d and p inside the panel
    if (p != d) {
      if (d >= r0 && d < r1)
        for (int q = threadIdx.x; q < w; q += PT) sm[q * R + (d - r0)] = s_u[q];
      if (p >= r0 && p < r1)
        for (int q = threadIdx.x; q < w; q += PT) sm[q * R + (p - r0)] = __ldcg(a.drow + ph * NB + q);
    }
    __syncthreads();
    // 5. scale the column below the pivot and update the rest of the panel
    const T pv = s_u[c];
    if (win >= 0) {
      for (int64_t r = threadIdx.x; r < nown; r += PT) {
        if (r0 + r <= d) continue;
        const T l = sm[c * R + r] / pv;
        sm[c * R + r] = l;
        for (int q = c + 1; q < w; ++q) sm[q * R + r] -= l * s_u[q];
      }
    }
    __syncthreads();
  }
  for (int64_t t = threadIdx.x; t < nown * w; t += PT) {
    const int64_t c = t / nown, r = t - c * nown;
    a.A[(r0 + r) + (a.j + c) * a.ld] = sm[c * R + r];
  }
}

// The same panel factorisation with the CTAs of one thread-block cluster:
// candidates, the pivot row and row d are read from the owning CTA's shared
// memory through the cluster's distributed shared memory, and the per-column
// meeting point is the cluster's hardware barrier (all CTAs of a cluster are
// co-resident, so the barrier needs no spin).  512 threads per CTA: thread
// (slot, seg) owns rows slot, slot + 128, ... of the CTA and panel columns
// 16 seg .. 16 seg + 15, so the rank-1 update of a column is spread over all
// threads.  Every warp selects the pivot from the CTAs' candidates itself,
// which saves a block barrier per column.  Used when the panel fits the
// cluster's shared memory.
constexpr int CPT = 512;
constexpr int CSLOTS = CPT / 4;

template <typename T>
__device__ __forceinline__ void argmax_step(T& v, int64_t& r, int& win, int off) {
  const T ov = __shfl_down_sync(0xffffffffu, v, off);
  const int64_t orr = __shfl_down_sync(0xffffffffu, r, off);
  const int ow = __shfl_down_sync(0xffffffffu, win, off);
  if (ov > v || (ov == v && orr < r)) { v = ov; r = orr; win = ow; }
}

template <typename T>
__global__ void __launch_bounds__(CPT) panel_cluster_kernel(const __grid_constant__ PanelArgs<T> a) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sm = reinterpret_cast<T*>(smraw);   // [w][R] column-major
  __shared__ T red_v[CPT / 32];
  __shared__ int64_t red_r[CPT / 32];
  __shared__ T c_val[2];                  // this CTA's candidate, per phase
  __shared__ int64_t c_row[2];
  __shared__ __align__(16) T c_data[2][NB];   // its candidate row
  __shared__ __align__(16) T c_drow[2][NB];   // row d when owned here
  __shared__ __align__(16) T s_u[NB];     // the pivot row
  __shared__ int64_t s_p;
  __shared__ int s_win;
  const unsigned int nranks = cl.num_blocks();
  const unsigned int rank = cl.block_rank();
  const int64_t R = a.rows_per_cta;
  const int64_t r0 = a.j + (int64_t)rank * R;
  const int64_t r1 = min(r0 + R, a.n);
  const int64_t nown = r1 > r0 ? r1 - r0 : 0;
  const int w = a.w;
  load_panel<CPT>(sm, a.A, a.ld, r0, a.j, nown, w, R);
  __syncthreads();
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int slot = tid & (CSLOTS - 1), seg = tid / CSLOTS;
  for (int c = 0; c < w; ++c) {
    const int64_t d = a.j + c;
    const int ph = c & 1;
    const unsigned int downer = (unsigned int)((d - a.j) / R);
    // A. this CTA's candidate: largest |value| of column c among rows >= d
    {
      T bv = (T)-1;
      int64_t br = INT64_MAX;
      int dummy = 0;
      for (int64_t r = tid; r < nown; r += CPT) {
        const int64_t g = r0 + r;
        if (g < d) continue;
        const T v = fabs(sm[c * R + r]);
        if (v > bv || (v == bv && g < br)) { bv = v; br = g; }
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) argmax_step(bv, br, dummy, off);
      if (lane == 0) { red_v[wid] = bv; red_r[wid] = br; }
      if (wid == 1 && rank == downer)
        for (int q = lane; q < w; q += 32) c_drow[ph][q] = sm[q * R + (d - r0)];
      __syncthreads();
      if (wid == 0) {
        bv = lane < CPT / 32 ? red_v[lane] : (T)-1;
        br = lane < CPT / 32 ? red_r[lane] : INT64_MAX;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) argmax_step(bv, br, dummy, off);
        br = __shfl_sync(0xffffffffu, br, 0);
        if (lane == 0) { c_val[ph] = bv; c_row[ph] = br; }
        if (br >= r0 && br < r1)
          for (int q = lane; q < w; q += 32) c_data[ph][q] = sm[q * R + (br - r0)];
      }
    }
    cl.sync();
    // C. warp 0 picks the pivot from the CTAs' candidates and copies the
    //    pivot row into this CTA's shared memory
    if (wid == 0) {
      T v = (T)-1;
      int64_t pp = INT64_MAX;
      int wn = -1;
      if ((unsigned int)lane < nranks) {
        v = *cl.map_shared_rank(&c_val[ph], (unsigned int)lane);
        pp = *cl.map_shared_rank(&c_row[ph], (unsigned int)lane);
        wn = lane;
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) argmax_step(v, pp, wn, off);
      v = __shfl_sync(0xffffffffu, v, 0);
      pp = __shfl_sync(0xffffffffu, pp, 0);
      wn = __shfl_sync(0xffffffffu, wn, 0);
      if (v <= (T)0) {                    // exact zero column: singular, keep going
        pp = d;
        wn = -1;
      }
      const T* src = wn >= 0 ? cl.map_shared_rank(&c_data[ph][0], (unsigned int)wn)
                             : cl.map_shared_rank(&c_drow[ph][0], downer);
      for (int q = lane; q < w; q += 32) s_u[q] = src[q];
      if (lane == 0) {
        s_p = pp;
        s_win = wn;
        if (rank == 0) {
          if (wn < 0 && atomicCAS(a.status, 0, (int32_t)ARMA_ERR_SINGULAR) == 0) *a.info = d + 1;
          a.piv[d] = (int32_t)pp;
        }
      }
    }
    __syncthreads();
    const int64_t p = s_p;
    const int win = s_win;
    T u[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) u[k] = seg * 16 + k < w ? s_u[seg * 16 + k] : (T)0;
    const T pv = s_u[c];
    // D. swap rows d and p (each thread its own columns), scale column c
    if (p != d) {
      const int64_t rd = d - r0, rp = p - r0;
      if (rd >= 0 && rd < nown && (rd & (CSLOTS - 1)) == slot) {
#pragma unroll
        for (int k = 0; k < 16; ++k)
          if (seg * 16 + k < w) sm[(seg * 16 + k) * R + rd] = u[k];
      }
      if (rp >= 0 && rp < nown && (rp & (CSLOTS - 1)) == slot) {
        const T* dr = cl.map_shared_rank(&c_drow[ph][0], downer);
#pragma unroll
        for (int k = 0; k < 16; ++k)
          if (seg * 16 + k < w) sm[(seg * 16 + k) * R + rp] = dr[seg * 16 + k];
      }
    }
    if (win >= 0 && seg == (c >> 4))
      for (int64_t r = slot; r < nown; r += CSLOTS)
        if (r0 + r > d) sm[c * R + r] = sm[c * R + r] / pv;
    __syncthreads();
    // E. rank-1 update of the remaining columns of this thread's rows
    if (win >= 0 && seg * 16 + 15 > c)
      for (int64_t r = slot; r < nown; r += CSLOTS) {
        if (r0 + r <= d) continue;
        const T l = sm[c * R + r];
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          const int q = seg * 16 + k;
          if (q > c && q < w) sm[q * R + r] -= l * u[k];
        }
      }
    __syncthreads();
  }
  cl.sync();                              // peers may still read this CTA's buffers
  for (int64_t t = threadIdx.x; t < nown * w; t += CPT) {
    const int64_t c = t / nown, r = t - c * nown;
    a.A[(r0 + r) + (a.j + c) * a.ld] = sm[c * R + r];
  }
}

// The cluster panel with the panel held in registers, one row per thread:
// thread t of a CTA keeps row t of the CTA's rows, all 64 panel columns, so
// a row's multiplier never leaves its thread and the rank-1 update touches
// no shared memory.  Per column: warp candidates -> CTA barrier -> the CTA's
// candidate and its row published -> cluster barrier -> warp 0 reads the
// CTAs' candidates, then (one more round trip) the winning row and, in the
// CTA that holds the pivot row, row d -> CTA barrier -> swap, multiplier,
// update.  The column loop is unrolled by 16 (static register index within a
// group of 16 columns, the group at run time).  Pivot candidates are compared
// as monotone integer keys of |value| (warp max/min reductions); ties go to
// the smallest row.  Pivots are kept in shared memory and stored once at the
// end.  Rows per CTA <= RT and >= w (the diagonal block lies in CTA 0).
constexpr int RT = 256;

__device__ __forceinline__ uint32_t abs_key(float v) { return (__float_as_uint(v) & 0x7fffffffu) + 1u; }
__device__ __forceinline__ uint64_t abs_key(double v) {
  return ((uint64_t)__double_as_longlong(v) & 0x7fffffffffffffffull) + 1ull;
}

// warp-wide largest key, and the smallest row holding it
__device__ __forceinline__ void warp_argmax(uint32_t& key, uint32_t& row) {
  const uint32_t m = __reduce_max_sync(0xffffffffu, key);
  row = __reduce_min_sync(0xffffffffu, key == m ? row : 0xffffffffu);
  key = m;
}
__device__ __forceinline__ void warp_argmax(uint64_t& key, uint32_t& row) {
  const uint32_t hi = __reduce_max_sync(0xffffffffu, (uint32_t)(key >> 32));
  const uint32_t lo = __reduce_max_sync(0xffffffffu, (uint32_t)(key >> 32) == hi ? (uint32_t)key : 0u);
  const uint64_t m = ((uint64_t)hi << 32) | lo;
  row = __reduce_min_sync(0xffffffffu, key == m ? row : 0xffffffffu);
  key = m;
}

// f(integral_constant<int, I>) for each I of the sequence, in order
template <typename F, int... Is>
__device__ __forceinline__ void static_for(F& f, std::integer_sequence<int, Is...>) {
  (f(std::integral_constant<int, Is>{}), ...);
}

// x[cb][k], the group cb at run time
template <typename T, int k>
__device__ __forceinline__ T group_col(const T (&x)[4][16], int cb) {
  T v = x[0][k];
#pragma unroll
  for (int g = 1; g < 4; ++g) v = cb == g ? x[g][k] : v;
  return v;
}

template <typename T>
__global__ void __launch_bounds__(RT, 1) panel_reg_kernel(const __grid_constant__ PanelArgs<T> a) {
  using K = typename std::conditional<sizeof(T) == 8, uint64_t, uint32_t>::type;
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  __shared__ K wkey[RT / 32];             // per warp
  __shared__ uint32_t wrow[RT / 32];
  __shared__ K c_key[2];                  // this CTA's candidate, per phase
  __shared__ uint32_t c_row[2];
  __shared__ __align__(16) T c_data[2][NB];   // its candidate row
  __shared__ __align__(16) T c_drow[2][NB];   // row d (CTA 0)
  __shared__ __align__(16) T s_u[NB];     // the pivot row
  __shared__ __align__(16) T s_d[NB];     // row d, in the CTA that holds the pivot row
  __shared__ int32_t s_piv[NB];           // pivot rows, stored once at the end
  __shared__ int64_t s_p;
  __shared__ int s_win;
  const unsigned int nranks = cl.num_blocks();
  const unsigned int rank = cl.block_rank();
  const int R = (int)a.rows_per_cta;
  const int64_t r0 = a.j + (int64_t)rank * R;
  const int64_t r1 = min(r0 + R, a.n);
  const int nown = r1 > r0 ? (int)(r1 - r0) : 0;
  const int w = a.w;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const bool own = tid < nown;
  const int64_t grow = r0 + tid;          // this thread's row
  T x[4][16];
#pragma unroll
  for (int g = 0; g < 4; ++g)
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      const int col = 16 * g + kk;
      x[g][kk] = (own && col < w) ? a.A[grow + (a.j + col) * a.ld] : (T)0;
    }
  for (int q = tid; q < NB; q += RT) s_u[q] = s_d[q] = (T)0;   // columns >= w stay zero
  __syncthreads();
  for (int cb = 0; cb < 4 && 16 * cb < w; ++cb) {
    auto column = [&](auto kc) {
      constexpr int k = decltype(kc)::value;
      const int c = 16 * cb + k;
      if (c >= w) return;
      const int64_t d = a.j + c;
      const int ph = c & 1;
      // A. warp candidates of column c (rows >= d)
      K key = 0;
      uint32_t row = 0xffffffffu;
      if (own && grow >= d) { key = abs_key(group_col<T, k>(x, cb)); row = (uint32_t)grow; }
      warp_argmax(key, row);
      if (lane == 0) { wkey[wid] = key; wrow[wid] = row; }
      if (rank == 0 && grow == d) {
#pragma unroll
        for (int g = 0; g < 4; ++g)
#pragma unroll
          for (int kk = 0; kk < 16; ++kk) c_drow[ph][16 * g + kk] = x[g][kk];
      }
      __syncthreads();
      // B. the CTA's candidate; its owner publishes the row
      K ck = wkey[0];
      uint32_t cr = wrow[0];
#pragma unroll
      for (int q = 1; q < RT / 32; ++q)
        if (wkey[q] > ck || (wkey[q] == ck && wrow[q] < cr)) { ck = wkey[q]; cr = wrow[q]; }
      if (tid == 0) { c_key[ph] = ck; c_row[ph] = cr; }
      if (ck != 0 && (uint32_t)grow == cr && own) {
#pragma unroll
        for (int g = 0; g < 4; ++g)
#pragma unroll
          for (int kk = 0; kk < 16; ++kk) c_data[ph][16 * g + kk] = x[g][kk];
      }
      cl.sync();
      // C. warp 0 selects the pivot among the CTAs' candidates and copies the
      //    pivot row (and, where the pivot row lies in this CTA, row d) into
      //    this CTA's shared memory: one remote read per value and CTA
      if (wid == 0) {
        K gk = 0;
        uint32_t gr = 0xffffffffu, mine = 0xffffffffu;
        if ((unsigned int)lane < nranks) {
          gk = *cl.map_shared_rank(&c_key[ph], (unsigned int)lane);
          gr = mine = *cl.map_shared_rank(&c_row[ph], (unsigned int)lane);
        }
        warp_argmax(gk, gr);
        const bool sing = gk <= (K)1;     // |value| = 0 everywhere below d
        const int wn = sing ? -1 : __ffs(__ballot_sync(0xffffffffu, mine == gr)) - 1;
        const int64_t p = sing ? d : (int64_t)gr;
        const T* src = wn >= 0 ? cl.map_shared_rank(&c_data[ph][0], (unsigned int)wn)
                               : cl.map_shared_rank(&c_drow[ph][0], 0u);
        const bool here = p != d && p >= r0 && p < r0 + nown;
        const T* drow = cl.map_shared_rank(&c_drow[ph][0], 0u);
        for (int q = lane; q < w; q += 32) {
          const T uq = src[q];
          const T dq = here ? drow[q] : (T)0;
          s_u[q] = uq;
          if (here) s_d[q] = dq;
        }
        if (lane == 0) {
          s_p = p;
          s_win = wn;
          s_piv[c] = (int32_t)p;
          if (rank == 0 && sing && atomicCAS(a.status, 0, (int32_t)ARMA_ERR_SINGULAR) == 0) *a.info = d + 1;
        }
      }
      __syncthreads();
      const int64_t p = s_p;
      if (s_win < 0) return;              // singular column: nothing to eliminate
      const T pv = s_u[c];
      // D. swap rows d and p
      if (p != d) {
        if (grow == d) {
#pragma unroll
          for (int g = 0; g < 4; ++g)
#pragma unroll
            for (int kk = 0; kk < 16; ++kk) x[g][kk] = s_u[16 * g + kk];
        } else if (grow == p) {
#pragma unroll
          for (int g = 0; g < 4; ++g)
#pragma unroll
            for (int kk = 0; kk < 16; ++kk) x[g][kk] = s_d[16 * g + kk];
        }
      }
      // E. the multiplier of this row, then the update of the columns right of c
      if (own && grow > d) {
        const T l = group_col<T, k>(x, cb) / pv;
#pragma unroll
        for (int g = 0; g < 4; ++g) {
          if (g == cb) {
            x[g][k] = l;
#pragma unroll
            for (int kk = k + 1; kk < 16; ++kk) x[g][kk] -= l * s_u[16 * g + kk];
          } else if (g > cb) {
#pragma unroll
            for (int kk = 0; kk < 16; ++kk) x[g][kk] -= l * s_u[16 * g + kk];
          }
        }
      }
    };
    static_for(column, std::make_integer_sequence<int, 16>{});
  }
  cl.sync();                              // peers may still read this CTA's buffers
  if (rank == 0)
    for (int q = tid; q < w; q += RT) a.piv[a.j + q] = s_piv[q];
#pragma unroll
  for (int g = 0; g < 4; ++g)
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      const int col = 16 * g + kk;
      if (own && col < w) a.A[grow + (a.j + col) * a.ld] = x[g][kk];
    }
}

// the panel's row swaps applied to columns outside [j, j + w)
template <typename T>
__global__ void laswp_kernel(T* A, int64_t ld, int64_t n, int64_t j, int w, const int32_t* piv) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t others = n - w;
  if (k >= others) return;
  const int64_t col = k < j ? k : k + w;
  for (int c = 0; c < w; ++c) {
    const int64_t d = j + c, p = piv[d];
    if (p != d) {
      const T t = A[d + col * ld];
      A[d + col * ld] = A[p + col * ld];
      A[p + col * ld] = t;
    }
  }
}

// the panel's row swaps (rows j .. j + w - 1 with piv[]) applied to the
// columns [c0, c1)
template <typename T>
__global__ void laswp_range_kernel(T* A, int64_t ld, int64_t j, int w, const int32_t* piv, int64_t c0, int64_t c1) {
  const int64_t col = c0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= c1) return;
  for (int c = 0; c < w; ++c) {
    const int64_t d = j + c, p = piv[d];
    if (p != d) {
      const T t = A[d + col * ld];
      A[d + col * ld] = A[p + col * ld];
      A[p + col * ld] = t;
    }
  }
}

// The next panel's columns of the trailing update, FP32:
// A(r, c0 + c) -= sum_{k < w} A(r, j + k) A(j + k, c0 + c) for rows r in
// [j + w, n) and c < nc <= 64.  A CTA takes 32 rows: the w x nc block of U
// and its 32 x w block of L in shared memory, each thread 8 outputs of one
// row (K in ascending order).  Both factorisations use it for these columns.
constexpr int NU_ROWS = 32;
__global__ void __launch_bounds__(256) next_update_kernel(float* A, int64_t ld, int64_t n, int64_t j, int w,
                                                          int64_t c0, int nc) {
  __shared__ float U[NB][NB + 1];          // U[k][c]
  __shared__ float Lt[NU_ROWS][NB + 1];    // Lt[row][k]
  const int t = threadIdx.x;
  const int64_t rb = j + w + (int64_t)blockIdx.x * NU_ROWS;
  for (int idx = t; idx < NB * NB; idx += 256) {
    const int k = idx % NB, c = idx / NB;
    U[k][c] = (k < w && c < nc) ? A[(j + k) + (c0 + c) * ld] : 0.f;
  }
  for (int idx = t; idx < NU_ROWS * NB; idx += 256) {
    const int row = idx % NU_ROWS, k = idx / NU_ROWS;
    Lt[row][k] = (rb + row < n && k < w) ? A[(rb + row) + (j + k) * ld] : 0.f;
  }
  __syncthreads();
  const int row = t >> 3, cg = t & 7;
  const int64_t r = rb + row;
  if (r >= n) return;
  float acc[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) acc[q] = 0.f;
  for (int k = 0; k < w; ++k) {
    const float l = Lt[row][k];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = fmaf(l, U[k][8 * cg + q], acc[q]);
  }
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int c = 8 * cg + q;
    if (c < nc) A[r + (c0 + c) * ld] -= acc[q];
  }
}

// U12 = L11^-1 A12 (L11 unit lower w x w): one warp per column of A12, lane
// l holding rows l and l + 32; the column is read and written coalesced
// (columns [c0, n) of the block row; c0 = 0 means j + w)
template <typename T>
__global__ void __launch_bounds__(256) trsm_kernel(T* A, int64_t ld, int64_t n, int64_t j, int w, int64_t c0 = 0) {
  __shared__ T L[NB * NB];
  for (int t = threadIdx.x; t < w * w; t += blockDim.x) {
    const int r = t % w, c = t / w;
    L[c * NB + r] = A[(j + r) + (j + c) * ld];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t col = (c0 ? c0 : j + w) + (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (col >= n) return;
  T* x = A + j + col * ld;
  T x0 = lane < w ? x[lane] : (T)0;
  T x1 = lane + 32 < w ? x[lane + 32] : (T)0;
  for (int r = 0; r < w; ++r) {
    const T xr = __shfl_sync(0xffffffffu, r < 32 ? x0 : x1, r & 31);
    if (lane > r) x0 -= L[r * NB + lane] * xr;
    if (lane + 32 > r && lane + 32 < w) x1 -= L[r * NB + lane + 32] * xr;
  }
  if (lane < w) x[lane] = x0;
  if (lane + 32 < w) x[lane + 32] = x1;
}

// ---- blocked substitution helpers (64 x 64 blocks, 256 threads) ----

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release(unsigned int* p, unsigned int v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// dst[c * NB + r] = src[r + c * ld] for r < rows, c < cols, zero elsewhere
template <typename T>
__device__ __forceinline__ void load_block(T* dst, const T* src, int64_t ld, int rows, int cols) {
  T v[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const int t = threadIdx.x + 256 * k, r = t & (NB - 1), c = t >> 6;
    v[k] = (r < rows && c < cols) ? src[r + (int64_t)c * ld] : (T)0;
  }
#pragma unroll
  for (int k = 0; k < 16; ++k) dst[threadIdx.x + 256 * k] = v[k];
}

// dst[c * (NB + 1) + r] = src[r + c * ld] (through L2: data other CTAs wrote)
template <typename T>
__device__ __forceinline__ void load_cols_cg(T* dst, const T* src, int64_t ld, int rows, int cols) {
  T v[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const int t = threadIdx.x + 256 * k, r = t & (NB - 1), c = t >> 6;
    v[k] = (r < rows && c < cols) ? __ldcg(src + r + (int64_t)c * ld) : (T)0;
  }
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const int t = threadIdx.x + 256 * k, r = t & (NB - 1), c = t >> 6;
    dst[c * (NB + 1) + r] = v[k];
  }
}

__device__ __forceinline__ void ld16(const float* p, float (&o)[16]) {
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    const float4 t = reinterpret_cast<const float4*>(p)[v];
    o[4 * v] = t.x; o[4 * v + 1] = t.y; o[4 * v + 2] = t.z; o[4 * v + 3] = t.w;
  }
}
__device__ __forceinline__ void ld16(const double* p, double (&o)[16]) {
#pragma unroll
  for (int v = 0; v < 8; ++v) {
    const double2 t = reinterpret_cast<const double2*>(p)[v];
    o[2 * v] = t.x; o[2 * v + 1] = t.y;
  }
}

// thread (col, q) holds rows q*16 .. q*16+15 of column col in y:
// y -= M X_k over m < kw, M column-major in Ms, X_k in Xs[col * (NB + 1) + m]
template <typename T>
__device__ __forceinline__ void block_update(T (&y)[16], const T* Ms, const T* Xs, int col, int q, int kw) {
  for (int m = 0; m < kw; ++m) {
    const T x = Xs[col * (NB + 1) + m];
    T mv[16];
    ld16(Ms + m * NB + q * 16, mv);
#pragma unroll
    for (int k = 0; k < 16; ++k) y[k] -= mv[k] * x;
  }
}

// lower (unit diagonal unless !unit) or upper solve with the diagonal block
// D (column-major, dinv = reciprocals of its diagonal), rows distributed as
// in block_update; the four threads of a column are consecutive lanes
template <typename T, bool LOWER>
__device__ __forceinline__ void block_solve(T (&y)[16], const T* D, const T* dinv, int w, int q, int lane,
                                            bool unit = true) {
  const int base = lane & ~3;
  if (LOWER) {
#pragma unroll
    for (int qq = 0; qq < 4; ++qq)
#pragma unroll
      for (int kk = 0; kk < 16; ++kk) {
        const int r = qq * 16 + kk;
        T yr = __shfl_sync(0xffffffffu, y[kk], base | qq);
        if (!unit && r < w) {
          yr *= dinv[r];
          if (q == qq) y[kk] = yr;
        }
        if (r < w && q >= qq) {
          T dv[16];
          ld16(D + r * NB + q * 16, dv);
#pragma unroll
          for (int k = 0; k < 16; ++k)
            if (q * 16 + k > r) y[k] -= dv[k] * yr;
        }
      }
  } else {
#pragma unroll
    for (int qq = 3; qq >= 0; --qq)
#pragma unroll
      for (int kk = 15; kk >= 0; --kk) {
        const int r = qq * 16 + kk;
        T yr = __shfl_sync(0xffffffffu, y[kk], base | qq);
        if (r < w) {
          yr *= dinv[r];
          if (q == qq) y[kk] = yr;
          if (q <= qq) {
            T dv[16];
            ld16(D + r * NB + q * 16, dv);
#pragma unroll
            for (int k = 0; k < 16; ++k)
              if (q * 16 + k < r) y[k] -= dv[k] * yr;
          }
        }
      }
  }
}

// Inverses of one diagonal block (w <= 64 rows at src, leading dimension
// lda): Linv = L^-1 of its lower part (unit diagonal unless lower_nonunit)
// and, when Uinv is not null, Uinv = U^-1 of its upper part; each 64 x 64
// column-major, zero-padded past w, by the block solve applied to the
// identity.  D (NB * NB) and dinv (NB) are shared memory; 256 threads.
template <typename T>
__device__ __forceinline__ void invert_block(const T* src, int64_t lda, int w, T* D, T* dinv, T* Linv, T* Uinv,
                                             bool lower_nonunit) {
  const int tid = threadIdx.x, lane = tid & 31, col = tid >> 2, q = tid & 3;
  load_block(D, src, lda, w, w);
  __syncthreads();
  if (tid < NB) {
    const T p = D[tid * NB + tid];
    dinv[tid] = (tid < w && p != (T)0) ? (T)1 / p : (T)0;
  }
  __syncthreads();
  {
    T y[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) y[k] = (q * 16 + k == col && col < w) ? (T)1 : (T)0;
    block_solve<T, true>(y, D, dinv, w, q, lane, !lower_nonunit);
#pragma unroll
    for (int k = 0; k < 16; ++k) Linv[col * NB + q * 16 + k] = y[k];
  }
  if (Uinv) {
    T y[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) y[k] = (q * 16 + k == col && col < w) ? (T)1 : (T)0;
    block_solve<T, false>(y, D, dinv, w, q, lane);
#pragma unroll
    for (int k = 0; k < 16; ++k) Uinv[col * NB + q * 16 + k] = y[k];
  }
}

// inverses of all diagonal blocks: Linv_i = L_ii^-1 (unit lower) and
// Uinv_i = U_ii^-1 of an LU factor (a zero pivot gives a zero row, as in the
// substitution); with lower_nonunit the matrix is a lower-triangular system
// matrix (or a Cholesky factor) and Linv_i inverts its whole lower block
template <typename T>
__global__ void __launch_bounds__(256) inv_diag_kernel(const T* __restrict__ LU, int64_t n, T* Linv, T* Uinv,
                                                       int64_t lda = 0, int lower_nonunit = 0) {
  __shared__ __align__(16) T D[NB * NB];
  __shared__ T dinv[NB];
  if (lda == 0) lda = n;
  const int64_t j = (int64_t)blockIdx.x * NB;
  const int w = (int)(n - j < NB ? n - j : NB);
  invert_block(LU + j + j * lda, lda, w, D, dinv, Linv + (int64_t)blockIdx.x * NB * NB,
               Uinv + (int64_t)blockIdx.x * NB * NB, lower_nonunit != 0);
}

constexpr int CW = 16;          // right-hand sides per CTA of the cooperative substitution
constexpr int XS = CW + 1;      // row stride of its right-hand-side tile in shared memory

template <typename T>
__host__ __device__ inline size_t coop_smem(void) {
  return sizeof(T) * (2 * (size_t)NB * NB + (size_t)NB * XS);
}

__device__ __forceinline__ void ld4(const float* p, float (&o)[4]) {
  const float4 t = *reinterpret_cast<const float4*>(p);
  o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
}
__device__ __forceinline__ void ld4(const double* p, double (&o)[4]) {
  const double2 t0 = reinterpret_cast<const double2*>(p)[0], t1 = reinterpret_cast<const double2*>(p)[1];
  o[0] = t0.x; o[1] = t0.y; o[2] = t1.x; o[3] = t1.y;
}

// The whole substitution y := U^-1 L^-1 y in one cooperative launch.  CTA
// (i, c) owns block row i (64 rows) of a 16-column slice c; thread (col, rq)
// holds rows 4 rq .. 4 rq + 3 of column col.  Forward: for k < i it
// subtracts L_ik z_k as soon as z_k is published (flag per block, release /
// acquire), applies the inverted diagonal block, z_i = Linv_i y_i, and
// publishes z_i to Z.  Backward: likewise with U_ik y_k for k > i and Uinv_i,
// publishing to Y.  The next off-diagonal block is fetched into registers
// while the current one is applied.  Every wait is bounded in time; a wait
// that runs out marks the control block and the status, and every other wait
// then gives up.
// lda is the leading dimension of LU; sweeps selects the forward (bit 0)
// and backward (bit 1) halves: a triangular system matrix needs only one,
// and the result is then in Z (forward only) or Y (backward only, whose
// input is then read from Y).
template <typename T>
__global__ void __launch_bounds__(256) sub_coop_kernel(const T* __restrict__ LU, const T* __restrict__ Linv,
                                                       const T* __restrict__ Uinv, int64_t n, T* Y, T* Z,
                                                       int64_t nrhs, unsigned int* flags, Ctl* ctl,
                                                       int32_t* status, const int* skip, int64_t lda,
                                                       int sweeps, uint64_t wait_ns) {
  if (skip && *skip) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* Ms = reinterpret_cast<T*>(smraw);   // off-diagonal block, Ms[m * NB + r]
  T* Ds = Ms + NB * NB;                  // inverted diagonal block, same layout
  T* Xs = Ds + NB * NB;                  // right-hand-side tile, Xs[m * XS + c]
  __shared__ int s_ok;
  const int nb = gridDim.x, bi = blockIdx.x;
  const int64_t j = (int64_t)bi * NB;
  const int w = (int)(n - j < NB ? n - j : NB);
  const int64_t c0 = (int64_t)blockIdx.y * CW;
  const int ncols = (int)(nrhs - c0 < CW ? nrhs - c0 : CW);
  unsigned int* fwd = flags;                   // one 128-byte line per flag
  unsigned int* bwd = flags + (size_t)nb * gridDim.y * FLAG_STRIDE;
  const int tid = threadIdx.x, col = tid & (CW - 1), rq = tid / CW;
  auto flag = [&](unsigned int* f, int k) { return f + ((size_t)k * gridDim.y + blockIdx.y) * FLAG_STRIDE; };
  auto rows_of = [&](int k) { return (int)(n - (int64_t)k * NB < NB ? n - (int64_t)k * NB : NB); };

  auto wait = [&](const unsigned int* f) -> bool {
    if (tid == 0) {
      int ok = 1;
      const uint64_t t0 = global_ns();
      for (unsigned int it = 0; ld_acquire(f) == 0u; ++it) {
        if (wait_ns == 0 || *(volatile int*)&ctl->err || it > SPIN_LIMIT ||
            ((it & 255u) == 255u && global_ns() - t0 > wait_ns)) {
          atomicExch(&ctl->err, 1);
          atomicCAS(status, 0, (int32_t)ARMA_ERR_TIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
      s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
  };
  // Xs := rows [0, rows) of src's 16-column slice (through L2), zero elsewhere
  auto load_x = [&](const T* src, int rows) {
    T v[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const int t = tid + 256 * p, m = t & (NB - 1), c = t >> 6;
      v[p] = (m < rows && c < ncols) ? __ldcg(src + m + (int64_t)c * n) : (T)0;
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const int t = tid + 256 * p, m = t & (NB - 1), c = t >> 6;
      Xs[m * XS + c] = v[p];
    }
  };
  T mv[16];
  auto fetch_m = [&](const T* src, int rows, int cols) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const int t = tid + 256 * k, r = t & (NB - 1), c = t >> 6;
      mv[k] = (r < rows && c < cols) ? src[r + (int64_t)c * lda] : (T)0;
    }
  };
  auto store_m = [&]() {
#pragma unroll
    for (int k = 0; k < 16; ++k) Ms[tid + 256 * k] = mv[k];
  };
  auto load_d = [&](const T* src) {
#pragma unroll
    for (int k = 0; k < 16; ++k) Ds[tid + 256 * k] = src[tid + 256 * k];
  };
  T y[4];
  // y -= Ms Xs over m < kw
  auto sub = [&](int kw) {
    for (int m = 0; m < kw; ++m) {
      const T x = Xs[m * XS + col];
      T a4[4];
      ld4(Ms + m * NB + 4 * rq, a4);
#pragma unroll
      for (int e = 0; e < 4; ++e) y[e] -= a4[e] * x;
    }
  };
  // y := Ds y (the whole tile goes through Xs)
  auto apply = [&]() {
#pragma unroll
    for (int e = 0; e < 4; ++e) Xs[(4 * rq + e) * XS + col] = y[e];
    __syncthreads();
    T acc[4] = {(T)0, (T)0, (T)0, (T)0};
#pragma unroll 8
    for (int m = 0; m < NB; ++m) {
      const T x = Xs[m * XS + col];
      T a4[4];
      ld4(Ds + m * NB + 4 * rq, a4);
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[e] += a4[e] * x;
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) y[e] = acc[e];
    __syncthreads();
  };
  auto publish = [&](T* dst, unsigned int* f) {
#pragma unroll
    for (int e = 0; e < 4; ++e) Xs[(4 * rq + e) * XS + col] = y[e];
    __syncthreads();
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const int t = tid + 256 * p, r = t & (NB - 1), c = t >> 6;
      if (r < w && c < ncols) dst[r + (int64_t)c * n] = Xs[r * XS + c];
    }
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      st_release(f, 1u);
    }
  };

  load_x(Y + j + c0 * n, w);
  if (sweeps & 1) load_d(Linv + (int64_t)bi * NB * NB);
  __syncthreads();
#pragma unroll
  for (int e = 0; e < 4; ++e) y[e] = Xs[(4 * rq + e) * XS + col];
  __syncthreads();

  if (sweeps & 1) {
    if (bi > 0) fetch_m(LU + j, w, NB);          // L_i0
    for (int k = 0; k < bi; ++k) {                // forward: L_ik, k < i
      store_m();
      if (k + 1 < bi) fetch_m(LU + j + (int64_t)(k + 1) * NB * lda, w, NB);
      if (!wait(flag(fwd, k))) return;
      load_x(Z + (int64_t)k * NB + c0 * n, NB);
      __syncthreads();
      sub(NB);
      __syncthreads();
    }
    apply();
    publish(Z + j + c0 * n, flag(fwd, bi));
  }
  if (!(sweeps & 2)) return;

  load_d(Uinv + (int64_t)bi * NB * NB);
  if (bi < nb - 1) fetch_m(LU + j + (int64_t)(nb - 1) * NB * lda, w, rows_of(nb - 1));
  for (int k = nb - 1; k > bi; --k) {           // backward: U_ik, k > i
    const int wk = rows_of(k);
    store_m();
    if (k - 1 > bi) fetch_m(LU + j + (int64_t)(k - 1) * NB * lda, w, rows_of(k - 1));
    if (!wait(flag(bwd, k))) return;
    load_x(Y + (int64_t)k * NB + c0 * n, wk);
    __syncthreads();
    sub(wk);
    __syncthreads();
  }
  __syncthreads();
  apply();
  publish(Y + j + c0 * n, flag(bwd, bi));
}

// One step of the blocked substitution for diagonal block j (w <= 64 rows)
// and a 64-column slice of the right-hand sides.  Every CTA solves the
// diagonal block redundantly (unit lower L_jj in the forward sweep, U_jj in
// the backward sweep) from Yio's rows [j, j + w), then subtracts the block
// column's product from its own SUB_ROWS rows of Yio in [r_begin,
// r_begin + rows); CTA 0 also writes the solved rows to Yout.  Yio's rows
// [j, j + w) are only read, so CTAs never race on them.
//   solve: 4 threads per column, thread q holding rows 16q .. 16q + 15
//   update: thread (i, g) computes row i for columns g, g + 8, ...
// The fallback when the cooperative substitution does not fit the GPU.
constexpr int SUB_ROWS = 32;

template <typename T>
__host__ __device__ inline size_t sub_smem(void) {
  return sizeof(T) * ((size_t)NB * NB + (size_t)NB * (NB + 1) + (size_t)NB * SUB_ROWS + NB);
}

template <typename T, bool LOWER>
__global__ void __launch_bounds__(256) sub_step_kernel(const T* __restrict__ LU, int64_t n, int64_t j, int w,
                                                       T* Yio, T* Yout, int64_t nrhs, int64_t r_begin,
                                                       int64_t rows, const int* skip, int64_t lda, int unit) {
  if (skip && *skip) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* D = reinterpret_cast<T*>(smraw);              // [NB][NB], D[c * NB + r]
  T* Ys = D + NB * NB;                              // [64][NB + 1], Ys[col * (NB + 1) + r]
  T* At = Ys + NB * (NB + 1);                       // [NB][SUB_ROWS], At[r * SUB_ROWS + i]
  T* dinv = At + NB * SUB_ROWS;                     // [NB]
  const int tid = threadIdx.x, lane = tid & 31;
  const int64_t c0 = (int64_t)blockIdx.y * 64;
  const int ncols = (int)(nrhs - c0 < 64 ? nrhs - c0 : 64);
  const int64_t rb = r_begin + (int64_t)blockIdx.x * SUB_ROWS;
  const int64_t rem = r_begin + rows - rb;
  const int nr = (int)(rem < SUB_ROWS ? (rem > 0 ? rem : 0) : SUB_ROWS);
  load_block(D, LU + j + j * lda, lda, w, w);
  load_cols_cg(Ys, Yio + j + c0 * n, n, w, ncols);
  {
    T v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int t = tid + 256 * k, i = t & (SUB_ROWS - 1), r = t / SUB_ROWS;
      v[k] = (i < nr && r < w) ? LU[(rb + i) + (j + r) * lda] : (T)0;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) At[tid + 256 * k] = v[k];
  }
  __syncthreads();
  if (tid < NB) {
    const T p = D[tid * NB + tid];
    dinv[tid] = (tid < w && p != (T)0) ? (T)1 / p : (T)0;
  }
  const int col = tid >> 2, q = tid & 3;
  T y[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) y[k] = Ys[col * (NB + 1) + q * 16 + k];
  __syncthreads();
  block_solve<T, LOWER>(y, D, dinv, w, q, lane, unit != 0);
#pragma unroll
  for (int k = 0; k < 16; ++k) Ys[col * (NB + 1) + q * 16 + k] = y[k];
  __syncthreads();
  if (blockIdx.x == 0)
    for (int t = tid; t < NB * 64; t += 256) {
      const int r = t & (NB - 1), c = t >> 6;
      if (r < w && c < ncols) Yout[(j + r) + (c0 + c) * n] = Ys[c * (NB + 1) + r];
    }
  if (nr == 0) return;
  const int i = tid & (SUB_ROWS - 1), g = tid / SUB_ROWS;
  T acc[8];
#pragma unroll
  for (int m = 0; m < 8; ++m) acc[m] = 0;
  for (int r = 0; r < w; ++r) {
    const T av = At[r * SUB_ROWS + i];
#pragma unroll
    for (int m = 0; m < 8; ++m) acc[m] += av * Ys[(g + 8 * m) * (NB + 1) + r];
  }
  if (i < nr)
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const int c = g + 8 * m;
      if (c < ncols) {
        T* p = Yio + (rb + i) + (c0 + c) * n;
        *p = *p - acc[m];
      }
    }
}


// perm = composition of the row swaps; Y(:, c) = P * B(:, c) (B null: identity).
// The swaps are sequential; with n <= PERM_SMEM they run in shared memory
// (one thread), after the whole block has staged piv and the identity.
constexpr int64_t PERM_SMEM = 24576;

__global__ void __launch_bounds__(1024) perm_kernel(const int32_t* piv, int32_t* perm, int64_t n) {
  extern __shared__ int32_t sp[];        // [n] perm, [n] piv when n <= PERM_SMEM
  if (n <= PERM_SMEM) {
    int32_t* sperm = sp;
    int32_t* spiv = sp + n;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
      sperm[i] = (int32_t)i;
      spiv[i] = piv[i];
    }
    __syncthreads();
    if (threadIdx.x == 0)
      for (int64_t d = 0; d < n; ++d) {
        const int32_t p = spiv[d];
        const int32_t t = sperm[d];
        sperm[d] = sperm[p];
        sperm[p] = t;
      }
    __syncthreads();
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) perm[i] = sperm[i];
    return;
  }
  if (threadIdx.x != 0) return;
  for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
  for (int64_t d = 0; d < n; ++d) {
    const int64_t p = piv[d];
    const int32_t t = perm[d];
    perm[d] = perm[p];
    perm[p] = t;
  }
}

cudaError_t launch_perm(const int32_t* piv, int32_t* perm, int64_t n, cudaStream_t s) {
  const size_t smem = n <= PERM_SMEM ? (size_t)n * 8 : 0;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(perm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  perm_kernel<<<1, 1024, smem, s>>>(piv, perm, n);
  return cudaGetLastError();
}

template <typename T>
__global__ void gather_kernel(const void* B, int64_t ldb, int32_t bdt, const int32_t* perm, T* Y, int64_t n,
                              int64_t nrhs, const int* skip) {
  if (skip && *skip) return;
  const int64_t total = n * nrhs;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = t / n, i = t - c * n;
    const int64_t src = perm[i];
    T v;
    if (B) v = load_as<T>(B, src + c * ldb, bdt);
    else v = (src == c) ? (T)1 : (T)0;
    Y[i + c * n] = v;
  }
}

// convert A into the LU work matrix
template <typename T>
__global__ void copy_kernel(const void* A, int64_t lda, int32_t adt, T* W, int64_t n) {
  const int64_t total = n * n;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = t / n, i = t - c * n;
    W[t] = load_as<T>(A, i + c * lda, adt);
  }
}

// X (output, any type) = Y
template <typename T>
__global__ void store_kernel(const T* Y, int64_t n, int64_t nrhs, void* X, int64_t ldx, int32_t xdt) {
  const int64_t total = n * nrhs;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = t / n, i = t - c * n;
    store_as<double>(X, i + c * ldx, xdt, (double)Y[t]);
  }
}

// refinement bookkeeping: sum of squares -> convergence flag
__global__ void ir_check_kernel(Ctl* c, const double* sq, int step, int32_t* status, int64_t* info, int last) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (c->done) return;
  const double nr = sqrt(sq[0]), nx = sqrt(sq[1]);
  const double denom = c->nrmA * nx + c->nrmB;
  const double bwd = denom > 0.0 ? nr / denom : nr;
  c->steps = step;
  if (bwd <= IR_TOL) {
    c->done = 1;
    if (*status == 0) *info = step;   // refinement steps taken
  } else if (last) {
    if (atomicCAS(status, 0, (int32_t)ARMA_ERR_NOCONVERGE) == 0) *info = step;
  }
}

__global__ void norms_init_kernel(Ctl* c, const double* sq) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  c->nrmA = sqrt(sq[0]);
  c->nrmB = sqrt(sq[1]);
}

// x += d (FP64), skipped once converged
__global__ void ir_update_kernel(double* X, const float* D, int64_t total, const int* skip) {
  if (*skip) return;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x)
    X[t] += (double)D[t];
}

// second stage of a sum of squares: add the per-block partials in order
__global__ void sum_partials_kernel(const double* part, int count, double* out, int k) {
  double s = 0.0;
  for (int t = threadIdx.x; t < count; t += blockDim.x) s += part[t];
  double q = 0.0;
  block_sum2(s, q);
  if (threadIdx.x == 0) out[k] = s;
}

__global__ void sumsq_any_kernel(const void* x, int32_t dt, int64_t ld, int64_t rows, int64_t cols,
                                 double* partial) {
  // per-block sums of squares, added up by sum_partials_kernel
  double s = 0.0;
  const int64_t total = rows * cols;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = t / rows, i = t - c * rows;
    const double v = load_as<double>(x, i + c * ld, dt);
    s = fma(v, v, s);
  }
  double q = 0.0;
  block_sum2(s, q);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

struct Layout {
  int64_t lu, piv, perm, cand_val, cand_row, cand_data, drow, ctl, flags, dinv, gemm, y, z, x64, r64, sq, part,
      total;
  int64_t tri_dinv, tri_y, tri_z, band;   // structured solvers (analysed solves only)
  int64_t gemm_bytes;
  int64_t gemm2, gemm2_bytes;              // the look-ahead's next-panel update (FP32 LU)
  bool f64;
  bool refine;
};

// the refinement residual r = B - A X by the sliced FP64 product (A sliced
// once per solve) rather than DFMA: large systems with several right-hand sides
bool sliced_residual(int64_t n, int64_t nrhs, int32_t dfma_residual) {
  return !dfma_residual && n >= 1024 && nrhs >= 8;
}

Layout layout(int64_t n, int64_t nrhs, int32_t tier, int32_t analyse = 0, int32_t dfma_residual = 0) {
  Layout L;
  L.f64 = tier == ARMA_TIER_F64;
  L.refine = tier == ARMA_TIER_LU32_IR64 || tier == ARMA_TIER_BF16;
  const int64_t es = L.f64 ? 8 : 4;
  int64_t off = 0;
  auto take = [&](int64_t bytes) { int64_t o = off; off += (bytes + 255) / 256 * 256; return o; };
  L.lu = take(n * n * es);
  L.piv = take(n * 4);
  L.perm = take(n * 4);
  L.cand_val = take(2 * MAX_CTAS * 8);
  L.cand_row = take(2 * MAX_CTAS * 8);
  L.cand_data = take(2 * MAX_CTAS * NB * es);
  L.drow = take(2 * NB * es);
  L.ctl = take(sizeof(Ctl));
  L.flags = take(2 * ((n + NB - 1) / NB) * ((nrhs + CW - 1) / CW) * 4 * FLAG_STRIDE);
  L.dinv = take(2 * ((n + NB - 1) / NB) * NB * NB * es);
  const int32_t gt = L.f64 ? ARMA_TIER_F64 : tier == ARMA_TIER_BF16 ? ARMA_TIER_BF16 : ARMA_TIER_SPLIT_BF16;
  int64_t gb = gemm_tc_scratch_bytes(n, n, NB, gt);
  if (gb < 64 * n * 8) gb = 64 * n * 8;            // GEMV partials for 1-wide updates
  if (L.f64) {
    const int64_t sb = gemm_simt_scratch_bytes(n, n, NB);
    if (gb < sb) gb = sb;
  }
  if (L.refine) {
    int64_t rb = gemm_simt_scratch_bytes(n, nrhs, n);   // FP64 residual
    if (sliced_residual(n, nrhs, dfma_residual)) {
      const int64_t ob = gemm_ozaki_scratch_bytes(n, nrhs, n);
      if (rb < ob) rb = ob;
    }
    if (gb < rb) gb = rb;
  }
  L.gemm_bytes = gb;
  L.gemm = take(gb);
  L.gemm2_bytes = L.f64 ? 0 : std::max<int64_t>(gemm_tc_scratch_bytes(n, NB, NB, gt) + 1024, 64 * n * 8);
  L.gemm2 = L.f64 ? 0 : take(L.gemm2_bytes);
  L.y = take(n * nrhs * es);
  L.z = take(n * nrhs * es);
  L.x64 = L.refine ? take(n * nrhs * 8) : 0;
  L.r64 = L.refine ? take(n * nrhs * 8) : 0;
  L.sq = take(8 * 8);
  L.part = take(1024 * 8);
  L.tri_dinv = L.tri_y = L.tri_z = L.band = 0;
  if (analyse) {   // sized for FP64 data
    L.tri_dinv = take(2 * ((n + NB - 1) / NB) * NB * NB * 8);
    L.tri_y = take(n * nrhs * 8);
    L.tri_z = take(n * nrhs * 8);
    L.band = take(band_work_bytes(n, nrhs, kBandMaxKl, kBandMaxKu, 8));
  }
  L.total = off + 256;
  return L;
}

// the panel of `rows` rows starting at column pa.j: one cluster of up to 16
// CTAs when it fits their shared memory, else the cooperative grid kernel
template <typename T>
cudaError_t launch_panel(PanelArgs<T>& pa, int64_t rows, int ctas, cudaStream_t s) {
  static std::atomic<int> cluster_probe{-1};   // largest usable cluster size, probed once
  int cluster_max = cluster_probe.load(std::memory_order_acquire);
  if (cluster_max < 0) {
    cluster_max = 8;
    if (cudaFuncSetAttribute(panel_cluster_kernel<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
        cudaSuccess)
      cluster_max = 16;
    cudaGetLastError();
    cluster_probe.store(cluster_max, std::memory_order_release);
  }
  auto cluster_cfg = [&](cudaLaunchConfig_t& cfg, cudaLaunchAttribute* attr, int cs, size_t smem, int threads) {
    memset(&cfg, 0, sizeof cfg);
    cfg.gridDim = dim3((unsigned)cs);
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
  };
  // registers: the smallest cluster with <= RT rows per CTA
  for (int cs = 1; cs <= cluster_max; cs *= 2) {
    const int64_t R = (rows + cs - 1) / cs;
    if (R > RT) continue;
    if (R < pa.w) break;
    if (cs > 8 && cudaFuncSetAttribute(panel_reg_kernel<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
                      cudaSuccess) {
      cudaGetLastError();
      break;
    }
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[1];
    cluster_cfg(cfg, attr, cs, 0, RT);
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, panel_reg_kernel<T>, &cfg) != cudaSuccess || nclusters < 1) {
      cudaGetLastError();
      break;
    }
    PanelArgs<T> pc = pa;
    pc.rows_per_cta = R;
    return cudaLaunchKernelEx(&cfg, panel_reg_kernel<T>, pc);
  }
  // shared memory
  for (int cs = 1; cs <= cluster_max; cs *= 2) {
    const int64_t R = (rows + cs - 1) / cs;
    if (R > PT && cs < cluster_max) continue;       // aim for one row per thread
    const size_t smem = (size_t)R * pa.w * sizeof(T);
    if (smem > 160 * 1024) break;
    if (cudaFuncSetAttribute(panel_cluster_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
      break;
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[1];
    cluster_cfg(cfg, attr, cs, smem, CPT);
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, panel_cluster_kernel<T>, &cfg) != cudaSuccess || nclusters < 1) {
      cudaGetLastError();
      break;
    }
    PanelArgs<T> pc = pa;
    pc.rows_per_cta = R;
    return cudaLaunchKernelEx(&cfg, panel_cluster_kernel<T>, pc);
  }
  cudaGetLastError();
  const size_t smem = (size_t)pa.rows_per_cta * pa.w * sizeof(T);
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(panel_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  void* kargs[] = {&pa};
  return cudaLaunchCooperativeKernel((const void*)panel_kernel<T>, dim3(ctas), dim3(PT), kargs, smem, s);
}

// The look-ahead FP32 factorisation (panels that all fit one register
// cluster, n <= 16 * 256 rows).  The update after panel j is cut in two:
// the next panel's 64 columns N, and the rest R.  A high-priority side
// stream carries the critical path: panel j, the swaps of the columns left of
// it and of N, N's triangular solve and its product update; the caller's
// stream then updates R (swaps, triangular solve, product limited to the SMs
// the panel cluster leaves) while the side stream already factors panel
// j + 1 from N.  Events order the two: the side stream touches N of panel
// j + 1 (part of R of panel j) only after R's update, and R's update starts
// only after panel j's pivots and L21 are final.
int side_stream(cudaStream_t* out) {
  thread_local cudaStream_t streams[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return -1;
  if (!streams[dev]) {
    int lo = 0, hi = 0;
    if (cudaDeviceGetStreamPriorityRange(&lo, &hi) != cudaSuccess) return -1;
    if (cudaStreamCreateWithPriority(&streams[dev], cudaStreamNonBlocking, hi) != cudaSuccess) {
      streams[dev] = nullptr;
      return -1;
    }
  }
  *out = streams[dev];
  return 0;
}

bool lookahead_ok(int64_t n) { return n >= 3 * NB && n <= 16 * RT; }

cudaError_t factor_lookahead(const SolveArgs& a, const Layout& L, char* base, cudaStream_t s, int* launches,
                             bool* done) {
  using T = float;
  *done = false;
  const int64_t n = a.n;
  cudaStream_t h = nullptr;
  if (side_stream(&h) != 0) return cudaSuccess;   // fall back to the one-stream factorisation
  cudaEvent_t ev[4] = {};
  for (int i = 0; i < 4; ++i)
    if (cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming) != cudaSuccess) {
      for (int k = 0; k < i; ++k) cudaEventDestroy(ev[k]);
      cudaGetLastError();
      return cudaSuccess;
    }
  cudaEvent_t ev_start = ev[0], ev_next = ev[1], ev_rest = ev[2], ev_end = ev[3];
  *done = true;
  T* W = reinterpret_cast<T*>(base + L.lu);
  int32_t* piv = reinterpret_cast<int32_t*>(base + L.piv);
  Ctl* ctl = reinterpret_cast<Ctl*>(base + L.ctl);
  const int sms = device_sm_count();
  const int32_t gt = a.tier == ARMA_TIER_BF16 ? ARMA_TIER_BF16 : ARMA_TIER_SPLIT_BF16;
  cudaError_t e = cudaSuccess;
  // the trailing update of columns [c0, c0 + nc) past the next panel's (the
  // tensor-core product; the next panel's columns take next_update_kernel)
  auto gemm = [&](int64_t m, int64_t nc, int64_t k, int64_t j, int64_t c0, char* scratch, int64_t sb, int max_ctas,
                  cudaStream_t st, int32_t tier, int32_t nosplit) -> cudaError_t {
    GemmArgs g;
    memset(&g, 0, sizeof g);
    g.m = m; g.n = nc; g.k = k;
    g.A = W + (j + k) + j * n; g.lda = n; g.ta = 0; g.adt = ARMA_F32;
    g.B = W + j + c0 * n; g.ldb = n; g.tb = 0; g.bdt = ARMA_F32;
    g.C = W + (j + k) + c0 * n; g.ldc = n; g.cdt = ARMA_F32;
    g.D = W + (j + k) + c0 * n; g.ldd = n; g.ddt = ARMA_F32;
    g.alpha = -1.0; g.beta = 1.0;
    g.tier = tier;
    g.nosplit = nosplit;
    g.scratch = scratch; g.scratch_bytes = sb;
    g.status = a.status_code;
    g.max_ctas = max_ctas;
    g.no_gemv = 1;     // the same product kernel for every block width
    return launch_gemm(g, st, launches);
  };
  {
    int64_t blocks = (n * n + 255) / 256, cap = (int64_t)sms * 8;
    copy_kernel<T><<<(unsigned)(blocks < cap ? blocks : cap), 256, 0, s>>>(a.A, a.lda, a.adt, W, n);
    if (launches) ++*launches;
  }
  if ((e = cudaEventRecord(ev_start, s)) != cudaSuccess) goto out;
  if ((e = cudaStreamWaitEvent(h, ev_start, 0)) != cudaSuccess) goto out;
  for (int64_t j = 0; j < n; j += NB) {
    const int w = (int)(n - j < NB ? n - j : NB);
    PanelArgs<T> pa;
    pa.A = W; pa.ld = n; pa.n = n; pa.j = j; pa.w = w;
    const int64_t rows = n - j;
    int ctas = (int)((rows + PT - 1) / PT);
    if (ctas < 1) ctas = 1;
    if (ctas > MAX_CTAS) ctas = MAX_CTAS;
    if (ctas > sms) ctas = sms;
    pa.rows_per_cta = (rows + ctas - 1) / ctas;
    ctas = (int)((rows + pa.rows_per_cta - 1) / pa.rows_per_cta);
    pa.piv = piv;
    pa.cand_val = reinterpret_cast<double*>(base + L.cand_val);
    pa.cand_row = reinterpret_cast<int64_t*>(base + L.cand_row);
    pa.cand_data = reinterpret_cast<T*>(base + L.cand_data);
    pa.drow = reinterpret_cast<T*>(base + L.drow);
    pa.ctl = ctl;
    pa.wait_ns = wait_limit_ns();
    pa.status = a.status_code;
    pa.info = a.status_info;
    if ((e = launch_panel<T>(pa, rows, ctas, h)) != cudaSuccess) goto out;
    if (launches) ++*launches;
    const int64_t rest = n - j - w;
    const int w2 = (int)(rest < NB ? rest : NB);     // the next panel's width
    // R of the previous panel is updated (it holds this panel's N)
    if (j > 0 && (e = cudaStreamWaitEvent(h, ev_rest, 0)) != cudaSuccess) goto out;
    if (w2 > 0) {
      laswp_range_kernel<T><<<1, 256, 0, h>>>(W, n, j, w, piv, j + w, j + w + w2);
      trsm_kernel<T><<<(unsigned)((w2 + 7) / 8), 256, 0, h>>>(W, n, j + w + w2, j, w, j + w);
      if (launches) *launches += 2;
      next_update_kernel<<<(unsigned)((rest + NU_ROWS - 1) / NU_ROWS), 256, 0, h>>>(W, n, n, j, w, j + w, w2);
      if (launches) ++*launches;
    }
    if ((e = cudaEventRecord(ev_next, h)) != cudaSuccess) goto out;
    // the caller's stream: R, then this panel's swaps of the factored columns
    // on the left (nothing on the side stream reads them again)
    if ((e = cudaStreamWaitEvent(s, ev_next, 0)) != cudaSuccess) goto out;
    const int64_t r0 = j + w + w2, rn = n - r0;       // R: columns [r0, n)
    if (rn > 0) {
      laswp_range_kernel<T><<<(unsigned)((rn + 255) / 256), 256, 0, s>>>(W, n, j, w, piv, r0, n);
      trsm_kernel<T><<<(unsigned)((rn + 7) / 8), 256, 0, s>>>(W, n, n, j, w, r0);
      if (launches) *launches += 2;
      if ((e = gemm(rest, rn, w, j, r0, base + L.gemm, L.gemm_bytes, sms - 16 > 1 ? sms - 16 : 1, s, gt, 0)) !=
          cudaSuccess)
        goto out;
      if ((e = cudaEventRecord(ev_rest, s)) != cudaSuccess) goto out;
    } else if (j + w < n) {
      if ((e = cudaEventRecord(ev_rest, h)) != cudaSuccess) goto out;   // nothing left of R
    }
    if (j > 0) {
      laswp_range_kernel<T><<<(unsigned)((j + 255) / 256), 256, 0, s>>>(W, n, j, w, piv, 0, j);
      if (launches) ++*launches;
    }
  }
  // the caller's stream continues after the side stream's last work
  if ((e = cudaEventRecord(ev_end, h)) != cudaSuccess) goto out;
  e = cudaStreamWaitEvent(s, ev_end, 0);
out:
  for (int i = 0; i < 4; ++i) cudaEventDestroy(ev[i]);
  if (e == cudaSuccess) e = cudaGetLastError();
  return e;
}

template <typename T>
cudaError_t factor(const SolveArgs& a, const Layout& L, char* base, cudaStream_t s, int* launches) {
  const int64_t n = a.n;
  T* W = reinterpret_cast<T*>(base + L.lu);
  int32_t* piv = reinterpret_cast<int32_t*>(base + L.piv);
  Ctl* ctl = reinterpret_cast<Ctl*>(base + L.ctl);
  const int sms = device_sm_count();
  {
    int64_t blocks = (n * n + 255) / 256, cap = (int64_t)sms * 8;
    copy_kernel<T><<<(unsigned)(blocks < cap ? blocks : cap), 256, 0, s>>>(a.A, a.lda, a.adt, W, n);
    if (launches) ++*launches;
  }
  const int32_t gt = L.f64 ? ARMA_TIER_F64 : a.tier == ARMA_TIER_BF16 ? ARMA_TIER_BF16 : ARMA_TIER_SPLIT_BF16;
  for (int64_t j = 0; j < n; j += NB) {
    const int w = (int)(n - j < NB ? n - j : NB);
    // panel
    PanelArgs<T> pa;
    pa.A = W; pa.ld = n; pa.n = n; pa.j = j; pa.w = w;
    int64_t rows = n - j;
    int ctas = (int)((rows + PT - 1) / PT);
    if (ctas < 1) ctas = 1;
    if (ctas > MAX_CTAS) ctas = MAX_CTAS;
    if (ctas > sms) ctas = sms;
    pa.rows_per_cta = (rows + ctas - 1) / ctas;
    ctas = (int)((rows + pa.rows_per_cta - 1) / pa.rows_per_cta);
    pa.piv = piv;
    pa.cand_val = reinterpret_cast<double*>(base + L.cand_val);
    pa.cand_row = reinterpret_cast<int64_t*>(base + L.cand_row);
    pa.cand_data = reinterpret_cast<T*>(base + L.cand_data);
    pa.drow = reinterpret_cast<T*>(base + L.drow);
    pa.ctl = ctl;
    pa.wait_ns = wait_limit_ns();
    pa.status = a.status_code;
    pa.info = a.status_info;
    cudaError_t e = launch_panel<T>(pa, rows, ctas, s);
    if (e != cudaSuccess) return e;
    if (launches) ++*launches;
    if (n > w) {
      const int64_t others = n - w;
      laswp_kernel<T><<<(unsigned)((others + 255) / 256), 256, 0, s>>>(W, n, n, j, w, piv);
      if (launches) ++*launches;
    }
    const int64_t rest = n - j - w;
    if (rest > 0) {
      trsm_kernel<T><<<(unsigned)((rest + 7) / 8), 256, 0, s>>>(W, n, n, j, w);
      if (launches) ++*launches;
      // FP32 factors: the next panel's columns through next_update_kernel and
      // the rest through the tensor-core product, as the look-ahead
      // factorisation splits them, so both give the same factors bit for bit
      const int dt = L.f64 ? ARMA_F64 : ARMA_F32;
      const int64_t w2 = L.f64 ? 0 : (rest < NB ? rest : NB);
      if constexpr (std::is_same<T, float>::value) {
        if (w2 > 0) {
          next_update_kernel<<<(unsigned)((rest + NU_ROWS - 1) / NU_ROWS), 256, 0, s>>>(W, n, n, j, w, j + w,
                                                                                        (int)w2);
          if (launches) ++*launches;
        }
      }
      const int64_t c0 = j + w + w2, nc = rest - w2;
      if (nc > 0) {
        GemmArgs g;
        memset(&g, 0, sizeof g);
        g.m = rest; g.n = nc; g.k = w;
        g.A = W + (j + w) + j * n; g.lda = n; g.ta = 0; g.adt = dt;
        g.B = W + j + c0 * n; g.ldb = n; g.tb = 0; g.bdt = dt;
        g.C = W + (j + w) + c0 * n; g.ldc = n; g.cdt = dt;
        g.D = W + (j + w) + c0 * n; g.ldd = n; g.ddt = dt;
        g.alpha = -1.0; g.beta = 1.0;
        g.tier = gt;
        g.scratch = base + L.gemm; g.scratch_bytes = L.gemm_bytes;
        g.status = a.status_code;
        g.no_gemv = 1;   // the same product kernel for every block width
        e = launch_gemm(g, s, launches);
        if (e != cudaSuccess) return e;
      }
    }
  }
  return cudaGetLastError();
}

// y := U^-1 L^-1 y for all nrhs columns.  One cooperative launch when all
// (block row, 64-column slice) CTAs fit on the GPU at once; otherwise one
// launch per diagonal block and sweep: the forward sweep reduces Y in place
// and writes the solved rows to Z, the backward sweep reduces Z in place and
// writes the result to Y.  Either way the result is in Y.
// y := U^-1 L^-1 y with LU factors W (ld = n), or with a triangular system
// matrix W (leading dimension lda): sweeps = 1 for lower (non-unit
// diagonal, result in Z), 2 for upper (result in Y), 3 for LU factors
// (unit lower L; result in Y).
// ---------------------------------------------------------------------------
// Cholesky A = L L^T for symmetric positive definite A (the symmetric branch
// of the solve trace, Fig. 3): right-looking, 64-column panels, no pivoting.
// Per panel: the diagonal block is factored in shared memory by one CTA and
// inverted (the substitution's inverse-diagonal-block kernel); the rows below
// become L_21 = A_21 L_jj^-T, a product; the trailing matrix takes
// A_22 -= L_21 L_21^T through the product kernels' lower-triangle schedule
// (sym = 2).  A pivot <= 0 (or NaN) means A is not positive definite: the
// column is recorded in the control block and every later kernel of the
// factorisation returns at once.
// ---------------------------------------------------------------------------
// The diagonal block: S holds the not yet factored part (lower triangle).
// Step c: every thread reads the pivot S[c][c] itself (no extra barrier),
// thread (r, g) = (tid % 64, tid / 64) subtracts l_r l_k from S[r][k] for
// k = c + 1 + g, c + 5 + g, ... <= r, and L's column c goes straight to
// global memory, so S's column c is only read during the step: one barrier
// per column.
template <typename T>
__global__ void __launch_bounds__(256) chol_diag_kernel(T* W, int64_t ld, int64_t j, int w, Ctl* ctl, T* Linv) {
  __shared__ __align__(16) T S[NB][NB + 1];   // S[r][c] = block (r, c), lower part
  __shared__ T dinv[NB];
  if (*(volatile int*)&ctl->chol_fail) return;
  const int tid = threadIdx.x, r = tid & (NB - 1), g = tid >> 6;
  for (int t = tid; t < NB * NB; t += 256) {
    const int rr = t & (NB - 1), cc = t >> 6;
    S[rr][cc] = (rr < w && cc < w && rr >= cc) ? W[(j + rr) + (j + cc) * ld] : (T)0;
  }
  for (int c = 0; c < w; ++c) {
    __syncthreads();
    const T d = S[c][c];
    if (!(d > (T)0)) {                       // uniform: every thread read the same pivot
      if (tid == 0) atomicCAS(&ctl->chol_fail, 0, (int)(j + c + 1));
      return;
    }
    const T sq = sqrt(d), inv = (T)1 / sq;
    if (r > c && r < w) {
      const T lr = S[r][c] * inv;
      for (int k = c + 1 + g; k <= r; k += 4) S[r][k] -= lr * (S[k][c] * inv);
      if (g == 0) W[(j + r) + (j + c) * ld] = lr;
    }
    if (tid == 0) W[(j + c) + (j + c) * ld] = sq;
  }
  // L_jj^-1 for the panel below, from the factor just written (the barrier
  // makes this block's global writes visible to all of its threads)
  if (!Linv) return;
  __syncthreads();
  invert_block(W + j + j * ld, ld, w, &S[0][0], dinv, Linv, (T*)nullptr, true);
}

__global__ void iota_kernel(int32_t* p, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = (int32_t)i;
}

// W := the Cholesky factor of A in its lower triangle (the upper triangle is
// left as scratch; the caller mirrors L into it for the substitution)
template <typename T>
cudaError_t factor_cholesky(const SolveArgs& a, const Layout& L, char* base, cudaStream_t s, int* launches) {
  const int64_t n = a.n;
  T* W = reinterpret_cast<T*>(base + L.lu);
  Ctl* ctl = reinterpret_cast<Ctl*>(base + L.ctl);
  const int sms = device_sm_count();
  {
    int64_t blocks = (n * n + 255) / 256, cap = (int64_t)sms * 8;
    copy_kernel<T><<<(unsigned)(blocks < cap ? blocks : cap), 256, 0, s>>>(a.A, a.lda, a.adt, W, n);
    if (launches) ++*launches;
  }
  const int32_t gt = L.f64 ? ARMA_TIER_F64 : a.tier == ARMA_TIER_BF16 ? ARMA_TIER_BF16 : ARMA_TIER_SPLIT_BF16;
  T* Dinv = reinterpret_cast<T*>(base + L.dinv);   // [2 ceil(n / NB)][NB][NB]; rewritten after the factorisation
  const int dt = L.f64 ? ARMA_F64 : ARMA_F32;
  for (int64_t j = 0; j < n; j += NB) {
    const int w = (int)(n - j < NB ? n - j : NB);
    const int64_t rest = n - j - w;
    // the block's factor and, when rows remain below, its inverse L_jj^-1;
    // then L_21 = A_21 (L_jj^-1)^T in place
    T* Li = Dinv + (j / NB) * NB * NB;
    chol_diag_kernel<T><<<1, 256, 0, s>>>(W, n, j, w, ctl, rest > 0 ? Li : nullptr);
    if (launches) ++*launches;
    if (rest <= 0) continue;
    {
      GemmArgs t;
      memset(&t, 0, sizeof t);
      t.m = rest; t.n = w; t.k = w;
      t.A = W + (j + w) + j * n; t.lda = n; t.ta = 0; t.adt = dt;
      t.B = Li; t.ldb = NB; t.tb = 1; t.bdt = dt;
      t.D = W + (j + w) + j * n; t.ldd = n; t.ddt = dt;
      t.alpha = 1.0;
      t.tier = gt;
      t.scratch = base + L.gemm; t.scratch_bytes = L.gemm_bytes;
      t.status = a.status_code;
      t.skip = &ctl->chol_fail;
      cudaError_t e = launch_gemm(t, s, launches);
      if (e != cudaSuccess) return e;
    }
    GemmArgs g;
    memset(&g, 0, sizeof g);
    g.m = rest; g.n = rest; g.k = w;
    g.A = W + (j + w) + j * n; g.lda = n; g.ta = 0; g.adt = dt;
    g.B = W + (j + w) + j * n; g.ldb = n; g.tb = 1; g.bdt = dt;
    g.C = W + (j + w) + (j + w) * n; g.ldc = n; g.cdt = dt;
    g.D = W + (j + w) + (j + w) * n; g.ldd = n; g.ddt = dt;
    g.alpha = -1.0; g.beta = 1.0;
    g.tier = gt;
    g.sym = 2;                                   // lower triangle only, C kept
    g.scratch = base + L.gemm; g.scratch_bytes = L.gemm_bytes;
    g.status = a.status_code;
    g.skip = &ctl->chol_fail;
    cudaError_t e = launch_gemm(g, s, launches);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t substitute(const T* W, const T* Linv, const T* Uinv, int64_t n, T* Y, T* Z, int64_t nrhs,
                       unsigned int* flags, Ctl* ctl, int32_t* status, const int* skip, cudaStream_t s,
                       int* launches, int64_t lda = 0, int sweeps = 3, int unit_lower = 1) {
  if (lda == 0) lda = n;
  const int64_t nb = (n + NB - 1) / NB;
  const int64_t gy = (nrhs + 63) / 64;
  if (gy > 65535) return cudaErrorInvalidConfiguration;
  {
    const int64_t gc = (nrhs + CW - 1) / CW;
    const size_t smem = coop_smem<T>();
    int per_sm = 0;
    if (gc <= 65535 &&
        cudaFuncSetAttribute(sub_coop_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) ==
            cudaSuccess &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sub_coop_kernel<T>, 256, smem) == cudaSuccess &&
        nb * gc <= (int64_t)per_sm * device_sm_count()) {
      cudaError_t e = cudaMemsetAsync(flags, 0, (size_t)2 * nb * gc * FLAG_STRIDE * sizeof(unsigned int), s);
      if (e != cudaSuccess) return e;
      uint64_t wait_ns = wait_limit_ns();
      void* args[] = {(void*)&W, (void*)&Linv, (void*)&Uinv, (void*)&n, (void*)&Y, (void*)&Z, (void*)&nrhs,
                      (void*)&flags, (void*)&ctl, (void*)&status, (void*)&skip, (void*)&lda, (void*)&sweeps,
                      (void*)&wait_ns};
      e = cudaLaunchCooperativeKernel((const void*)sub_coop_kernel<T>, dim3((unsigned)nb, (unsigned)gc), dim3(256),
                                      args, smem, s);
      if (e == cudaSuccess) {
        if (launches) ++*launches;
        return cudaSuccess;
      }
    }
    cudaGetLastError();
  }
  const size_t smem = sub_smem<T>();
  cudaError_t e = cudaFuncSetAttribute(sub_step_kernel<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(sub_step_kernel<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  auto gx = [](int64_t rows) { return (unsigned)(rows > 0 ? (rows + SUB_ROWS - 1) / SUB_ROWS : 1); };
  // the forward steps read Y and write Z; the backward steps read Z and write Y
  if (sweeps & 1) {
    for (int64_t j = 0; j < n; j += NB) {
      const int w = (int)(n - j < NB ? n - j : NB);
      const int64_t rows = n - j - w;
      sub_step_kernel<T, true><<<dim3(gx(rows), (unsigned)gy), 256, smem, s>>>(W, n, j, w, Y, Z, nrhs, j + w, rows,
                                                                               skip, lda, unit_lower);
      if (launches) ++*launches;
    }
  } else {
    e = cudaMemcpyAsync(Z, Y, (size_t)n * nrhs * sizeof(T), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
  }
  if (sweeps & 2) {
    for (int64_t j = ((n - 1) / NB) * NB; j >= 0; j -= NB) {
      const int w = (int)(n - j < NB ? n - j : NB);
      sub_step_kernel<T, false><<<dim3(gx(j), (unsigned)gy), 256, smem, s>>>(W, n, j, w, Z, Y, nrhs, 0, j, skip,
                                                                             lda, 1);
      if (launches) ++*launches;
    }
  }
  return cudaGetLastError();
}

}  // namespace lu

namespace lu {

template <typename T>
__global__ void rhs_kernel(const void* B, int64_t ldb, int32_t bdt, T* Y, int64_t n, int64_t nrhs) {
  const int64_t total = n * nrhs;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = t / n, i = t - c * n;
    Y[t] = B ? load_as<T>(B, i + c * ldb, bdt) : (T)(i == c ? 1 : 0);
  }
}

// A triangular system solved by substitution with A itself (no
// factorisation): the inverted diagonal blocks of A, then one sweep of the
// cooperative substitution, in the data's own precision.
template <typename T>
cudaError_t solve_triangular(const SolveArgs& a, const Layout& L, char* base, bool lower, Ctl* ctl, cudaStream_t s,
                             int* launches) {
  const int64_t n = a.n, nrhs = a.nrhs, nb = (n + NB - 1) / NB;
  const T* W = static_cast<const T*>(a.A);
  T* Linv = reinterpret_cast<T*>(base + L.tri_dinv);
  T* Uinv = Linv + nb * NB * NB;
  inv_diag_kernel<T><<<(unsigned)nb, 256, 0, s>>>(W, n, Linv, Uinv, a.lda, lower ? 1 : 0);
  T* Y = reinterpret_cast<T*>(base + L.tri_y);
  T* Z = reinterpret_cast<T*>(base + L.tri_z);
  int64_t blocks = (n * nrhs + 255) / 256, cap = (int64_t)device_sm_count() * 8;
  const unsigned g = (unsigned)(blocks < 1 ? 1 : blocks < cap ? blocks : cap);
  rhs_kernel<T><<<g, 256, 0, s>>>(a.B, a.ldb, a.bdt, Y, n, nrhs);
  if (launches) *launches += 2;
  cudaError_t e = substitute<T>(W, Linv, Uinv, n, Y, Z, nrhs, reinterpret_cast<unsigned int*>(base + L.flags), ctl,
                                a.status_code, nullptr, s, launches, a.lda, lower ? 1 : 2, 0);
  if (e != cudaSuccess) return e;
  store_kernel<T><<<g, 256, 0, s>>>(lower ? Z : Y, n, nrhs, a.X, a.ldx, a.xdt);
  if (launches) ++*launches;
  return cudaGetLastError();
}

// The analysis of A (bandwidths, symmetry, zero diagonal) and the choice of
// solver, in the order of the solve trace of Fig. 3: diagonal, band, then
// triangular; anything else is the general LU solve (returns false).  The
// host waits for the analysis: the choice is made on the host, as the
// library's CPU counterpart does.  Under stream capture nothing is analysed.
bool solve_structured(const SolveArgs& a, const Layout& L, char* base, Ctl* ctl, cudaStream_t s, int* launches,
                      cudaError_t* err, bool* try_chol) {
  *err = cudaSuccess;
  *try_chol = false;
  if (!a.analyse || !a.props) return false;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if ((*err = cudaStreamIsCapturing(s, &cs)) != cudaSuccess) return true;
  if (cs != cudaStreamCaptureStatusNone) return false;
  const int64_t n = a.n;
  if ((*err = launch_analyse(a.A, a.lda, a.adt, n, a.props, s, launches)) != cudaSuccess) return true;
  int32_t h[SP_WORDS] = {};
  if ((*err = cudaMemcpyAsync(h, a.props, sizeof h, cudaMemcpyDeviceToHost, s)) != cudaSuccess) return true;
  if ((*err = cudaStreamSynchronize(s)) != cudaSuccess) return true;
  const int32_t kl = h[SP_KL], ku = h[SP_KU], zd = h[SP_ZDIAG];
  const bool typed = a.adt == ARMA_F64 || a.adt == ARMA_F32;
  const bool f64 = a.adt == ARMA_F64;
  int32_t path = ARMA_SOLVE_GENERAL;
  if (typed) {
    if (kl == 0 && ku == 0) path = ARMA_SOLVE_DIAGONAL;
    else if (kl <= kBandMaxKl && ku <= kBandMaxKu && (int64_t)(2 * kl + ku + 1) * 4 <= n) path = ARMA_SOLVE_BAND;
    else if (kl == 0) path = ARMA_SOLVE_UPPER;
    else if (ku == 0) path = ARMA_SOLVE_LOWER;
  }
  // a triangular (or diagonal) matrix is singular exactly when a diagonal element is zero
  const bool tri = path == ARMA_SOLVE_DIAGONAL || path == ARMA_SOLVE_UPPER || path == ARMA_SOLVE_LOWER;
  const int64_t sing = (tri && zd > 0) ? n - zd + 1 : 0;
  if ((*err = launch_set_props(a.props, path, a.status_code, a.status_info, sing, s, launches)) != cudaSuccess)
    return true;
  if (path == ARMA_SOLVE_GENERAL) {
    // symmetric with a positive diagonal: worth a Cholesky attempt (recorded
    // by the caller once the factorisation has shown whether it succeeded)
    *try_chol = typed && h[SP_ASYM] == 0 && h[SP_NONPOS] == 0 && n > 1;
    return false;
  }
  if (sing) return true;
  switch (path) {
    case ARMA_SOLVE_DIAGONAL:
      *err = launch_diag_solve(a, f64, s, launches);
      break;
    case ARMA_SOLVE_BAND: {
      BandArgs b;
      memset(&b, 0, sizeof b);
      b.n = n; b.nrhs = a.nrhs; b.kl = kl; b.ku = ku;
      b.A = a.A; b.lda = a.lda; b.adt = a.adt;
      b.B = a.B; b.ldb = a.ldb; b.bdt = a.bdt;
      b.X = a.X; b.ldx = a.ldx; b.xdt = a.xdt;
      b.work = base + L.band;
      b.status = a.status_code; b.info = a.status_info;
      b.refine = a.tier != ARMA_TIER_F64 ? 1 : 0;
      b.fallback = a.props + SP_FALLBACK;
      *err = launch_band_solve(b, f64, s, launches);
      break;
    }
    default:
      *err = f64 ? solve_triangular<double>(a, L, base, path == ARMA_SOLVE_LOWER, ctl, s, launches)
                 : solve_triangular<float>(a, L, base, path == ARMA_SOLVE_LOWER, ctl, s, launches);
  }
  return true;
}

}  // namespace lu

int64_t solve_scratch_bytes(int64_t n, int64_t nrhs, int32_t tier, int32_t analyse, int32_t dfma_residual) {
  return lu::layout(n, nrhs, tier, analyse, dfma_residual).total;
}

cudaError_t launch_solve(const SolveArgs& a, cudaStream_t s, int* launches) {
  using namespace lu;
  const int64_t n = a.n, nrhs = a.nrhs;
  if (n == 0 || nrhs == 0) return cudaSuccess;
  Layout L = layout(n, nrhs, a.tier, a.analyse, a.dfma_residual);
  if (a.scratch_bytes < L.total) return cudaErrorInvalidValue;
  char* base = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(a.scratch) + 255) & ~uintptr_t(255));
  Ctl* ctl = reinterpret_cast<Ctl*>(base + L.ctl);
  cudaError_t e = cudaMemsetAsync(ctl, 0, sizeof(Ctl), s);
  if (e != cudaSuccess) return e;
  bool chol = false;
  if (solve_structured(a, L, base, ctl, s, launches, &e, &chol)) return e;
  if (e != cudaSuccess) return e;
  const int sms = device_sm_count();
  int32_t* piv = reinterpret_cast<int32_t*>(base + L.piv);
  int32_t* perm = reinterpret_cast<int32_t*>(base + L.perm);
  unsigned int* flags = reinterpret_cast<unsigned int*>(base + L.flags);
  const int64_t nb = (n + NB - 1) / NB;
  auto grid_for = [&](int64_t total) {
    int64_t b = (total + 255) / 256, cap = (int64_t)sms * 8;
    return (unsigned)(b < 1 ? 1 : b < cap ? b : cap);
  };
  // Cholesky first when the analysis allows it; a pivot <= 0 sends the
  // solve to the LU factorisation (the host waits once more to know)
  auto try_cholesky = [&](auto tag) -> cudaError_t {
    using T = decltype(tag);
    cudaError_t ee = factor_cholesky<T>(a, L, base, s, launches);
    if (ee != cudaSuccess) return ee;
    int fail = 0;
    if ((ee = cudaMemcpyAsync(&fail, &ctl->chol_fail, sizeof fail, cudaMemcpyDeviceToHost, s)) != cudaSuccess) return ee;
    if ((ee = cudaStreamSynchronize(s)) != cudaSuccess) return ee;
    chol = fail == 0;
    if ((ee = launch_set_props(a.props, chol ? ARMA_SOLVE_CHOLESKY : ARMA_SOLVE_GENERAL, a.status_code,
                               a.status_info, 0, s, launches)) != cudaSuccess)
      return ee;
    if (!chol) return factor<T>(a, L, base, s, launches);
    // the substitution reads U from the upper triangle: U = L^T, and an
    // identity permutation
    T* W = reinterpret_cast<T*>(base + L.lu);
    if ((ee = launch_mirror_lower(W, n, n, L.f64 ? ARMA_F64 : ARMA_F32, s, launches)) != cudaSuccess) return ee;
    iota_kernel<<<grid_for(n), 256, 0, s>>>(piv, n);
    if (launches) ++*launches;
    return cudaGetLastError();
  };
  if (L.f64) {
    e = chol ? try_cholesky(0.0) : factor<double>(a, L, base, s, launches);
    if (e != cudaSuccess) return e;
    const double* W = reinterpret_cast<const double*>(base + L.lu);
    double* Linv = reinterpret_cast<double*>(base + L.dinv);
    double* Uinv = Linv + nb * NB * NB;
    inv_diag_kernel<double><<<(unsigned)nb, 256, 0, s>>>(W, n, Linv, Uinv, 0, chol ? 1 : 0);
    double* Y = reinterpret_cast<double*>(base + L.y);
    e = launch_perm(piv, perm, n, s);
    if (e != cudaSuccess) return e;
    gather_kernel<double><<<grid_for(n * nrhs), 256, 0, s>>>(a.B, a.ldb, a.bdt, perm, Y, n, nrhs, nullptr);
    e = substitute<double>(W, Linv, Uinv, n, Y, reinterpret_cast<double*>(base + L.z), nrhs, flags, ctl,
                           a.status_code, nullptr, s, launches, 0, 3, chol ? 0 : 1);
    if (e != cudaSuccess) return e;
    store_kernel<double><<<grid_for(n * nrhs), 256, 0, s>>>(Y, n, nrhs, a.X, a.ldx, a.xdt);
    if (launches) *launches += 4;
    return cudaGetLastError();
  }
  bool la = false;
  if (!chol && !a.no_lookahead && lookahead_ok(n)) {
    e = factor_lookahead(a, L, base, s, launches, &la);
    if (e != cudaSuccess) return e;
  }
  if (!la) e = chol ? try_cholesky(0.0f) : factor<float>(a, L, base, s, launches);
  if (e != cudaSuccess) return e;
  const float* W = reinterpret_cast<const float*>(base + L.lu);
  float* Linv = reinterpret_cast<float*>(base + L.dinv);
  float* Uinv = Linv + nb * NB * NB;
  inv_diag_kernel<float><<<(unsigned)nb, 256, 0, s>>>(W, n, Linv, Uinv, 0, chol ? 1 : 0);
  if (launches) ++*launches;
  float* Y = reinterpret_cast<float*>(base + L.y);
  e = launch_perm(piv, perm, n, s);
  if (e != cudaSuccess) return e;
  gather_kernel<float><<<grid_for(n * nrhs), 256, 0, s>>>(a.B, a.ldb, a.bdt, perm, Y, n, nrhs, nullptr);
  float* Z = reinterpret_cast<float*>(base + L.z);
  e = substitute<float>(W, Linv, Uinv, n, Y, Z, nrhs, flags, ctl, a.status_code, nullptr, s, launches, 0, 3,
                        chol ? 0 : 1);
  if (e != cudaSuccess) return e;
  if (launches) *launches += 2;
  if (!L.refine || !a.B) {
    store_kernel<float><<<grid_for(n * nrhs), 256, 0, s>>>(Y, n, nrhs, a.X, a.ldx, a.xdt);
    if (launches) ++*launches;
    return cudaGetLastError();
  }
  // ---- FP64 iterative refinement ----
  double* X64 = reinterpret_cast<double*>(base + L.x64);
  double* R64 = reinterpret_cast<double*>(base + L.r64);
  double* sq = reinterpret_cast<double*>(base + L.sq);
  double* part = reinterpret_cast<double*>(base + L.part);
  store_kernel<float><<<grid_for(n * nrhs), 256, 0, s>>>(Y, n, nrhs, X64, n, ARMA_F64);
  // |A|_F, |B|_F once
  sumsq_any_kernel<<<512, 256, 0, s>>>(a.A, a.adt, a.lda, n, n, part);
  sum_partials_kernel<<<1, 256, 0, s>>>(part, 512, sq, 0);
  sumsq_any_kernel<<<512, 256, 0, s>>>(a.B, a.bdt, a.ldb, n, nrhs, part);
  sum_partials_kernel<<<1, 256, 0, s>>>(part, 512, sq, 1);
  norms_init_kernel<<<1, 32, 0, s>>>(ctl, sq);
  if (launches) *launches += 6;
  const int max_ir = a.max_ir >= 1 && a.max_ir <= MAX_IR_LIMIT ? a.max_ir : MAX_IR;
  const bool resid_sliced = sliced_residual(n, nrhs, a.dfma_residual) && a.adt == ARMA_F64 &&
                            a.A != nullptr;
  for (int it = 1; it <= max_ir; ++it) {
    // r = B - A x (FP64)
    GemmArgs g;
    memset(&g, 0, sizeof g);
    g.m = n; g.n = nrhs; g.k = n;
    g.A = a.A; g.lda = a.lda; g.ta = 0; g.adt = a.adt;
    g.B = X64; g.ldb = n; g.tb = 0; g.bdt = ARMA_F64;
    g.C = a.B; g.ldc = a.ldb; g.cdt = a.bdt;
    g.D = R64; g.ldd = n; g.ddt = ARMA_F64;
    g.alpha = -1.0; g.beta = 1.0;
    // FP64-accurate either way: the sliced product on the tensor cores, with
    // A's slices made by the first step and reused, or DFMA
    g.tier = resid_sliced ? ARMA_TIER_F64_SLICED : ARMA_TIER_F64;
    g.reuse_a = resid_sliced && it > 1 ? 1 : 0;
    g.scratch = base + L.gemm; g.scratch_bytes = L.gemm_bytes;
    g.status = a.status_code;
    g.skip = &ctl->done;
    e = launch_gemm(g, s, launches);
    if (e != cudaSuccess) return e;
    sumsq_any_kernel<<<512, 256, 0, s>>>(R64, ARMA_F64, n, n, nrhs, part);
    sum_partials_kernel<<<1, 256, 0, s>>>(part, 512, sq + 2, 0);
    sumsq_any_kernel<<<512, 256, 0, s>>>(X64, ARMA_F64, n, n, nrhs, part);
    sum_partials_kernel<<<1, 256, 0, s>>>(part, 512, sq + 2, 1);
    ir_check_kernel<<<1, 32, 0, s>>>(ctl, sq + 2, it, a.status_code, a.status_info, it == max_ir);
    // d = (LU)^-1 P r in FP32; x += d
    gather_kernel<float><<<grid_for(n * nrhs), 256, 0, s>>>(R64, n, ARMA_F64, perm, Y, n, nrhs, &ctl->done);
    e = substitute<float>(W, Linv, Uinv, n, Y, Z, nrhs, flags, ctl, a.status_code, &ctl->done, s, launches, 0, 3,
                          chol ? 0 : 1);
    if (e != cudaSuccess) return e;
    ir_update_kernel<<<grid_for(n * nrhs), 256, 0, s>>>(X64, Y, n * nrhs, &ctl->done);
    if (launches) *launches += 7;
  }
  store_kernel<double><<<grid_for(n * nrhs), 256, 0, s>>>(X64, n, nrhs, a.X, a.ldx, a.xdt);
  if (launches) ++*launches;
  return cudaGetLastError();
}

}  // namespace arma
