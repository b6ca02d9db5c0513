// K1: fused elementwise pass with optional sum / sum-of-squares reduction.
//
// The paper's delayed evaluation turns an elementwise expression into one
// loop that reads every operand once and writes the result once, with no
// temporaries (Sec. II, the Z = 0.4*X + 0.6*Y example), vectorised with
// SIMD (Sec. II, last paragraphs; Sec. III (1)).  Here the expression is a
// short program for an accumulator machine (EwIns), interpreted per element
// by every thread; the program is uniform across the grid, so dispatch never
// diverges.  The flat path loads each operand with two 128-bit loads per
// thread and iteration (all operands of a chunk are in flight together),
// runs the program on registers, stores with 128-bit stores and folds
// accu / norm into the same pass.  A strided path serves transposed views,
// row/column broadcasts (diagmat(v)*B), diagonal masks and the diagonal-only
// mode of trace().
#include <cuda_bf16.h>

#include <type_traits>

#include <atomic>
#include <mutex>

#include "common.cuh"

namespace arma {

// Host-side caches in this library are safe for concurrent evaluations from
// several threads: values that every thread would compute alike are atomics
// (a race only repeats the query), lookup tables take a mutex.
int device_sm_count() {
  static std::atomic<int> cached[64];
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  int v = cached[dev].load(std::memory_order_relaxed);
  if (!v) {
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    v = n > 0 ? n : 1;
    cached[dev].store(v, std::memory_order_relaxed);
  }
  return v;
}

namespace {

template <typename CT>
__device__ __forceinline__ CT ew_in(int op, CT acc, CT x, double s) {
  switch (op) {
    case EW_LD: return x;
    case EW_ADD: return acc + x;
    case EW_SUB: return acc - x;
    case EW_RSUB: return x - acc;
    case EW_MUL: return acc * x;
    case EW_DIV: return acc / x;
    case EW_RDIV: return x / acc;
    case EW_AXPY: return fma((CT)s, x, acc);
    case EW_LDP2: return (CT)s * x;   // exact: s is a power of two
    default: return acc;
  }
}

template <typename CT>
__device__ __forceinline__ CT ew_pop(int op, CT st, CT acc) {
  switch (op) {
    case EW_POPADD: return st + acc;
    case EW_POPSUB: return st - acc;
    case EW_POPMUL: return st * acc;
    default: return st / acc;
  }
}

template <typename CT>
__device__ __forceinline__ CT ew_self(int op, CT acc, double s) {
  switch (op) {
    case EW_SCAL: return (CT)s * acc;
    case EW_DIVS: return acc / (CT)s;
    case EW_ADDS: return acc + (CT)s;
    default: return -acc;  // EW_NEG
  }
}

__device__ __forceinline__ bool uses_operand(int op) { return op <= EW_AXPY || op == EW_LDP2; }
__device__ __forceinline__ bool uses_two(int op) { return op == EW_FMA || op == EW_FNMA; }
__device__ __forceinline__ bool is_pop(int op) { return op >= EW_POPADD && op <= EW_POPDIV; }

// ---- strided path: one element per step, any operand layout ----
template <typename CT>
__global__ void __launch_bounds__(256) ew_strided_kernel(const __grid_constant__ EwArgs a) {
  int64_t total = a.mode == EW_DIAG ? (a.m < a.n ? a.m : a.n) : a.m * a.n;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  double rs = 0.0, rq = 0.0;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += stride) {
    int64_t i, j;
    if (a.mode == EW_DIAG) { i = t; j = t; }
    else { j = t / a.m; i = t - j * a.m; }
    CT acc = 0, s0 = 0, s1 = 0, s2 = 0, s3 = 0;
    for (int pc = 0; pc < a.nops; ++pc) {
      const int op = a.ops[pc].op, arg = a.ops[pc].arg;
      const double s = a.ops[pc].s;
      if (uses_operand(op)) {
        CT x;
        if ((a.in_flags[arg] & EWF_DIAGMASK) && i != j) x = 0;
        else x = load_as<CT>(a.in[arg], i * a.rs[arg] + j * a.cs[arg], a.in_dtype[arg]);
        acc = ew_in<CT>(op, acc, x, s);
      } else if (uses_two(op)) {
        const int arg2 = a.ops[pc].arg2;
        CT x, y;
        if ((a.in_flags[arg] & EWF_DIAGMASK) && i != j) x = 0;
        else x = load_as<CT>(a.in[arg], i * a.rs[arg] + j * a.cs[arg], a.in_dtype[arg]);
        if ((a.in_flags[arg2] & EWF_DIAGMASK) && i != j) y = 0;
        else y = load_as<CT>(a.in[arg2], i * a.rs[arg2] + j * a.cs[arg2], a.in_dtype[arg2]);
        acc = op == EW_FMA ? fma(x, y, acc) : fma(-x, y, acc);
      } else if (op == EW_PUSH) {
        if (arg == 0) s0 = acc; else if (arg == 1) s1 = acc; else if (arg == 2) s2 = acc; else s3 = acc;
      } else if (is_pop(op)) {
        CT st = arg == 0 ? s0 : arg == 1 ? s1 : arg == 2 ? s2 : s3;
        acc = ew_pop<CT>(op, st, acc);
      } else {
        acc = ew_self<CT>(op, acc, s);
      }
    }
    if (a.out) store_as<CT>(a.out, i + j * a.out_ld, a.out_dtype, acc);
    if (a.red) {
      double v = (double)acc;
      rs += v;
      rq = fma(v, v, rq);
    }
  }
  if (a.red)
    reduce_finish(rs, rq, a.partials, a.ticket, (a.red & 1) ? a.sum_out : nullptr,
                  (a.red & 2) ? a.norm_out : nullptr, 1.0);
}

// ---- exact float-float accumulation for FP64 reductions ----
// GB300 issues FP64 at a small fraction of its FP32 rate, so the two
// running sums of an FP64 pass (sum, sum of squares) are kept as unevaluated
// float pairs (hi + lo, about 48 significant bits) on the FP32 pipes: Knuth's
// two-sum for additions, an FMA-exact product for squares.  The double is
// split into its pair with integer operations only.  Values outside the
// pair's exponent range take the FP64 route.
__device__ __forceinline__ bool split_ff(double x, float& hi, float& lo) {
  // 32-bit halves only: 64-bit integer operations on the bit pattern issue
  // to the FP64 pipe on this GPU
  const unsigned int uh = (unsigned int)__double2hiint(x), ul = (unsigned int)__double2loint(x);
  const unsigned int e = (uh >> 20) & 0x7ffu;
  if (e == 0u && ((uh << 1) | ul) == 0u) { hi = 0.f; lo = 0.f; return true; }  // +-0
  // |x| in [2^-51, 2^51): hi, lo, hi^2 and its rounding error all stay
  // normal floats, and per-thread sums of squares cannot overflow
  if (e < 972u || e > 1073u) return false;
  const unsigned int sign = uh & 0x80000000u;
  hi = __uint_as_float(sign | ((e - 896u) << 23) | ((uh & 0xFFFFFu) << 3) | (ul >> 29));
  // lo from the low 29 significand bits, assembled as float bits with
  // integer operations (no conversion instruction, which would use the FP64
  // pipe); truncated to 24 bits
  const unsigned int rr = ul & 0x1FFFFFFFu;
  if (rr == 0u) { lo = 0.f; return true; }
  const int nb = 32 - __clz(rr);
  const unsigned int m24 = nb > 24 ? rr >> (nb - 24) : rr << (24 - nb);
  lo = __uint_as_float(sign | ((e - 1075u + (unsigned int)(nb - 1) + 127u) << 23) | (m24 & 0x7FFFFFu));
  return true;
}

__device__ __forceinline__ void ff_add(float& sh, float& sl, float xh, float xl) {
  const float s = __fadd_rn(sh, xh);
  const float bb = __fsub_rn(s, sh);
  float e = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, bb)), __fsub_rn(xh, bb));
  e = __fadd_rn(e, __fadd_rn(sl, xl));
  sh = __fadd_rn(s, e);
  sl = __fsub_rn(e, __fsub_rn(sh, s));
}

struct FFAcc {
  float sh = 0.f, sl = 0.f, qh = 0.f, ql = 0.f;
  double s64 = 0.0, q64 = 0.0;  // values outside the pair's range
  __device__ __forceinline__ void add_pair(float hi, float lo) {
    ff_add(sh, sl, hi, lo);
    const float p = __fmul_rn(hi, hi);
    float pe = __fmaf_rn(hi, hi, -p);
    pe = __fmaf_rn(__fmul_rn(2.f, hi), lo, pe);
    ff_add(qh, ql, p, pe);
  }
  __device__ __forceinline__ void add_f64(double x) {
    s64 += x;
    q64 = fma(x, x, q64);
  }
  // FP32 chunk sums (already float): plain two-sums, no FP64 instruction
  __device__ __forceinline__ void add_f32(float ps, float pq) {
    ff_add(sh, sl, ps, 0.f);
    ff_add(qh, ql, pq, 0.f);
  }
  __device__ __forceinline__ double sum() const { return ((double)sh + (double)sl) + s64; }
  __device__ __forceinline__ double sumsq() const { return ((double)qh + (double)ql) + q64; }
};

// ---- flat path: contiguous operands of one storage type T ----
template <typename T> struct VecTraits;
template <> struct VecTraits<double> { static constexpr int V = 2; typedef double CT; };
template <> struct VecTraits<float> { static constexpr int V = 8; typedef float CT; };
template <> struct VecTraits<__nv_bfloat16> { static constexpr int V = 8; typedef float CT; };

template <typename T, int V, typename CT>
__device__ __forceinline__ void load_chunk(const T* __restrict__ p, int64_t c, CT (&x)[V]) {
  const uint4* q = reinterpret_cast<const uint4*>(p + c * V);
  constexpr int NV = (V * (int)sizeof(T)) / 16;
  uint4 r[NV];
#pragma unroll
  for (int u = 0; u < NV; ++u) r[u] = __ldcs(q + u);   // streamed: read once
  const T* e = reinterpret_cast<const T*>(r);
#pragma unroll
  for (int v = 0; v < V; ++v) {
    if constexpr (std::is_same<T, __nv_bfloat16>::value) x[v] = __bfloat162float(e[v]);
    else x[v] = (CT)e[v];
  }
}

template <typename T, int V, typename CT>
__device__ __forceinline__ void store_chunk(T* __restrict__ p, int64_t c, const CT (&x)[V]) {
  constexpr int NV = (V * (int)sizeof(T)) / 16;
  uint4 r[NV];
  T* e = reinterpret_cast<T*>(r);
#pragma unroll
  for (int v = 0; v < V; ++v) {
    if constexpr (std::is_same<T, __nv_bfloat16>::value) e[v] = __float2bfloat16_rn(x[v]);
    else e[v] = (T)x[v];
  }
  uint4* q = reinterpret_cast<uint4*>(p + c * V);
#pragma unroll
  for (int u = 0; u < NV; ++u) __stcs(q + u, r[u]);
}

// STK: spill slots the program may use (0 when it never pushes), so that
// programs without spills do not hold dead registers.  FP64 passes run 4
// blocks per SM (at most 64 registers): more warps hide more of the memory
// and FP64-pipe latency, measured 0.538 -> 0.504 ms at 8192^2; FP32 passes
// keep 3, where the fourth block cost more than it hid.
template <typename T, int NIN, int STK>
__global__ void __launch_bounds__(256, std::is_same<T, double>::value ? 4 : 3)
    ew_flat_kernel(const __grid_constant__ EwArgs a) {
  constexpr int V = VecTraits<T>::V;
  typedef typename VecTraits<T>::CT CT;
  constexpr bool kFF = std::is_same<T, double>::value;
  const int64_t total = a.m * a.n;
  const int64_t nchunk = total / V;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  double rs = 0.0, rq = 0.0;
  FFAcc ff;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nchunk; c += stride) {
    CT x[NIN][V];
#pragma unroll
    for (int k = 0; k < NIN; ++k) load_chunk<T, V, CT>(static_cast<const T*>(a.in[k]), c, x[k]);
    CT acc[V], st[STK > 0 ? STK : 1][V];
#pragma unroll
    for (int v = 0; v < V; ++v) acc[v] = 0;
    // one uniform branch per instruction; the element loops inside each
    // case are branch-free (no if-conversion of the whole instruction set)
    for (int pc = 0; pc < a.nops; ++pc) {
      const int op = a.ops[pc].op, arg = a.ops[pc].arg;
      CT sc;
      if constexpr (kFF) sc = a.ops[pc].s; else sc = a.ops[pc].sf;
#define ARMA_EW_SEL(BODY)                        \
  _Pragma("unroll") for (int k = 0; k < NIN; ++k) \
    if (k == arg) {                              \
      _Pragma("unroll") for (int v = 0; v < V; ++v) { BODY; } \
    }
#define ARMA_EW_STK(BODY)                        \
  _Pragma("unroll") for (int q = 0; q < STK; ++q) \
    if (q == arg) {                              \
      _Pragma("unroll") for (int v = 0; v < V; ++v) { BODY; } \
    }
      switch (op) {
        case EW_LD: ARMA_EW_SEL(acc[v] = x[k][v]) break;
        case EW_ADD: ARMA_EW_SEL(acc[v] = acc[v] + x[k][v]) break;
        case EW_SUB: ARMA_EW_SEL(acc[v] = acc[v] - x[k][v]) break;
        case EW_RSUB: ARMA_EW_SEL(acc[v] = x[k][v] - acc[v]) break;
        case EW_MUL: ARMA_EW_SEL(acc[v] = acc[v] * x[k][v]) break;
        case EW_DIV: ARMA_EW_SEL(acc[v] = acc[v] / x[k][v]) break;
        case EW_RDIV: ARMA_EW_SEL(acc[v] = x[k][v] / acc[v]) break;
        case EW_AXPY: ARMA_EW_SEL(acc[v] = fma(sc, x[k][v], acc[v])) break;
        case EW_SCAL:
#pragma unroll
          for (int v = 0; v < V; ++v) acc[v] = sc * acc[v];
          break;
        case EW_DIVS:
#pragma unroll
          for (int v = 0; v < V; ++v) acc[v] = acc[v] / sc;
          break;
        case EW_ADDS:
#pragma unroll
          for (int v = 0; v < V; ++v) acc[v] = acc[v] + sc;
          break;
        case EW_NEG:
#pragma unroll
          for (int v = 0; v < V; ++v) acc[v] = -acc[v];
          break;
        case EW_PUSH: ARMA_EW_STK(st[q][v] = acc[v]) break;
        case EW_POPADD: ARMA_EW_STK(acc[v] = st[q][v] + acc[v]) break;
        case EW_POPSUB: ARMA_EW_STK(acc[v] = st[q][v] - acc[v]) break;
        case EW_POPMUL: ARMA_EW_STK(acc[v] = st[q][v] * acc[v]) break;
        case EW_POPDIV: ARMA_EW_STK(acc[v] = st[q][v] / acc[v]) break;
        case EW_FMA:
        case EW_FNMA: {
          const int arg2 = a.ops[pc].arg2;
          CT y[V];
#pragma unroll
          for (int v = 0; v < V; ++v) y[v] = 0;
#pragma unroll
          for (int k = 0; k < NIN; ++k)
            if (k == arg2)
#pragma unroll
              for (int v = 0; v < V; ++v) y[v] = x[k][v];
          if (op == EW_FMA) {
            ARMA_EW_SEL(acc[v] = fma(x[k][v], y[v], acc[v]))
          } else {
            ARMA_EW_SEL(acc[v] = fma(-x[k][v], y[v], acc[v]))
          }
          break;
        }
        case EW_LDP2:
          if constexpr (kFF) {
            // sign and exponent of the bit pattern adjusted with integer
            // operations; zeros, subnormals, infinities and results outside
            // the normal range take an FP64 multiply behind a warp vote
            // (32-bit halves: 64-bit integer operations issue to the FP64 pipe)
            const int e2 = a.ops[pc].arg2;
            // the sign from the bit pattern: an FP64 compare would take the FP64 pipe per chunk
            const unsigned int flip = (unsigned int)__double2hiint((double)sc) & 0x80000000u;
            uint32_t bad = 0u;
            ARMA_EW_SEL({
              const unsigned int uh = (unsigned int)__double2hiint(x[k][v]);
              const unsigned int ul = (unsigned int)__double2loint(x[k][v]);
              const int ex = (int)((uh >> 20) & 0x7ffu);
              const int ne = ex + e2;
              const bool ok = ex != 0 && ex != 0x7ff && ne > 0 && ne < 0x7ff;
              const unsigned int nh = (uh + ((unsigned int)e2 << 20)) ^ flip;
              acc[v] = __hiloint2double((int)(ok ? nh : uh), (int)ul);
              bad |= ok ? 0u : (1u << v);
            })
            if (__any_sync(__activemask(), bad != 0u)) {
#pragma unroll
              for (int v = 0; v < V; ++v)
                if (bad & (1u << v)) acc[v] = sc * acc[v];
            }
          } else {
            ARMA_EW_SEL(acc[v] = sc * x[k][v])
          }
          break;
        default: break;
      }
#undef ARMA_EW_SEL
#undef ARMA_EW_STK
    }
    if (a.out) store_chunk<T, V, CT>(static_cast<T*>(a.out), c, acc);
    if (a.red) {
      if constexpr (kFF) {
        // float-pair accumulation; the FP64 route for out-of-range values
        // runs only when an active lane needs it, so that it is a branch
        // and not FP64 instructions issued for every element
        uint32_t bad = 0u;
#pragma unroll
        for (int v = 0; v < V; ++v) {
          float hi, lo;
          if (split_ff((double)acc[v], hi, lo)) ff.add_pair(hi, lo);
          else bad |= 1u << v;
        }
        if (__any_sync(__activemask(), bad != 0u)) {
          for (int v = 0; v < V; ++v)
            if (bad & (1u << v)) ff.add_f64((double)acc[v]);
        }
      } else {
        float ps = 0.f, pq = 0.f;
#pragma unroll
        for (int v = 0; v < V; ++v) {
          ps += (float)acc[v];
          pq = fmaf((float)acc[v], (float)acc[v], pq);
        }
        ff.add_f32(ps, pq);
      }
    }
    if constexpr (kFF && 4 * NIN <= 32) {
      // this warp's chunks two grid-stride steps ahead into L2, one 128-byte
      // line (8 chunks of 16 bytes) per lane: those reads are in flight while
      // the FP64 pipe works on the next step
      const int lane = threadIdx.x & 31;
      const int64_t nx = c - lane + 2 * stride + (int64_t)(lane & 3) * 8;
      if (lane < 4 * NIN && nx < nchunk)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(static_cast<const T*>(a.in[lane >> 2]) + nx * V));
    }
  }
  rs += ff.sum();
  rq += ff.sumsq();
  // ragged tail: the last total % V elements, one per thread
  for (int64_t t = nchunk * V + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += stride) {
    CT acc = 0, s0 = 0, s1 = 0, s2 = 0, s3 = 0;
    for (int pc = 0; pc < a.nops; ++pc) {
      const int op = a.ops[pc].op, arg = a.ops[pc].arg;
      const double s = a.ops[pc].s;
      if (uses_operand(op)) {
        CT x = load_as<CT>(a.in[arg], t, a.in_dtype[arg]);
        acc = ew_in<CT>(op, acc, x, s);
      } else if (uses_two(op)) {
        const int arg2 = a.ops[pc].arg2;
        const CT x = load_as<CT>(a.in[arg], t, a.in_dtype[arg]);
        const CT y = load_as<CT>(a.in[arg2], t, a.in_dtype[arg2]);
        acc = op == EW_FMA ? fma(x, y, acc) : fma(-x, y, acc);
      } else if (op == EW_PUSH) {
        if (arg == 0) s0 = acc; else if (arg == 1) s1 = acc; else if (arg == 2) s2 = acc; else s3 = acc;
      } else if (is_pop(op)) {
        CT stv = arg == 0 ? s0 : arg == 1 ? s1 : arg == 2 ? s2 : s3;
        acc = ew_pop<CT>(op, stv, acc);
      } else {
        acc = ew_self<CT>(op, acc, s);
      }
    }
    if (a.out) store_as<CT>(a.out, t, a.out_dtype, acc);
    if (a.red) {
      double v = (double)acc;
      rs += v;
      rq = fma(v, v, rq);
    }
  }
  if (a.red)
    reduce_finish(rs, rq, a.partials, a.ticket, (a.red & 1) ? a.sum_out : nullptr,
                  (a.red & 2) ? a.norm_out : nullptr, 1.0);
}

typedef void (*EwKernel)(EwArgs);

// Resident 256-thread blocks per SM for a kernel (cached): the streaming
// passes launch exactly one wave and stride through the data.
int resident_blocks(const void* k) {
  static std::mutex mu;
  static const void* keys[128];
  static int vals[128];
  static int n = 0;
  std::lock_guard<std::mutex> lock(mu);
  for (int i = 0; i < n; ++i)
    if (keys[i] == k) return vals[i];
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, 256, 0) != cudaSuccess || occ < 1) occ = 1;
  if (n < 128) { keys[n] = k; vals[n] = occ; ++n; }
  return occ;
}

template <typename T, int STK>
EwKernel pick_flat(int nin) {
  switch (nin) {
    case 1: return ew_flat_kernel<T, 1, STK>;
    case 2: return ew_flat_kernel<T, 2, STK>;
    case 3: return ew_flat_kernel<T, 3, STK>;
    case 4: return ew_flat_kernel<T, 4, STK>;
    case 5: return ew_flat_kernel<T, 5, STK>;
    case 6: return ew_flat_kernel<T, 6, STK>;
    case 7: return ew_flat_kernel<T, 7, STK>;
    case 8: return ew_flat_kernel<T, 8, STK>;
    default: return nullptr;
  }
}

template <typename T>
EwKernel pick_flat_t(const EwArgs& a) {
  bool stack = false;
  for (int i = 0; i < a.nops; ++i) stack |= a.ops[i].op == EW_PUSH;
  return stack ? pick_flat<T, kMaxStack>(a.nin) : pick_flat<T, 0>(a.nin);
}

bool al16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

}  // namespace

cudaError_t launch_ew(const EwArgs& a, cudaStream_t s, int* launches) {
  const int64_t total = a.mode == EW_DIAG ? (a.m < a.n ? a.m : a.n) : a.m * a.n;
  if (total == 0 && !a.red) return cudaSuccess;
  if (a.nin < 1 || a.nin > kMaxIn) return cudaErrorInvalidValue;
  const int sms = device_sm_count();
  // flat fast path: one storage type, 16-byte aligned, contiguous
  bool flat = a.mode == EW_FLAT;
  int dt = a.in_dtype[0];
  if (flat) {
    for (int k = 0; k < a.nin; ++k) flat &= a.in_dtype[k] == dt && al16(a.in[k]) && a.in_flags[k] == 0;
    if (a.out) flat &= a.out_dtype == dt && al16(a.out);
    flat &= (a.compute_f64 != 0) == (dt == ARMA_F64);
  }
  EwKernel k;
  if (flat) k = dt == ARMA_F64 ? pick_flat_t<double>(a) : dt == ARMA_F32 ? pick_flat_t<float>(a)
                                                                 : pick_flat_t<__nv_bfloat16>(a);
  else k = a.compute_f64 ? ew_strided_kernel<double> : ew_strided_kernel<float>;
  if (!k) return cudaErrorInvalidValue;
  int64_t work = total;
  if (flat) work = total / (dt == ARMA_F64 ? 4 : 8) + 1;
  int64_t need = (work + 255) / 256;
  int64_t cap = (int64_t)sms * resident_blocks(reinterpret_cast<const void*>(k));
  if (cap > kMaxRedBlocks) cap = kMaxRedBlocks;
  int grid = (int)(need < 1 ? 1 : need > cap ? cap : need);
  k<<<grid, 256, 0, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (launches) ++*launches;
  return e;
}

}  // namespace arma
