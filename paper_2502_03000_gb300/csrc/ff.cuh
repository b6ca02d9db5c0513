// Float-pair ("double-float") arithmetic on the FP32 / integer pipes.
//
// GB300 issues FP64 instructions at about one per SM per clock -- too slow
// for an FP64 stream at HBM speed (2.7 GB per 8192^2 elementwise pass needs
// ~170 G elements/s).  A value x is carried as an unevaluated pair of floats
// hi + lo with |lo| <= ulp(hi)/2 (about 48 significand bits).  Conversions
// between double and pair use integer operations only, additions use
// Knuth's two-sum, products an FMA-exact product (Dekker / Knuth; Hida, Li
// and Bailey's double-double library uses the same error-free transforms).
// Relative error per operation is ~2^-45, far inside the 1e-12 FP64
// tolerance; callers check ranges and fall back to native FP64 where a pair
// would leave float's exponent range.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace arma {
namespace ff {

struct F2 {
  float h, l;
};

// Values handled as pairs: zero, or magnitudes in [2^-40, 2^40].  Then any
// product of two such values lies in [2^-80, 2^80], whose low parts are
// still normal floats, so every operation below is exact up to its stated
// rounding.  Anything else takes the native FP64 route.
constexpr float kLo = 0x1p-40f, kHi = 0x1p40f;

// split x exactly into hi (leading 24 bits) and lo (next 24 bits,
// rounded); returns false outside [2^-40, 2^40) (zero is accepted)
__device__ __forceinline__ bool split(double x, F2& r) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const unsigned int e = (unsigned int)(u >> 52) & 0x7ffu;
  if (e == 0u && (u << 1) == 0ull) { r.h = 0.f; r.l = 0.f; return true; }
  if (e < 983u || e > 1062u) return false;
  const unsigned int sign = (unsigned int)(u >> 32) & 0x80000000u;
  const unsigned long long mant = u & 0xFFFFFFFFFFFFFull;
  r.h = __uint_as_float(sign | ((e - 896u) << 23) | (unsigned int)(mant >> 29));
  // lo: the low 29 significand bits, value rr * 2^(e-1075), built as float
  // bits with integer operations (truncated to 24 bits)
  const unsigned int rr = (unsigned int)(mant & 0x1FFFFFFFull);
  if (rr == 0u) { r.l = 0.f; return true; }
  const int nb = 32 - __clz(rr);                       // significant bits, 1..29
  const unsigned int m24 = nb > 24 ? rr >> (nb - 24) : rr << (24 - nb);
  const unsigned int el = e - 1075u + (unsigned int)(nb - 1) + 127u;   // >= 983-1075+127 > 0
  r.l = __uint_as_float(sign | (el << 23) | (m24 & 0x7FFFFFu));
  return true;
}

// double -> float, round to nearest even, integer operations only.  Returns
// false (and r unspecified) unless the result is a normal float or zero.
// Works on the two 32-bit halves: 64-bit integer operations issue to the
// FP64 pipe on this GPU.
__device__ __forceinline__ bool d2f_rn(double x, float& r) {
  const unsigned int uh = (unsigned int)__double2hiint(x), ul = (unsigned int)__double2loint(x);
  const unsigned int e = (uh >> 20) & 0x7ffu;
  const unsigned int sign = uh & 0x80000000u;
  if (e == 0u && ((uh << 1) | ul) == 0u) { r = __uint_as_float(sign); return true; }
  if (e < 897u || e > 1150u) return false;              // float exponent 1..254
  unsigned int m = ((uh & 0xFFFFFu) << 3) | (ul >> 29);  // 23 fraction bits
  const unsigned int rem = ul & 0x1FFFFFFFu;
  unsigned int be = e - 896u;
  if (rem > 0x10000000u || (rem == 0x10000000u && (m & 1u))) {
    if (++m == 0x800000u) { m = 0u; ++be; }
  }
  if (be >= 255u) return false;
  r = __uint_as_float(sign | (be << 23) | m);
  return true;
}

// exact float -> double (normal floats and zero), from 32-bit halves
__device__ __forceinline__ double f2d_exact(float f) {
  const unsigned int u = __float_as_uint(f);
  const unsigned int e = (u >> 23) & 0xffu;
  if (e == 0u) return __hiloint2double((int)(u & 0x80000000u), 0);   // zero (denormals flushed)
  const unsigned int hi = (u & 0x80000000u) | ((e + 896u) << 20) | ((u & 0x7fffffu) >> 3);
  return __hiloint2double((int)hi, (int)(u << 29));
}

// the same as a 64-bit pattern
__device__ __forceinline__ unsigned long long f2d_bits(float f) {
  return (unsigned long long)__double_as_longlong(f2d_exact(f));
}

// hi + lo as a double, by integer operations (no FP64 instruction).  Needs a
// normalised pair (|lo| <= ulp(hi)/2, hi normal or zero).
__device__ __forceinline__ double to_double(F2 a) {
  const unsigned int uh = __float_as_uint(a.h), ul = __float_as_uint(a.l);
  const unsigned int eh = (uh >> 23) & 0xffu, el = (ul >> 23) & 0xffu;
  if (eh == 0u) return __longlong_as_double((long long)f2d_bits(a.l));
  if (el == 0u) return __longlong_as_double((long long)f2d_bits(a.h));
  unsigned long long M = ((unsigned long long)((uh & 0x7fffffu) | 0x800000u)) << 29;  // 53-bit frame
  int E = (int)eh;                                                                   // float-biased
  const int shift = (int)eh - (int)el;                                               // >= 24
  const unsigned long long ml = ((unsigned long long)((ul & 0x7fffffu) | 0x800000u));
  unsigned long long L;
  if (shift <= 29) L = ml << (29 - shift);
  else if (shift < 29 + 24) L = ml >> (shift - 29);
  else L = 0ull;
  if ((uh ^ ul) & 0x80000000u) {
    M -= L;
    if (M < (1ull << 52)) { M <<= 1; E -= 1; }
  } else {
    M += L;
    if (M >= (1ull << 53)) { M >>= 1; E += 1; }
  }
  const unsigned long long bits = ((unsigned long long)(uh & 0x80000000u) << 32) |
                                  ((unsigned long long)(E + 896) << 52) | (M & 0xFFFFFFFFFFFFFull);
  return __longlong_as_double((long long)bits);
}

__device__ __forceinline__ F2 from_float(float f) { return F2{f, 0.f}; }

// hi + lo, renormalised (fast two-sum; |s| >= |e| holds here)
__device__ __forceinline__ F2 renorm(float s, float e) {
  const float h = __fadd_rn(s, e);
  return F2{h, __fsub_rn(e, __fsub_rn(h, s))};
}

__device__ __forceinline__ F2 add(F2 a, F2 b) {
  const float s = __fadd_rn(a.h, b.h);
  const float bb = __fsub_rn(s, a.h);
  float e = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bb)), __fsub_rn(b.h, bb));
  e = __fadd_rn(e, __fadd_rn(a.l, b.l));
  return renorm(s, e);
}

__device__ __forceinline__ F2 neg(F2 a) { return F2{-a.h, -a.l}; }
__device__ __forceinline__ F2 sub(F2 a, F2 b) { return add(a, neg(b)); }

__device__ __forceinline__ F2 mul(F2 a, F2 b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  return renorm(p, e);
}

__device__ __forceinline__ F2 div(F2 a, F2 b) {
  const float q1 = __fdiv_rn(a.h, b.h);
  const F2 r = sub(a, mul(F2{q1, 0.f}, b));
  const float q2 = __fdiv_rn(r.h, b.h);
  return renorm(q1, q2);
}

// a + s * x with s a pair constant
__device__ __forceinline__ F2 axpy(F2 s, F2 x, F2 a) { return add(a, mul(s, x)); }

// magnitude guard for intermediate results (see kLo, kHi); false for
// inf / NaN too
__device__ __forceinline__ bool in_range(F2 a) {
  const float m = fabsf(a.h);
  return (m <= kHi && m >= kLo) || m == 0.f;
}

}  // namespace ff
}  // namespace arma
