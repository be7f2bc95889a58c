// Double-float ("df64") arithmetic: a value is an unevaluated sum hi + lo of two
// FP32 numbers with |lo| <= ulp(hi)/2, about 48 significant bits.  GB300 runs
// FP32 at ~58x its FP64 rate, so an FP64-class stencil in df64 costs far less
// issue time than native FP64.
//
// The algorithms are the error-free transformations of Dekker (1971, "A
// floating-point technique for extending the available precision") and Knuth
// (TAOCP vol. 2, TwoSum), in the "accurate" addition and FMA-based product
// forms of Hida, Li and Bailey's double-double library (2001), transposed to
// FP32 pairs.  Conversions to and from FP64 use integer operations on the
// IEEE-754 bit layouts, so they issue no FP64 instructions on the fast path.
#pragma once

#include <cuda_runtime.h>

namespace mfg {

struct df {
  float hi, lo;
};

__device__ __forceinline__ df quick_two_sum(float a, float b) {  // requires |a| >= |b|
  const float s = a + b;
  return df{s, b - (s - a)};
}

__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = a + b;
  const float v = s - a;
  return df{s, (a - (s - v)) + (b - v)};
}

// a + b with relative error ~2^-48 even under cancellation.
__device__ __forceinline__ df df_add(df a, df b) {
  df s = two_sum(a.hi, b.hi);
  const df t = two_sum(a.lo, b.lo);
  s.lo += t.hi;
  s = quick_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return quick_two_sum(s.hi, s.lo);
}

// a + b for operands of the same sign (no cancellation): the cheaper
// "sloppy" addition, relative error ~2^-47.
__device__ __forceinline__ df df_add_same(df a, df b) {
  const df s = two_sum(a.hi, b.hi);
  return quick_two_sum(s.hi, s.lo + (a.lo + b.lo));
}

// a + b with b a single FP32 number.
__device__ __forceinline__ df df_add_f(df a, float b) {
  const df s = two_sum(a.hi, b);
  return quick_two_sum(s.hi, s.lo + a.lo);
}

__device__ __forceinline__ df df_neg(df a) { return df{-a.hi, -a.lo}; }

// a < b, a <= b on the represented values (|lo| <= ulp(hi)/2 makes the pairs
// ordered by hi first).
__device__ __forceinline__ bool df_lt(df a, df b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ bool df_le(df a, df b) { return a.hi < b.hi || (a.hi == b.hi && a.lo <= b.lo); }
__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

// a * b: the exact product of the high parts by FMA, plus the cross terms.
__device__ __forceinline__ df df_mul(df a, df b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return quick_two_sum(p, e);
}

// 2^k as an FP32 number, for -126 <= k <= 127 (built from its bit pattern).
__device__ __forceinline__ float pow2f(int k) { return __uint_as_float((unsigned)(k + 127) << 23); }

// FP64 -> df64.  Fast path (2^-74 <= |x| < 2^128): hi takes the sign, the
// exponent and the top 23 explicit mantissa bits; lo is the remaining 29 bits,
// converted as an integer and scaled by a power of two; a final quick_two_sum
// restores |lo| <= ulp(hi)/2.  Zero and subnormals give 0; other magnitudes
// take the FP64 conversion path.
__device__ __forceinline__ df df_from_double(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7FF);
  if (e == 0) return df{0.0f, 0.0f};
  if (e < 949 || e > 1150) {
    const float h = __double2float_rn(x);
    return df{h, __double2float_rn(x - (double)h)};
  }
  const unsigned int sign = (unsigned int)(b >> 32) & 0x80000000u;
  const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  const float hi = __uint_as_float(sign | ((unsigned)(e - 896) << 23) | (unsigned)(m >> 29));
  float lo = (float)(unsigned)(m & 0x1FFFFFFFull) * pow2f(e - 1075);
  if (sign) lo = -lo;
  return quick_two_sum(hi, lo);
}

// FP32 -> FP64 by bits (normal numbers exactly; zero and subnormals give 0).
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned int u = __float_as_uint(f);
  const unsigned int ex = (u >> 23) & 0xFF;
  if (ex == 0) return 0.0;
  if (ex == 255) return (double)f;  // keep Inf and NaN visible
  const unsigned long long s = (unsigned long long)(u & 0x80000000u) << 32;
  const unsigned long long d = s | ((unsigned long long)(ex + 896) << 52) |
                               ((unsigned long long)(u & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)d);
}

// df64 -> FP64: one FP64 addition.
__device__ __forceinline__ double df_to_double(df a) { return f2d_bits(a.hi) + f2d_bits(a.lo); }

}  // namespace mfg
