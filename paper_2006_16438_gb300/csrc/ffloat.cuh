// Float-pair ("double-float") arithmetic on the FP32 pipe: a value is hi + lo with
// |lo| <= ulp(hi) / 2.  GB300's FP64 pipe issues at 1/64 of the FP32 rate, so kernels
// whose FP64 products and sums dominate use these instead (about 2^-44 relative per
// operation chain, against 2^-53 for FP64).  TwoSum (Knuth) gives the exact error of
// a float addition; fma(a, b, -ab) that of a product.  The _rn intrinsics keep the
// compiler from contracting the error-free steps.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace cpa {

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float z = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}

// (hi, lo) += (ah + al) (bh + bl), the product's al*bl term dropped (below 2^-46).
__device__ __forceinline__ void ff_fma(float ah, float al, float bh, float bl, float& hi, float& lo) {
  const float p = __fmul_rn(ah, bh);
  const float e = __fmaf_rn(ah, bh, -p);
  const float cross = __fmaf_rn(ah, bl, __fmul_rn(al, bh));
  float s, t;
  two_sum(hi, p, s, t);
  hi = s;
  lo = __fadd_rn(lo, __fadd_rn(t, __fadd_rn(e, cross)));
}

// (ah + al)(bh + bl) as a normalised pair (al*bl dropped).
__device__ __forceinline__ float2 ff_mul(float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  const float e = __fmaf_rn(a.x, b.y, __fmaf_rn(a.y, b.x, __fmaf_rn(a.x, b.x, -p)));
  const float s = __fadd_rn(p, e);
  return make_float2(s, __fsub_rn(e, __fsub_rn(s, p)));
}

// (ah + al) + (bh + bl) as a normalised pair.
__device__ __forceinline__ float2 ff_add(float2 a, float2 b) {
  float s, e;
  two_sum(a.x, b.x, s, e);
  e = __fadd_rn(e, __fadd_rn(a.y, b.y));
  const float h = __fadd_rn(s, e);
  return make_float2(h, __fsub_rn(e, __fsub_rn(h, s)));
}

// Splits an FP64 value into floats hi + lo with integer operations only (a conversion
// or an FP64 subtraction would issue on the FP64 pipe): hi's bits are the sign, the
// rebiased exponent and the top 23 stored mantissa bits of v; lo is the remaining 29
// mantissa bits, scaled by 2^(E - 1075) and normalised to a float by their leading one
// (its lowest bits dropped when there are more than 24: 2^-47 relative to v).  Values
// whose hi or lo falls outside FP32's normal range (zero, magnitudes below about 2^-97
// or from 2^128) take the conversions.
__device__ __forceinline__ float2 split_ff(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const unsigned hi32 = (unsigned)(b >> 32);
  const unsigned sign = hi32 & 0x80000000u;
  const int E = (int)((hi32 >> 20) & 0x7ffu);
  const int fe = E - 896;  // FP32 exponent field of hi
  const unsigned low = (unsigned)b & 0x1fffffffu;  // v - hi = low * 2^(E - 1075)
  const int top = low ? 31 - __clz(low) : 0;       // position of lo's leading one (0..28)
  const int le = E - 1075 + top + 127;             // FP32 exponent field of lo
  if (fe >= 1 && fe <= 254 && (!low || le >= 1)) {
    const float h = __uint_as_float(sign | ((unsigned)fe << 23) | ((unsigned)(b >> 29) & 0x7fffffu));
    float l = 0.f;
    if (low) {
      const unsigned m = top >= 23 ? (low >> (top - 23)) : (low << (23 - top));
      l = __uint_as_float(sign | ((unsigned)le << 23) | (m & 0x7fffffu));
    }
    return make_float2(h, l);
  }
  const double vh = __longlong_as_double((long long)(b & ~((1ull << 29) - 1)));
  return make_float2((float)vh, (float)(v - vh));
}

}  // namespace cpa
