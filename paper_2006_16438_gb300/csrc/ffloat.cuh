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

// (hi, lo) += (ah + al) (bh + bl), the product's al*bl term dropped (below 2^-46): the
// rounding error of ah*bh (exact by the FMA) and the cross terms folded into it by two
// more FMAs, TwoSum of the running high part, twelve FP32 instructions in all.
__device__ __forceinline__ void ff_fma(float ah, float al, float bh, float bl, float& hi, float& lo) {
  const float p = __fmul_rn(ah, bh);
  const float low = __fmaf_rn(ah, bl, __fmaf_rn(al, bh, __fmaf_rn(ah, bh, -p)));
  float s, t;
  two_sum(hi, p, s, t);
  hi = s;
  lo = __fadd_rn(lo, __fadd_rn(t, low));
}

// The FP64 value of a float by integer operations only (exact; the FP32-to-FP64
// conversion issues on the FP64 pipe, and a rarely taken branch to it is still issued,
// predicated off, on every call): sign, exponent rebiased by 1023 - 127, significand
// moved up by 29 bits; infinities and NaNs keep an all-ones exponent, and a subnormal
// m 2^-149 is normalised by its leading one.
__device__ __forceinline__ double f2d_exact(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned sign = u & 0x80000000u, mag = u & 0x7fffffffu;
  const unsigned e = mag >> 23;
  unsigned hi = sign | ((mag >> 3) + (896u << 20)), lo = u << 29;
  if (e == 255u) hi = sign | 0x7ff00000u | ((mag & 0x7fffffu) >> 3);
  if (e == 0u) {
    const int k = mag ? 31 - __clz(mag) : 0;  // leading one of the subnormal's significand
    const unsigned long long m = ((unsigned long long)mag << (52 - k)) & ((1ull << 52) - 1);
    hi = mag ? sign | ((unsigned)(k + 874) << 20) | (unsigned)(m >> 32) : sign;
    lo = mag ? (unsigned)m : 0u;
  }
  return __hiloint2double((int)hi, (int)lo);
}

// Splits an FP64 value into floats hi + lo without the FP64 pipe (a conversion or an
// FP64 subtraction issues there, and a rarely taken branch to one is still issued,
// predicated off, for every element): hi's bits are the sign, the rebiased exponent
// and the top 23 stored mantissa bits of v; lo is the remaining 29 mantissa bits as an
// integer, rounded to a float by the integer-to-float conversion (2^-48 relative to v)
// and scaled by 2^(E - 1075) with an integer add to its exponent field.  Outside FP32's
// normal range the pair saturates: |v| < 2^-126 gives (0, 0), a lo below 2^-126 gives
// lo = 0 (so the 2^-48 holds for |v| >= 2^-97), |v| >= 2^128 gives (+-inf, 0) and a NaN
// (NaN, 0).
__device__ __forceinline__ float2 split_ff(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const unsigned hi32 = (unsigned)(b >> 32);
  const unsigned sign = hi32 & 0x80000000u;
  const int E = (int)((hi32 >> 20) & 0x7ffu);
  const int fe = E - 896;  // FP32 exponent field of hi
  unsigned hb = sign | ((unsigned)fe << 23) | ((unsigned)(b >> 29) & 0x7fffffu);
  const unsigned low = (unsigned)b & 0x1fffffffu;  // v - hi = low * 2^(E - 1075)
  const unsigned lf = __float_as_uint(__uint2float_rn(low));
  const int le = (int)(lf >> 23) + E - 1075;       // FP32 exponent field of lo
  unsigned lb = low && le >= 1 ? sign | (lf + ((unsigned)(E - 1075) << 23)) : 0u;
  if (fe < 1) {
    hb = sign;
    lb = 0u;
  } else if (fe > 254) {
    hb = sign | (E == 2047 && (b << 12) ? 0x7fc00000u : 0x7f800000u);
    lb = 0u;
  }
  return make_float2(__uint_as_float(hb), __uint_as_float(lb));
}

}  // namespace cpa
