// Float-float helpers for the FP64 offload mode: splitting a double into two floats with
// integer operations (no FP64 instruction), an exact-product multiply-accumulate, and the
// exact float -> double widening, also by integer operations.
#pragma once

#include "kc_internal.cuh"

namespace kc {

// x ~ hi + lo (to 2^-46 relative) using integer operations only; returns false when x is
// outside the range where the split is exact enough (then use FP64 for this element).
__device__ __forceinline__ bool split_df(double x, float& hi, float& lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned int H = (unsigned int)(b >> 32), L = (unsigned int)b;
  const unsigned int e = (H >> 20) & 0x7ffu;
  const unsigned int sgn = H & 0x80000000u;
  const unsigned int hb = sgn | ((e - 896u) << 23) | ((H & 0xfffffu) << 3) | (L >> 29);
  const float rf = __uint_as_float(0x4b000000u | ((L >> 6) & 0x7fffffu)) - 8388608.0f;
  const float sc = __uint_as_float((e - 942u) << 23);
  const bool zero = e == 0u;
  hi = zero ? 0.0f : __uint_as_float(hb);
  lo = zero ? 0.0f : __uint_as_float(__float_as_uint(rf * sc) | sgn);
  return zero || (e - 943u) <= (1120u - 943u);
}

// The split of split_df for an operand that passed split_fast_ok (non-zero, magnitude in
// [2^-80, 2^98)): no zero or range handling, the high float by one funnel shift.
__device__ __forceinline__ void split_fast(double x, float& hi, float& lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned int H = (unsigned int)(b >> 32), L = (unsigned int)b;
  const unsigned int sgn = H & 0x80000000u;
  // exponent e - 896 (1..255 in range) and the top 23 significand bits, truncated
  hi = __uint_as_float(__funnelshift_l(L, H - (896u << 20), 3) | sgn);
  // the next 23 significand bits as an integer, times 2^(e - 1069) (in range: a normal float)
  const float rf = __uint_as_float(0x4b000000u | ((L >> 6) & 0x7fffffu)) - 8388608.0f;
  const float sc = __uint_as_float(((H & 0x7ff00000u) << 3) - (942u << 23));
  lo = __uint_as_float(__float_as_uint(rf * sc) | sgn);
}

// true for the operands split_fast takes: non-zero with a magnitude in [2^-80, 2^98)
__device__ __forceinline__ bool split_fast_ok(double x) {
  const unsigned int H = (unsigned int)((unsigned long long)__double_as_longlong(x) >> 32);
  return ((H & 0x7ff00000u) - (943u << 20)) <= (177u << 20);
}

// the range test of split_df alone: zero, or a magnitude in [2^-80, 2^98)
__device__ __forceinline__ bool df_in_range(double x) {
  const unsigned int e = ((unsigned int)((unsigned long long)__double_as_longlong(x) >> 52)) & 0x7ffu;
  return e == 0u || (e - 943u) <= (1120u - 943u);
}

// (sh, sl) += (ah + al)(bh + bl), float-float with an exact leading product
__device__ __forceinline__ void df_mac(float& sh, float& sl, float ah, float al, float bh,
                                       float bl) {
  const float p = ah * bh;
  const float pe = fmaf(ah, bh, -p);
  const float c = fmaf(ah, bl, fmaf(al, bh, pe));
  const float t = sh + p;
  const float bp = t - sh;
  const float err = (sh - (t - bp)) + (p - bp);
  sh = t;
  sl += err + c;
}

// double from a float, by integer operations (exact for normal floats and zero)
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned int u = __float_as_uint(f);
  const unsigned int e = (u >> 23) & 0xffu;
  if (e == 0u) return 0.0;
  const unsigned long long d = ((unsigned long long)(u & 0x80000000u) << 32) |
                               ((unsigned long long)(e + 896u) << 52) |
                               ((unsigned long long)(u & 0x7fffffu) << 29);
  return __longlong_as_double((long long)d);
}

// FP32 value of a double by truncation to 24 significant bits, by integer operations (no
// FP64 instruction): 0 below the FP32 normal range, NaN from 2^128 (and for Inf / NaN).
__device__ __forceinline__ float d2f_trunc(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned int H = (unsigned int)(b >> 32), L = (unsigned int)b;
  const unsigned int ef = H & 0x7ff00000u;
  const unsigned int f = __funnelshift_l(L, H - (896u << 20), 3) | (H & 0x80000000u);
  return ef < (897u << 20) ? 0.0f
                           : (ef < (1151u << 20) ? __uint_as_float(f) : __int_as_float(0x7fc00000));
}

}  // namespace kc
