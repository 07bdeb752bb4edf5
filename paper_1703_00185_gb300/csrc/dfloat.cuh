// Double-float ("df") arithmetic on the FP32 pipes: a value is the unevaluated
// sum hi + lo of two floats with |lo| <= ulp(hi)/2, about 48 significant bits.
//
// GB300 runs FP32 at 64x its FP64 rate, so where a kernel needs more than
// FP32 precision but not the full FP64 exponent range, df keeps the work on
// the FP32 pipes.  Algorithms: Knuth's two-sum, Dekker's fast two-sum and the
// fma-based exact product, composed as in Hida, Li & Bailey's QD library
// ("accurate" addition).  Every operation uses the _rn intrinsics so the
// compiler cannot contract or reassociate them.
#pragma once

#include <cstdint>

namespace d2q37 {

struct dfloat {
  float hi, lo;
};

__device__ __forceinline__ dfloat df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}

__device__ __forceinline__ dfloat df_fast_two_sum(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ dfloat df_two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ dfloat df(float a) { return {a, 0.0f}; }

__device__ __forceinline__ dfloat df_neg(dfloat x) { return {-x.hi, -x.lo}; }

__device__ __forceinline__ dfloat df_add(dfloat x, dfloat y) {
  dfloat s = df_two_sum(x.hi, y.hi);
  const dfloat t = df_two_sum(x.lo, y.lo);
  s.lo = __fadd_rn(s.lo, t.hi);
  s = df_fast_two_sum(s.hi, s.lo);
  s.lo = __fadd_rn(s.lo, t.lo);
  return df_fast_two_sum(s.hi, s.lo);
}

// "Sloppy" addition (one two-sum instead of two): relative error about
// 2^-44 even when the low parts cancel, 11 FP32 operations instead of 20.
__device__ __forceinline__ dfloat df_add_fast(dfloat x, dfloat y) {
  dfloat s = df_two_sum(x.hi, y.hi);
  s.lo = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
  return df_fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ dfloat df_add(dfloat x, float y) {
  dfloat s = df_two_sum(x.hi, y);
  s.lo = __fadd_rn(s.lo, x.lo);
  return df_fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ dfloat df_mul(dfloat x, dfloat y) {
  dfloat p = df_two_prod(x.hi, y.hi);
  p.lo = __fmaf_rn(x.hi, y.lo, __fmaf_rn(x.lo, y.hi, p.lo));
  return df_fast_two_sum(p.hi, p.lo);
}

__device__ __forceinline__ dfloat df_mul(dfloat x, float y) {
  dfloat p = df_two_prod(x.hi, y);
  p.lo = __fmaf_rn(x.lo, y, p.lo);
  return df_fast_two_sum(p.hi, p.lo);
}

// K0 + x (K1 + x K2) (Horner) with sloppy additions.
__device__ __forceinline__ dfloat df_quad(dfloat K0, dfloat K1, dfloat K2, dfloat x) {
  const dfloat t = df_add_fast(K1, df_mul(x, K2));
  return df_add_fast(K0, df_mul(x, t));
}

// 1 / y for y > 0, about 2^-45 relative, in 8 FP32 operations: r = 1 / y_hi
// rounded, e = 1 - y r by two FMAs (the first is exact to ~2^-48 because
// y_hi r = 1 - O(2^-24)), 1 / y = r / (1 - e) ~ r + r e up to r e^2 ~ 2^-46.
__device__ __forceinline__ dfloat df_rcp_fast(dfloat y) {
  const float r = __frcp_rn(y.hi);
  float e = __fmaf_rn(-y.hi, r, 1.0f);
  e = __fmaf_rn(-y.lo, r, e);
  return df_fast_two_sum(r, __fmul_rn(r, e));
}

__device__ __forceinline__ float df_to_float(dfloat x) { return __fadd_rn(x.hi, x.lo); }

// An integer below 2^23 as a float, exactly, without a conversion instruction
// (conversions share the slow FP64 pipe on GB300): 2^23 + v has v as its
// mantissa bits.
__device__ __forceinline__ float df_small_uint(unsigned v) {
  return __fsub_rn(__int_as_float(0x4B000000 | v), 8388608.0f);
}

// v 2^scale_exp rounded to a float within one ulp (|v| < 2^53): the top bits
// through a 32-bit conversion, the low 23 exactly, one FMA to join them.
__device__ __forceinline__ float float_from_int64(long long v, int scale_exp) {
  const float hi = __int2float_rn((int)(v >> 23));       // |v >> 23| < 2^30
  const float lo = df_small_uint((unsigned)(v & 0x7FFFFF));  // exact, v - (v >> 23) 2^23 >= 0
  const float s = __int_as_float((scale_exp + 127) << 23);
  return __fmul_rn(__fmaf_rn(hi, 8388608.0f, lo), s);
}

// Exact-ish conversion of a 64-bit integer scaled by 2^scale_exp: the value
// is split into 23-bit pieces (each exact in FP32) and summed in df.
__device__ __forceinline__ dfloat df_from_int64(long long v, int scale_exp) {
  const bool neg = v < 0;
  const unsigned long long m = neg ? (unsigned long long)(-v) : (unsigned long long)v;
  const float a = df_small_uint((unsigned)(m >> 46));              // bits 46..63 (< 2^18)
  const float b = df_small_uint((unsigned)((m >> 23) & 0x7FFFFF)); // bits 23..45
  const float c = df_small_uint((unsigned)(m & 0x7FFFFF));         // bits 0..22
  dfloat r = df_two_sum(__fmul_rn(a, 70368744177664.0f), __fmul_rn(b, 8388608.0f));  // 2^46, 2^23
  r = df_add(r, c);
  const float s = __int_as_float((scale_exp + 127) << 23);  // 2^scale_exp, scale_exp in [-126, 127]
  r.hi = __fmul_rn(r.hi, s);
  r.lo = __fmul_rn(r.lo, s);
  return neg ? df_neg(r) : r;
}

}  // namespace d2q37
