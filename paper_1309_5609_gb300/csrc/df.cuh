// Double-float arithmetic: a value is the unevaluated sum hi + lo of two float32
// numbers with |lo| <= ulp(hi) / 2, about 48 significant bits.  Built from the
// error-free transformations of Knuth (TwoSum), Dekker (Fast2Sum) and the FMA
// form of the exact product; the layout follows the double-double scheme of
// Hida, Li & Bailey.  It lets the float32 pipes do the compensated per-sample
// sums of the accurate passes, which on GB300 run far faster than float64.
//
// Every operation uses the explicitly rounded intrinsics so that the compiler
// can neither contract nor reassociate them.
#pragma once

namespace ds {

struct df {
  float hi, lo;
};

__device__ __forceinline__ df df_make(float hi) { return df{hi, 0.f}; }

// s + e = a + b exactly (no precondition)
__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return df{s, e};
}

// s + e = a + b exactly, valid when |a| >= |b| or a == 0
__device__ __forceinline__ df fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return df{s, __fsub_rn(b, __fsub_rn(s, a))};
}

// p + e = a * b exactly (barring underflow)
__device__ __forceinline__ df two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return df{p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ df df_add(df x, df y) {
  df s = two_sum(x.hi, y.hi);
  const float e = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
  return fast_two_sum(s.hi, e);
}

__device__ __forceinline__ df df_neg(df x) { return df{-x.hi, -x.lo}; }

__device__ __forceinline__ df df_sub(df x, df y) { return df_add(x, df_neg(y)); }

// x * f for a float32 factor f
__device__ __forceinline__ df df_mul_f(df x, float f) {
  df p = two_prod(x.hi, f);
  return fast_two_sum(p.hi, __fmaf_rn(x.lo, f, p.lo));
}

// x * y for two double-float numbers (the lo * lo term is below the precision)
__device__ __forceinline__ df df_mul(df x, df y) {
  df p = two_prod(x.hi, y.hi);
  const float e = __fmaf_rn(x.hi, y.lo, __fmul_rn(x.lo, y.hi));
  return fast_two_sum(p.hi, __fadd_rn(p.lo, e));
}

// float64 <-> double-float
__device__ __forceinline__ df df_from_double(double d) {
  const float hi = __double2float_rn(d);
  return df{hi, __double2float_rn(d - (double)hi)};
}

// float32 -> float64 by re-encoding the IEEE 754 fields with integer operations
// (exponent rebiased by 1023 - 127, the 23 fraction bits moved to the top of the
// 52): exact for normal numbers, infinities and NaNs; float32 subnormals (below
// 1.2e-38) become signed zero.  It keeps the conversions off GB300's float64
// pipe, which the run flushes of the accurate passes would otherwise saturate.
__device__ __forceinline__ double f64_of_f32(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned sign = u & 0x80000000u;
  const unsigned e = (u >> 23) & 0xFFu;
  const unsigned m = u & 0x7FFFFFu;
  unsigned hi = sign, lo = 0u;
  if (e == 0xFFu) {
    hi = sign | 0x7FF00000u | (m >> 3);
    lo = m << 29;
  } else if (e != 0u) {
    hi = sign | ((e + 896u) << 20) | (m >> 3);
    lo = m << 29;
  }
  return __hiloint2double((int)hi, (int)lo);
}

// hi + lo in float64: one float64 addition (exact, the pair holds <= 48 bits)
__device__ __forceinline__ double df_to_double(df x) { return f64_of_f32(x.hi) + f64_of_f32(x.lo); }

__device__ __forceinline__ df df_shfl_down(df x, int d) {
  return df{__shfl_down_sync(0xffffffffu, x.hi, d), __shfl_down_sync(0xffffffffu, x.lo, d)};
}

}  // namespace ds
