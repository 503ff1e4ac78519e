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

// Lazily normalised compensated sum (the Sum2 / Dot2 scheme of Ogita, Rump and
// Oishi, "Accurate sum and dot product", SIAM J. Sci. Comput. 26 (2005)): hi is
// the float32 sum of the terms, each added by an error-free TwoSum, and lo the
// float32 sum of the TwoSum errors, the product errors and the terms' low parts.
// hi + lo is as accurate as a double-float sum over the few dozen terms a pass
// adds between renormalisations (ds_norm) at about half the instructions, since
// no step renormalises and no product is rounded to a pair first.
struct dsum {
  float hi, lo;
};

__device__ __forceinline__ dsum ds_zero() { return dsum{0.f, 0.f}; }

__device__ __forceinline__ void ds_add(dsum& a, float x) {
  const df s = two_sum(a.hi, x);
  a.hi = s.hi;
  a.lo = __fadd_rn(a.lo, s.lo);
}

// a += x for a double-float (or unnormalised) pair x
__device__ __forceinline__ void ds_add(dsum& a, df x) {
  const df s = two_sum(a.hi, x.hi);
  a.hi = s.hi;
  a.lo = __fadd_rn(a.lo, __fadd_rn(s.lo, x.lo));
}

// a += u * v for float32 factors (the product is exact as p + pe)
__device__ __forceinline__ void ds_add_prod(dsum& a, float u, float v) {
  const df p = two_prod(u, v);
  const df s = two_sum(a.hi, p.hi);
  a.hi = s.hi;
  a.lo = __fadd_rn(a.lo, __fadd_rn(s.lo, p.lo));
}

// a += x * f for a pair x and a float32 f (x.lo * f is rounded: below the precision)
__device__ __forceinline__ void ds_add_prod(dsum& a, df x, float f) {
  const float p = __fmul_rn(x.hi, f);
  const float pe = __fmaf_rn(x.hi, f, -p);
  const df s = two_sum(a.hi, p);
  a.hi = s.hi;
  a.lo = __fadd_rn(a.lo, __fadd_rn(s.lo, __fmaf_rn(x.lo, f, pe)));
}

// a += x * y for two pairs (the lo * lo term is below the precision)
__device__ __forceinline__ void ds_add_prod(dsum& a, df x, df y) {
  const float p = __fmul_rn(x.hi, y.hi);
  const float pe = __fmaf_rn(x.hi, y.hi, -p);
  const float cross = __fmaf_rn(x.hi, y.lo, __fmul_rn(x.lo, y.hi));
  const df s = two_sum(a.hi, p);
  a.hi = s.hi;
  a.lo = __fadd_rn(a.lo, __fadd_rn(s.lo, __fadd_rn(pe, cross)));
}

// hi + lo renormalised to a double-float (TwoSum: no ordering precondition)
__device__ __forceinline__ void ds_norm(dsum& a) {
  const df s = two_sum(a.hi, a.lo);
  a.hi = s.hi;
  a.lo = s.lo;
}

__device__ __forceinline__ df ds_pair(dsum a) { return df{a.hi, a.lo}; }

__device__ __forceinline__ bool ds_nonzero(dsum a) { return a.hi != 0.f || a.lo != 0.f; }

// hi + lo in float64 (one float64 addition; exact while the pair spans <= 53 bits)
__device__ __forceinline__ double ds_to_double(dsum a) { return f64_of_f32(a.hi) + f64_of_f32(a.lo); }


}  // namespace ds
