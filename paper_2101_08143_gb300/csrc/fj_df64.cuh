// fj_df64.cuh - double-float ("df64") arithmetic for the refinement path.
//
// A df64 value is the unevaluated sum hi + lo of two float32 numbers with
// |lo| <= ulp(hi)/2, about 48 bits of significand.  GB300 runs float64 at a
// small fraction of its float32 rate, so the float64-accurate parts of the
// mixed-precision solve (residuals, refined iterate, quantity sums) are
// computed with these float32 sequences instead.  A df64 has float32's
// exponent range (normal numbers from about 1e-38 to 3e38); the solver keeps
// its values near 1 by scaling each right-hand side by a power of two first.
// The sequences:
//   two_sum         Knuth's error-free sum (TAOCP vol. 2, 4.2.2)
//   quick_two_sum   Dekker's fast two-sum for |a| >= |b| (Dekker 1971)
//   exact product   p = a*b, e = fma(a, b, -p)  (Dekker's product via FMA)
//   add / mul       the "sloppy" double-double sum and product of Hida, Li
//                   and Bailey's QD library (2001), relative error ~2^-47
// Every step uses the _rn intrinsics so that the compiler cannot contract or
// reassociate them.
#pragma once

#include <cuda_runtime.h>

namespace fj {

struct df64 {
  float hi, lo;
};

__device__ __forceinline__ df64 df_make(float hi, float lo) {
  df64 r;
  r.hi = hi;
  r.lo = lo;
  return r;
}

__device__ __forceinline__ df64 df_from_float(float x) { return df_make(x, 0.0f); }

__device__ __forceinline__ df64 df_from_double(double x) {
  const float hi = __double2float_rn(x);
  const float lo = __double2float_rn(x - (double)hi);
  return df_make(hi, lo);
}

__device__ __forceinline__ double df_to_double(df64 a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ df64 quick_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float e = __fsub_rn(b, __fsub_rn(s, a));
  return df_make(s, e);
}

__device__ __forceinline__ df64 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return df_make(s, e);
}

__device__ __forceinline__ df64 df_add(df64 a, df64 b) {
  const df64 s = two_sum(a.hi, b.hi);
  return quick_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ df64 df_neg(df64 a) { return df_make(-a.hi, -a.lo); }

__device__ __forceinline__ df64 df_sub(df64 a, df64 b) { return df_add(a, df_neg(b)); }

__device__ __forceinline__ df64 df_add_f(df64 a, float b) {
  const df64 s = two_sum(a.hi, b);
  return quick_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}

__device__ __forceinline__ df64 df_mul(df64 a, df64 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return quick_two_sum(p, e);
}

__device__ __forceinline__ df64 df_mul_f(df64 a, float w) {
  const float p = __fmul_rn(a.hi, w);
  float e = __fmaf_rn(a.hi, w, -p);
  e = __fmaf_rn(a.lo, w, e);
  return quick_two_sum(p, e);
}

// Operators, so that the templated walks run unchanged on df64.
__device__ __forceinline__ df64 operator+(df64 a, df64 b) { return df_add(a, b); }
__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return df_sub(a, b); }
__device__ __forceinline__ df64 operator*(df64 a, df64 b) { return df_mul(a, b); }
__device__ __forceinline__ df64& operator+=(df64& a, df64 b) {
  a = df_add(a, b);
  return a;
}

// Value construction and conversion used by the templated code paths.
template <typename T>
__device__ __forceinline__ T num(float x) {
  return T(x);
}
template <>
__device__ __forceinline__ df64 num<df64>(float x) {
  return df_from_float(x);
}
__device__ __forceinline__ double to_double(float x) { return (double)x; }
__device__ __forceinline__ double to_double(double x) { return x; }
__device__ __forceinline__ double to_double(df64 x) { return df_to_double(x); }

// w * d for an edge weight w: one exact-product step for df64.
__device__ __forceinline__ float mul_w(float d, float w) { return w * d; }
__device__ __forceinline__ double mul_w(double d, float w) { return (double)w * d; }
__device__ __forceinline__ df64 mul_w(df64 d, float w) { return df_mul_f(d, w); }

// Refinement arithmetic per inner type: float32 inner iterations are refined
// in double-float, float64 inner iterations in plain float64 (the FP64 mode
// is float64 throughout).
template <typename VI>
struct Refine {
  using type = df64;
};
template <>
struct Refine<double> {
  using type = double;
};

template <typename R>
__device__ __forceinline__ R from_double(double x);
template <>
__device__ __forceinline__ double from_double<double>(double x) {
  return x;
}
template <>
__device__ __forceinline__ df64 from_double<df64>(double x) {
  return df_from_double(x);
}

// A refinement value rounded to the inner type.
template <typename VI>
__device__ __forceinline__ VI to_inner(df64 r) {
  return (VI)r.hi + (VI)r.lo;
}
template <typename VI>
__device__ __forceinline__ VI to_inner(double r) {
  return (VI)r;
}

// q + e for a refined iterate q and an inner correction e.
__device__ __forceinline__ df64 add_inner(df64 q, float e) { return df_add_f(q, e); }
__device__ __forceinline__ double add_inner(double q, double e) { return q + e; }

// Warp xor-shuffle for every value type of the walks.
__device__ __forceinline__ float shfl_xor_v(float v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
__device__ __forceinline__ double shfl_xor_v(double v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
__device__ __forceinline__ df64 shfl_xor_v(df64 v, int m) {
  return df_make(__shfl_xor_sync(0xffffffffu, v.hi, m), __shfl_xor_sync(0xffffffffu, v.lo, m));
}

}  // namespace fj
