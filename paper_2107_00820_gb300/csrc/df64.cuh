// Double-float ("df64") arithmetic: a value is the unevaluated sum hi + lo of two
// FP32 numbers with |lo| <= ulp(hi) / 2, which carries about 48 significant bits
// (unit roundoff near 2^-48 ~ 3.6e-15).  The building blocks are the error-free
// transformations of Dekker (1971) and Knuth: TwoSum gives a + b = s + e exactly,
// and with a fused multiply-add the exact product a b = p + e, e = fma(a, b, -p).
// Addition uses the accurate form (two TwoSums and two renormalisations), so a
// sum with cancellation keeps its relative accuracy; multiplication adds the
// cross terms to the exact product of the high parts; division takes three
// correction steps from the FP32 quotient.
//
// Every operation is written with round-to-nearest intrinsics, which the
// compiler neither contracts into fused operations nor reorders.  On this GPU
// an FP32 instruction issues at about 70 times the FP64 rate, so the 7 (product)
// to 20 (sum) FP32 instructions of a df64 operation still beat one FP64 one.
// Exponent range and subnormals are those of FP32 (about 1e-38 .. 3e38).
#pragma once
#include <cuda_runtime.h>

namespace als {

struct DF64 {
  float hi, lo;
};

__device__ __forceinline__ DF64 df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return DF64{s, e};
}

// |a| >= |b| (or a == 0)
__device__ __forceinline__ DF64 df_quick_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float e = __fsub_rn(b, __fsub_rn(s, a));
  return DF64{s, e};
}

__device__ __forceinline__ DF64 df_from(double d) {
  const float h = __double2float_rn(d);
  return DF64{h, __double2float_rn(d - (double)h)};
}
__device__ __forceinline__ DF64 df_from(float f) { return DF64{f, 0.f}; }
__device__ __forceinline__ double df_to_double(DF64 a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ DF64 operator+(DF64 a, DF64 b) {
  DF64 s = df_two_sum(a.hi, b.hi);
  const DF64 t = df_two_sum(a.lo, b.lo);
  s = df_quick_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
  return df_quick_two_sum(s.hi, __fadd_rn(s.lo, t.lo));
}
__device__ __forceinline__ DF64 operator-(DF64 a) { return DF64{-a.hi, -a.lo}; }
__device__ __forceinline__ DF64 operator-(DF64 a, DF64 b) { return a + (-b); }
__device__ __forceinline__ DF64 operator*(DF64 a, DF64 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_quick_two_sum(p, e);
}
__device__ __forceinline__ DF64 operator/(DF64 a, DF64 b) {
  const float q1 = __fdiv_rn(a.hi, b.hi);
  DF64 r = a - b * DF64{q1, 0.f};
  const float q2 = __fdiv_rn(r.hi, b.hi);
  r = r - b * DF64{q2, 0.f};
  const float q3 = __fdiv_rn(r.hi, b.hi);
  return df_quick_two_sum(q1, q2) + DF64{q3, 0.f};
}
__device__ __forceinline__ DF64& operator+=(DF64& a, DF64 b) { return a = a + b; }
__device__ __forceinline__ DF64& operator-=(DF64& a, DF64 b) { return a = a - b; }
__device__ __forceinline__ bool operator>(DF64 a, float b) { return a.hi > b || (a.hi == b && a.lo > 0.f); }

// a + q p with one renormalisation (the accumulation form of df_sub_prod)
__device__ __forceinline__ DF64 df_add_prod(DF64 a, DF64 q, DF64 p) {
  const float ph = __fmul_rn(q.hi, p.hi);
  float pl = __fmaf_rn(q.hi, p.hi, -ph);
  pl = __fmaf_rn(q.hi, p.lo, pl);
  pl = __fmaf_rn(q.lo, p.hi, pl);
  const DF64 s = df_two_sum(a.hi, ph);
  return df_quick_two_sum(s.hi, __fadd_rn(__fadd_rn(s.lo, pl), a.lo));
}
// a + b with one renormalisation (error a few units of 2^-48 relative to |a| + |b|)
__device__ __forceinline__ DF64 df_add_fast(DF64 a, DF64 b) {
  const DF64 s = df_two_sum(a.hi, b.hi);
  return df_quick_two_sum(s.hi, __fadd_rn(__fadd_rn(s.lo, b.lo), a.lo));
}

// m - q p with one renormalisation: the exact product of the high parts plus the
// cross terms, one TwoSum of the high parts, the low parts added once.  The error
// is a few units of 2^-48 relative to |m| + |q p| (not to the result), which is the
// bound the backward error analysis of elimination uses for each update.
__device__ __forceinline__ DF64 df_sub_prod(DF64 m, DF64 q, DF64 p) {
  const float ph = __fmul_rn(q.hi, p.hi);
  float pl = __fmaf_rn(q.hi, p.hi, -ph);
  pl = __fmaf_rn(q.hi, p.lo, pl);
  pl = __fmaf_rn(q.lo, p.hi, pl);
  const DF64 s = df_two_sum(m.hi, -ph);
  return df_quick_two_sum(s.hi, __fadd_rn(__fsub_rn(s.lo, pl), m.lo));
}

// The two arithmetic types of the setup kernels, FP64 and DF64, behind one interface:
// conversions from FP64 inputs and to FP64/FP32 outputs, and the fused forms
// a + q p, m - q p and a + b (FP64: contracted to FMAs; DF64: one renormalisation).
template <typename R> struct RealOps;
template <> struct RealOps<double> {
  static __device__ __forceinline__ double from(double d) { return d; }
  static __device__ __forceinline__ double sub_prod(double m, double q, double p) { return m - q * p; }
  static __device__ __forceinline__ double add_prod(double a, double q, double p) { return a + q * p; }
  static __device__ __forceinline__ double add(double a, double b) { return a + b; }
  static __device__ __forceinline__ double to_double(double v) { return v; }
  static __device__ __forceinline__ float to_float(double v) { return (float)v; }
};
template <> struct RealOps<DF64> {
  static __device__ __forceinline__ DF64 from(double d) { return df_from(d); }
  static __device__ __forceinline__ DF64 sub_prod(DF64 m, DF64 q, DF64 p) { return df_sub_prod(m, q, p); }
  static __device__ __forceinline__ DF64 add_prod(DF64 a, DF64 q, DF64 p) { return df_add_prod(a, q, p); }
  static __device__ __forceinline__ DF64 add(DF64 a, DF64 b) { return df_add_fast(a, b); }
  static __device__ __forceinline__ double to_double(DF64 v) { return df_to_double(v); }
  static __device__ __forceinline__ float to_float(DF64 v) { return v.hi; }
};

}  // namespace als
