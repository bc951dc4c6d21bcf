// igks_df64.cuh -- double-float numbers for the LU-SGS sweeps: a value is the unevaluated
// sum hi + lo of two FP32 numbers (|lo| <= ulp(hi) / 2), about 48 significant bits.
//
// Why: on GB300 a dependent FP64 instruction takes 64 cycles and an SM issues one FP64
// warp instruction per ~19 cycles whatever the number of active lanes, while FP32 runs
// at 7 cycles and more than three warp instructions per cycle. The sweeps are a chain of
// dependent arithmetic over a few cells per level, so FP64-grade accuracy is cheaper on
// the FP32 pipes. The arithmetic is Dekker's (1971) error-free transformations: the sum
// of two floats is s + e exactly with s = a + b (Knuth's two-sum), and the product is
// p + e exactly with p = a b, e = fma(a, b, -p); a result is renormalised with the
// quick two-sum (|a| >= |b|). Addition folds the low parts into the error of the high
// parts (the "sloppy" sum, error a few units of 2^-48 of the larger operand); division
// takes one Newton correction of the FP32 quotient. Every step is an explicitly rounded
// operation (__fadd_rn, __fmul_rn, __fmaf_rn): the transformations are exact only if the
// compiler does not fuse a product into a following sum, which it may do with plain
// operators.
#pragma once
#include <cuda_runtime.h>

namespace igks {

struct __align__(8) df64 {
  float hi, lo;
  __host__ __device__ constexpr df64() : hi(0.0f), lo(0.0f) {}
  __host__ __device__ constexpr df64(float h, float l) : hi(h), lo(l) {}
  // from a double: the nearest float and the float nearest the remainder (constant-folded
  // for constant arguments)
  __host__ __device__ constexpr df64(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
  __host__ __device__ constexpr df64(int x) : hi((float)x), lo(0.0f) {}
};

__device__ __forceinline__ double to_double(df64 a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ double to_double(double a) { return a; }
__device__ __forceinline__ double to_double(float a) { return (double)a; }

// |a| >= |b| (or a = 0): s + e = a + b exactly
__device__ __forceinline__ df64 df_quick(float a, float b) {
  const float s = __fadd_rn(a, b);
  return df64(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ df64 operator+(df64 a, df64 b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));   // s + e = a.hi + b.hi exactly
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  return df_quick(s, e);
}

__device__ __forceinline__ df64 operator-(df64 a) { return df64(-a.hi, -a.lo); }
__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }

__device__ __forceinline__ df64 operator*(df64 a, df64 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);         // p + e = a.hi b.hi exactly
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_quick(p, e);
}

__device__ __forceinline__ df64 operator/(df64 a, df64 b) {
  const float q1 = __fdiv_rn(a.hi, b.hi);
  const df64 r = a - b * df64(q1, 0.0f);       // remainder of the FP32 quotient
  const float q2 = __fdiv_rn(r.hi, b.hi);
  return df_quick(q1, q2);
}

__device__ __forceinline__ df64& operator+=(df64& a, df64 b) { return a = a + b; }
__device__ __forceinline__ df64& operator-=(df64& a, df64 b) { return a = a - b; }

}  // namespace igks
