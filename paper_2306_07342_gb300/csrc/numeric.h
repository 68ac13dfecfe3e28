// Scalar and complex element types of the state, shared by the CUDA sources.
//
// float (complex64), double (complex128) and df, a float-float number: an unevaluated sum
// hi + lo of two floats with |lo| <= ulp(hi)/2, about 48 significant bits.  A df state stores each
// amplitude as (re.hi, re.lo, im.hi, im.lo), 16 bytes like complex128, but its arithmetic runs on the
// FP32 pipes, which on this GPU are about 58 times faster than its FP64 pipes.  The arithmetic uses
// the error-free transformations of Knuth (two-sum), Dekker (fast two-sum) and the FMA-based exact
// product (Ogita, Rump and Oishi, "Accurate sum and dot product", SIAM J. Sci. Comput. 2005); the
// double-word formulas follow Joldes, Muller and Popescu, "Tight and rigorous error bounds for basic
// building blocks of double-word arithmetic", ACM TOMS 2017 (the "sloppy" sum and the product with
// one FMA chain).  The CUDA sources are compiled without fast-math, so no float operation below is
// reassociated.
#pragma once

#include <cuda_runtime.h>

namespace vqd {
namespace dev {

// the float and double fma overloads stay visible next to the df one declared below
using ::fma;

struct df {
  float hi, lo;
  df() = default;
  __host__ __device__ constexpr df(float h, float l) : hi(h), lo(l) {}
  // nearest float, then the rounding error of that float as the low word
  __host__ __device__ constexpr df(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
  __host__ __device__ explicit constexpr operator double() const { return (double)hi + (double)lo; }
};

// s + e = a + b exactly (Knuth two-sum)
__device__ __forceinline__ df df_two_sum(float a, float b) {
  const float s = a + b;
  const float v = s - a;
  const float e = (a - (s - v)) + (b - v);
  return df(s, e);
}
// s + e = a + b exactly when |a| >= |b| or a == 0 (Dekker fast two-sum)
__device__ __forceinline__ df df_fast_two_sum(float a, float b) {
  const float s = a + b;
  const float e = b - (s - a);
  return df(s, e);
}

__device__ __forceinline__ df operator+(df a, df b) {
  const df s = df_two_sum(a.hi, b.hi);
  return df_fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}
__device__ __forceinline__ df operator-(df a) { return df(-a.hi, -a.lo); }
__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }
__device__ __forceinline__ df operator*(df a, df b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);  // exact low part of a.hi * b.hi
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return df_fast_two_sum(p, e);
}
// a * b + c, with the exact product's low part carried into the sum
__device__ __forceinline__ df fma(df a, df b, df c) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  const df s = df_two_sum(p, c.hi);
  return df_fast_two_sum(s.hi, s.lo + (e + c.lo));
}
__device__ __forceinline__ df& operator+=(df& a, df b) { return a = a + b; }
__device__ __forceinline__ df& operator*=(df& a, df b) { return a = a * b; }

struct __align__(16) cdf {
  df x, y;
};

template <class T> struct V2;
template <> struct V2<float> { using t = float2; };
template <> struct V2<double> { using t = double2; };
template <> struct V2<df> { using t = cdf; };
template <class T> using cx = typename V2<T>::t;

}  // namespace dev
}  // namespace vqd
