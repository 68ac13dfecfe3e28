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
#include <type_traits>

#include <cuda_runtime.h>

#include <complex>

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

// Structure of an operator coefficient, uniform across a launch (or a sweep): the structured kernels
// branch on it so that a zero costs nothing, a one an add, and a real or imaginary coefficient two real
// multiply-adds instead of four.
enum { FL_ZERO = 0, FL_ONE = 1, FL_REAL = 2, FL_IMAG = 3, FL_CPLX = 4 };

template <class T> struct V2;
template <> struct V2<float> { using t = float2; };
template <> struct V2<double> { using t = double2; };
template <> struct V2<df> { using t = cdf; };
template <class T> using cx = typename V2<T>::t;

// acc += c x for a coefficient of structure fl.  CPLX_FIRST tests the complex case first: most terms of a
// composed (fused) operator are complex, and the FP64 fused sweeps measured 10% faster so; the plain FP64
// passes and the float-float accumulator below measured faster with the complex case last.
template <class T, bool CPLX_FIRST = false>
__device__ __forceinline__ void cmac_flag(cx<T>& acc, const cx<T>& c, int fl, const cx<T>& x) {
  if (CPLX_FIRST && fl == FL_CPLX) {
    acc.x = fma(c.x, x.x, acc.x);
    acc.x = fma(-c.y, x.y, acc.x);
    acc.y = fma(c.x, x.y, acc.y);
    acc.y = fma(c.y, x.x, acc.y);
    return;
  }
  if (fl == FL_ZERO) return;
  if (fl == FL_ONE) { acc.x += x.x; acc.y += x.y; return; }
  if (fl == FL_REAL) { acc.x = fma(c.x, x.x, acc.x); acc.y = fma(c.x, x.y, acc.y); return; }
  if (fl == FL_IMAG) { acc.x = fma(-c.y, x.y, acc.x); acc.y = fma(c.y, x.x, acc.y); return; }
  acc.x = fma(c.x, x.x, acc.x);
  acc.x = fma(-c.y, x.y, acc.x);
  acc.y = fma(c.x, x.y, acc.y);
  acc.y = fma(c.y, x.x, acc.y);
}

// x <- f x for a diagonal factor of structure fl (FL_ONE leaves x as it is); CPLX_FIRST as in cmac_flag
template <class T, bool CPLX_FIRST = false>
__device__ __forceinline__ void cscale_flag(cx<T>& x, const cx<T>& f, int fl) {
  if (CPLX_FIRST && fl == FL_CPLX) {
    const T re = fma(x.x, f.x, -(x.y * f.y));
    x.y = fma(x.x, f.y, x.y * f.x);
    x.x = re;
    return;
  }
  if (fl == FL_ONE) return;
  if (fl == FL_ZERO) { x.x = T(0.0f); x.y = T(0.0f); return; }
  if (fl == FL_REAL) { x.x = x.x * f.x; x.y = x.y * f.x; return; }
  if (fl == FL_IMAG) { const T re = -(x.y * f.y); x.y = x.x * f.y; x.x = re; return; }
  const T re = fma(x.x, f.x, -(x.y * f.y));
  x.y = fma(x.x, f.y, x.y * f.x);
  x.x = re;
}

// Accumulator of a complex sum of products sum_j c_j x_j.  For float and double it is the complex value
// itself (one FMA per real product).  For float-float it keeps, per real and imaginary part, a running
// float sum s whose rounding errors (Knuth two-sum) and the products' low parts (exact FMA residue and
// the cross terms with the low words) are gathered in a second float l, normalised once at the end:
// the compensated dot product "Dot2" of Ogita, Rump and Oishi (SIAM J. Sci. Comput. 2005), as accurate
// as a float-float evaluation, with one float add on the critical path per term instead of a
// renormalisation after every term.
template <class T>
struct CAcc {
  cx<T> v;
  __device__ __forceinline__ void zero() { v.x = T(0.0f); v.y = T(0.0f); }
  __device__ __forceinline__ void mac(const cx<T>& c, int fl, const cx<T>& x) {
    cmac_flag<T, std::is_same<T, double>::value>(v, c, fl, x);
  }
  __device__ __forceinline__ cx<T> get() const { return v; }
};

__device__ __forceinline__ void dot2_step(float& s, float& l, const df& a, const df& b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  const float s2 = s + p;
  const float v = s2 - s;
  const float err = (s - (s2 - v)) + (p - v);
  s = s2;
  l = l + (err + e);
}
__device__ __forceinline__ void dot2_add(float& s, float& l, const df& a) {
  const float s2 = s + a.hi;
  const float v = s2 - s;
  const float err = (s - (s2 - v)) + (a.hi - v);
  s = s2;
  l = l + (err + a.lo);
}

template <>
struct CAcc<df> {
  float rs, rl, is, il;
  __device__ __forceinline__ void zero() { rs = rl = is = il = 0.0f; }
  __device__ __forceinline__ void mac(const cdf& c, int fl, const cdf& x) {
    if (fl == FL_ZERO) return;
    if (fl == FL_ONE) {
      dot2_add(rs, rl, x.x);
      dot2_add(is, il, x.y);
      return;
    }
    if (fl == FL_REAL) {
      dot2_step(rs, rl, c.x, x.x);
      dot2_step(is, il, c.x, x.y);
      return;
    }
    if (fl == FL_IMAG) {
      dot2_step(rs, rl, -c.y, x.y);
      dot2_step(is, il, c.y, x.x);
      return;
    }
    dot2_step(rs, rl, c.x, x.x);
    dot2_step(rs, rl, -c.y, x.y);
    dot2_step(is, il, c.x, x.y);
    dot2_step(is, il, c.y, x.x);
  }
  __device__ __forceinline__ cdf get() const {
    cdf r;
    r.x = df_fast_two_sum(rs, rl);
    r.y = df_fast_two_sum(is, il);
    return r;
  }
};

}  // namespace dev

// Host-side structure of a coefficient (FL_*), for the structured kernels.
inline int flag_of(const std::complex<double>& c) {
  if (c == 0.0) return dev::FL_ZERO;
  if (c == 1.0) return dev::FL_ONE;
  if (c.imag() == 0.0) return dev::FL_REAL;
  if (c.real() == 0.0) return dev::FL_IMAG;
  return dev::FL_CPLX;
}

}  // namespace vqd
