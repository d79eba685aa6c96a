// Float-pair ("double-float") arithmetic: a value is hi + lo with two floats, |lo| <= ulp(hi)/2,
// giving a ~48-bit significand on the FP32 pipes.  On GB300 the FP64 pipe runs at 1/69 of
// the FP32 rate, so transforms in float-pair arithmetic are much faster than in double while
// keeping an error bound ~2^-48 (vs 2^-53 for double).
//
// Built from the classical error-free transformations:
//   two_sum (Knuth):        s = a + b, e = (a - (s - bb)) + (b - bb) with bb = s - a
//   fast_two_sum (Dekker):  s = a + b, e = b - (s - a)            (|a| >= |b|)
//   two_prod (with FMA):    p = a b,   e = fma(a, b, -p)
// Addition is the "sloppy" variant (the low parts are added without compensation): its
// absolute error is bounded by a small multiple of 2^-48 (|a| + |b|), which is the normwise
// bound an FFT needs.
#pragma once

#include <cuda_runtime.h>

namespace vd {

struct dd {
  float hi, lo;
  dd() = default;
  __host__ __device__ constexpr dd(float h, float l) : hi(h), lo(l) {}
  // exact for |v| < 2^24 integers and for float values
  __host__ __device__ constexpr dd(int v) : hi((float)v), lo(0.0f) {}
  // split of a double (constant-folded for literals)
  __host__ __device__ constexpr dd(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
};

__device__ __forceinline__ dd dd_fast_two_sum(float a, float b) {
  const float s = a + b;
  return dd(s, b - (s - a));
}

__device__ __forceinline__ dd dd_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return dd(s, (a - (s - bb)) + (b - bb));
}

__device__ __forceinline__ dd operator+(dd a, dd b) {
  dd s = dd_two_sum(a.hi, b.hi);
  return dd_fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}

__device__ __forceinline__ dd operator-(dd a) { return dd(-a.hi, -a.lo); }
__device__ __forceinline__ dd operator-(dd a, dd b) { return a + (-b); }

__device__ __forceinline__ dd operator*(dd a, dd b) {
  const float p = a.hi * b.hi;
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return dd_fast_two_sum(p, e);
}

__device__ __forceinline__ dd& operator*=(dd& a, dd b) {
  a = a * b;
  return a;
}
__device__ __forceinline__ dd& operator+=(dd& a, dd b) {
  a = a + b;
  return a;
}

// conversions to and from double (exact split / exact sum of the two parts)
__device__ __forceinline__ dd dd_from_double(double v) {
  const float h = __double2float_rn(v);
  return dd(h, __double2float_rn(v - (double)h));
}
__device__ __forceinline__ double dd_to_double(dd a) { return (double)a.hi + (double)a.lo; }

}  // namespace vd
