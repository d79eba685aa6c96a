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

#include "vd_common.cuh"

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

// a b + c d with one renormalisation: both products are formed as (p, e) with p = fl(hi hi)
// and e its FMA error plus the cross terms, the high parts are summed exactly (two_sum) and
// the error terms in float.  19 float operations against 25 for two products and a sum;
// absolute error ~2^-47 (|a b| + |c d|), the normwise bound a transform needs.
__device__ __forceinline__ dd dd_sum_prod(dd a, dd b, dd c, dd d) {
  const float p = a.hi * b.hi;
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const float q = c.hi * d.hi;
  float f = __fmaf_rn(c.hi, d.hi, -q);
  f = __fmaf_rn(c.hi, d.lo, f);
  f = __fmaf_rn(c.lo, d.hi, f);
  const dd s = dd_two_sum(p, q);
  return dd_fast_two_sum(s.hi, s.lo + (e + f));
}

// complex products on float pairs (preferred over the generic templates by overload
// resolution): a w and a conj(w)
__device__ __forceinline__ cpx<dd> cmul(cpx<dd> a, cpx<dd> w) {
  return mk<dd>(dd_sum_prod(a.x, w.x, -a.y, w.y), dd_sum_prod(a.x, w.y, a.y, w.x));
}
__device__ __forceinline__ cpx<dd> cmulc(cpx<dd> a, cpx<dd> w) {
  return mk<dd>(dd_sum_prod(a.x, w.x, a.y, w.y), dd_sum_prod(a.y, w.x, -a.x, w.y));
}

// a + b without the final renormalisation: exact sum of the high parts, low parts added in
// float, so |lo| may reach a few ulp(hi).  Only for values that go straight into normalising
// additions (the first layer of a radix-4 butterfly); the pair still carries ~2^-47 relative
// accuracy.
__device__ __forceinline__ dd dd_add_lazy(dd a, dd b) {
  const dd s = dd_two_sum(a.hi, b.hi);
  return dd(s.hi, s.lo + (a.lo + b.lo));
}
__device__ __forceinline__ cpx<dd> cadd_lazy(cpx<dd> a, cpx<dd> b) {
  return mk<dd>(dd_add_lazy(a.x, b.x), dd_add_lazy(a.y, b.y));
}
__device__ __forceinline__ cpx<dd> csub_lazy(cpx<dd> a, cpx<dd> b) {
  return mk<dd>(dd_add_lazy(a.x, -b.x), dd_add_lazy(a.y, -b.y));
}

// Conversions to and from double, on the integer pipes.  The FP64 pipe of GB300 runs at ~1/64
// of the float rate, so the conversions are done on the IEEE bit patterns.
//
// float -> double, exact for normal floats, zero, inf and nan (subnormal floats flush to zero).
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned long long s = (unsigned long long)(u & 0x80000000u) << 32;
  const unsigned e = (u >> 23) & 0xffu;
  const unsigned long long m = (unsigned long long)(u & 0x7fffffu) << 29;
  unsigned long long out = s;   // zero and subnormal floats
  if (e == 0xffu) out = s | (0x7ffull << 52) | m;
  else if (e != 0u) out = s | ((unsigned long long)(e - 127u + 1023u) << 52) | m;
  return __longlong_as_double((long long)out);
}

// double -> float pair: hi = the 53-bit significand rounded (half up) to 24 bits, lo = the
// exact remainder (at most 29 bits) rounded to a float, so v = hi + lo to ~2^-48 |v| and
// |lo| <= ulp(hi) / 2.  |v| >= 2^128 gives hi = +-inf, |v| < 2^-126 gives zero (subnormal
// floats are not formed), inf and nan pass to hi; lo is dropped below 2^-149 |scale|.
__device__ __forceinline__ dd dd_from_double(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const unsigned sgn = (unsigned)(b >> 32) & 0x80000000u;
  const int E = (int)((b >> 52) & 0x7ffu);
  if (E == 0x7ff) return dd(__uint_as_float(sgn | 0x7f800000u | (unsigned)((b >> 29) & 0x7fffffu)), 0.0f);
  const unsigned long long sig = (1ull << 52) | (b & 0xfffffffffffffull);
  const unsigned long long sig_r = ((sig >> 29) + ((sig >> 28) & 1ull)) << 29;
  const long long diff = (long long)sig - (long long)sig_r;   // |diff| <= 2^28
  const unsigned long long hr = sig_r >> 29;                 // 2^23 .. 2^24
  const int carry = (hr >> 24) ? 1 : 0;
  const int fe = E - 1023 + 127 + carry;
  if (E == 0 || fe <= 0) return dd(__uint_as_float(sgn), 0.0f);
  if (fe >= 255) return dd(__uint_as_float(sgn | 0x7f800000u), 0.0f);
  const float hi = __uint_as_float(sgn | ((unsigned)fe << 23) | (carry ? 0u : (unsigned)(hr & 0x7fffffu)));
  // lo = diff * 2^(E - 1075): the 2^k factor as float bits when it is a normal float
  const int ke = E - 1075 + 127;
  float lo = 0.0f;
  if (ke >= 1 && ke <= 254) {
    const float mag = (float)(int)diff * __uint_as_float((unsigned)ke << 23);   // |diff| < 2^31
    lo = sgn ? -mag : mag;
  }
  return dd(hi, lo);
}
__device__ __forceinline__ double dd_to_double(dd a) { return f2d_bits(a.hi) + f2d_bits(a.lo); }

}  // namespace vd
