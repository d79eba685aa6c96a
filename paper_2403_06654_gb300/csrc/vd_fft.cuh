// Shared-memory Stockham FFT engine (device side).
//
// A transform of length n = R_0 R_1 ... R_{s-1} runs s radix stages between two shared
// memory buffers (ping-pong).  Stage with radix R and span p (product of the radices before
// it) maps butterfly i in [0, n/R), with k = i mod p, as
//     u_r = src[i + r n/R] * W_{pR}^{r k}        (r = 0..R-1)
//     u   = DFT_R(u)
//     dst[(i - k) R + k + r p] = u_r
// which leaves the result in natural order (Stockham autosort).  Forward transforms use
// W = exp(-2 pi i/.), inverse ones its conjugate; neither is normalised.
//
// Many independent lines are transformed together: element idx of line l lives at
// buf[l * ls + idx * es].  Strided-axis tiles use (es, ls) = (W, 1) (W lines side by side),
// contiguous x lines use (1, n + 1).  Each thread keeps one line for the whole transform, so
// the index arithmetic needs no division by run-time widths.
#pragma once

#include "vd_common.cuh"
#include "vd_dd.cuh"

#include <type_traits>

namespace vd {

// ---------------------------------------------------------------------------------------
// small DFT codelets; S = -1 forward, +1 inverse
// ---------------------------------------------------------------------------------------

// multiply by (S i): forward -> -i, inverse -> +i
template <typename T, int S>
__device__ __forceinline__ cpx<T> mul_si(cpx<T> a) {
  return (S < 0) ? mk<T>(a.y, -a.x) : mk<T>(-a.y, a.x);
}

template <typename T, int S>
__device__ __forceinline__ void dft2(cpx<T>& a, cpx<T>& b) {
  cpx<T> t = a - b;
  a = a + b;
  b = t;
}

// LAZY_OUT (float pairs only): the outputs are left unnormalised too, for a caller whose next
// operations on them normalise (the final layer of dft8)
template <typename T, int S, bool LAZY_OUT = false>
__device__ __forceinline__ void dft4(cpx<T>* u) {
  cpx<T> a, b, c, d;
  if constexpr (std::is_same<T, dd>::value) {
    // first layer unnormalised: its sums only feed the normalising sums below
    a = cadd_lazy(u[0], u[2]);
    b = csub_lazy(u[0], u[2]);
    c = cadd_lazy(u[1], u[3]);
    d = mul_si<T, S>(csub_lazy(u[1], u[3]));
    if constexpr (LAZY_OUT) {
      u[0] = cadd_lazy(a, c);
      u[2] = csub_lazy(a, c);
      u[1] = cadd_lazy(b, d);
      u[3] = csub_lazy(b, d);
      return;
    }
  } else {
    a = u[0] + u[2];
    b = u[0] - u[2];
    c = u[1] + u[3];
    d = mul_si<T, S>(u[1] - u[3]);
  }
  u[0] = a + c;
  u[2] = a - c;
  u[1] = b + d;
  u[3] = b - d;
}

template <typename T, int S>
__device__ __forceinline__ void dft3(cpx<T>* u) {
  const T h = T(0.5);
  const T s3 = T(0.86602540378443864676372317075294);  // sqrt(3)/2
  cpx<T> t1 = u[1] + u[2];
  cpx<T> t2 = u[0] - scal(t1, h);
  cpx<T> t3 = mul_si<T, S>(scal(u[1] - u[2], s3));
  u[0] = u[0] + t1;
  u[1] = t2 + t3;
  u[2] = t2 - t3;
}

template <typename T, int S>
__device__ __forceinline__ void dft5(cpx<T>* u) {
  const T c1 = T(0.30901699437494742410229341718282);    // cos(2 pi/5)
  const T c2 = T(-0.80901699437494742410229341718282);   // cos(4 pi/5)
  const T s1 = T(0.95105651629515357211643933337938);    // sin(2 pi/5)
  const T s2 = T(0.58778525229247312916870595463907);    // sin(4 pi/5)
  cpx<T> a1 = u[1] + u[4], a2 = u[2] + u[3];
  cpx<T> b1 = u[1] - u[4], b2 = u[2] - u[3];
  cpx<T> p1 = u[0] + scal(a1, c1) + scal(a2, c2);
  cpx<T> p2 = u[0] + scal(a1, c2) + scal(a2, c1);
  cpx<T> q1 = mul_si<T, S>(scal(b1, s1) + scal(b2, s2));
  cpx<T> q2 = mul_si<T, S>(scal(b1, s2) - scal(b2, s1));
  u[0] = u[0] + a1 + a2;
  u[1] = p1 + q1;
  u[4] = p1 - q1;
  u[2] = p2 + q2;
  u[3] = p2 - q2;
}

template <typename T, int S>
__device__ __forceinline__ void dft8(cpx<T>* u) {
  const T r2 = T(0.70710678118654752440084436210485);  // 1/sqrt(2)
  cpx<T> e[4] = {u[0], u[2], u[4], u[6]};
  cpx<T> o[4] = {u[1], u[3], u[5], u[7]};
  // float pairs: the half-size transforms and the twiddle sums stay unnormalised (two lazy
  // layers, |lo| of a few ulp(hi)); the final layer and the products normalise
  constexpr bool lazy = std::is_same<T, dd>::value;
  dft4<T, S, lazy>(e);
  dft4<T, S, lazy>(o);
  // o_k *= W8^k, W8 = exp(S 2 pi i / 8)
  cpx<T> o1 = o[1], o3 = o[3];
  // W8^1 = (1 + S i)/sqrt 2 ; W8^2 = S i ; W8^3 = (-1 + S i)/sqrt 2
  if constexpr (lazy) {
    o[1] = scal(cadd_lazy(o1, mul_si<T, S>(o1)), r2);
    o[3] = scal(csub_lazy(mul_si<T, S>(o3), o3), r2);
  } else {
    o[1] = scal(o1 + mul_si<T, S>(o1), r2);
    o[3] = scal(mul_si<T, S>(o3) - o3, r2);
  }
  o[2] = mul_si<T, S>(o[2]);
  u[0] = e[0] + o[0];
  u[4] = e[0] - o[0];
  u[1] = e[1] + o[1];
  u[5] = e[1] - o[1];
  u[2] = e[2] + o[2];
  u[6] = e[2] - o[2];
  u[3] = e[3] + o[3];
  u[7] = e[3] - o[3];
}

// 16-point DFT as 4 x 4 (n = 4a + b, k = c + 4d) with the internal twiddles W16^{bc}
template <typename T, int S>
__device__ __forceinline__ cpx<T> w16(cpx<T> v, int m) {
  // v * exp(S 2 pi i m / 16), m in {0, 1, 2, 3, 4, 6, 9}
  const T c1 = T(0.92387953251128675612818318939679);   // cos(pi/8)
  const T s1 = T(0.38268343236508977172845998403040);   // sin(pi/8)
  const T r2 = T(0.70710678118654752440084436210485);   // 1/sqrt(2)
  switch (m) {
    case 0: return v;
    case 1: return cmul(v, mk<T>(c1, T(S) * s1));
    case 2: return scal(v + mul_si<T, S>(v), r2);
    case 3: return cmul(v, mk<T>(s1, T(S) * c1));
    case 4: return mul_si<T, S>(v);
    case 6: return scal(mul_si<T, S>(v) - v, r2);
    default: return cmul(v, mk<T>(-c1, T(-S) * s1));   // m = 9: cos(9pi/8), S sin(9pi/8)
  }
}

template <typename T, int S>
__device__ __forceinline__ void dft16(cpx<T>* u) {
  cpx<T> v[4][4];
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    cpx<T> t[4] = {u[b], u[4 + b], u[8 + b], u[12 + b]};
    dft4<T, S>(t);
#pragma unroll
    for (int c = 0; c < 4; ++c) v[b][c] = w16<T, S>(t[c], b * c);
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    cpx<T> t[4] = {v[0][c], v[1][c], v[2][c], v[3][c]};
    dft4<T, S>(t);
#pragma unroll
    for (int d = 0; d < 4; ++d) u[c + 4 * d] = t[d];
  }
}

template <typename T, int S, int R>
__device__ __forceinline__ void dftR(cpx<T>* u) {
  if constexpr (R == 2) {
    dft2<T, S>(u[0], u[1]);
  } else if constexpr (R == 3) {
    dft3<T, S>(u);
  } else if constexpr (R == 4) {
    dft4<T, S>(u);
  } else if constexpr (R == 5) {
    dft5<T, S>(u);
  } else if constexpr (R == 16) {
    dft16<T, S>(u);
  } else {
    dft8<T, S>(u);
  }
}

// One Stockham stage.  Every thread owns one line (element idx of it at
// buf[lofs + idx * es]) and the butterflies i0, i0 + istep, ... of that line.  k = i mod p
// uses a mask when p is a power of two (pmask >= 0), an integer division otherwise.
template <typename T, int S, int R>
__device__ __forceinline__ void stockham_stage(const cpx<T>* __restrict__ src, cpx<T>* __restrict__ dst, int es,
                                               int lofs, int i0, int istep, int n, int p,
                                               const cpx<T>* __restrict__ tw) {
  const int nb = n / R;
  const int tws = n / (p * R);
  const int pmask = ((p & (p - 1)) == 0) ? p - 1 : -1;
#pragma unroll 1
  for (int i = i0; i < nb; i += istep) {
    const int k = (pmask >= 0) ? (i & pmask) : (i % p);
    const cpx<T>* s = src + lofs;
    cpx<T> u[R];
#pragma unroll
    for (int r = 0; r < R; ++r) u[r] = s[(i + r * nb) * es];
    if (p > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        const cpx<T> w = tw[r * k * tws];
        u[r] = (S < 0) ? cmul(u[r], w) : cmulc(u[r], w);
      }
    }
    dftR<T, S, R>(u);
    cpx<T>* d = dst + lofs + ((i - k) * R + k) * es;
#pragma unroll
    for (int r = 0; r < R; ++r) d[r * p * es] = u[r];
  }
}

// Full transform of every line of the block; input in a.  Returns the buffer holding the
// result.  Must be called by all threads of the block (syncs before every stage and at the end).
template <typename T, int S>
__device__ cpx<T>* fft_lines(cpx<T>* a, cpx<T>* b, int es, int lofs, int i0, int istep, const FftPlan& pl,
                             const cpx<T>* tw) {
  cpx<T>* src = a;
  cpx<T>* dst = b;
  int p = 1;
  for (int s = 0; s < pl.nst; ++s) {
    const int R = pl.rad[s];
    __syncthreads();
    switch (R) {
      case 2: stockham_stage<T, S, 2>(src, dst, es, lofs, i0, istep, pl.n, p, tw); break;
      case 3: stockham_stage<T, S, 3>(src, dst, es, lofs, i0, istep, pl.n, p, tw); break;
      case 4: stockham_stage<T, S, 4>(src, dst, es, lofs, i0, istep, pl.n, p, tw); break;
      case 5: stockham_stage<T, S, 5>(src, dst, es, lofs, i0, istep, pl.n, p, tw); break;
      default: stockham_stage<T, S, 8>(src, dst, es, lofs, i0, istep, pl.n, p, tw); break;
    }
    p *= R;
    cpx<T>* t = src;
    src = dst;
    dst = t;
  }
  __syncthreads();
  return src;
}

// 1/x: for double an FP32 seed refined by two Newton steps r <- r (2 - x r); for float the
// correctly rounded single-precision reciprocal.
__device__ __forceinline__ double recip(double x) {
  double r = (double)__frcp_rn((float)x);
  double e = fma(-x, r, 1.0);
  r = fma(r, e, r);
  e = fma(-x, r, 1.0);
  return fma(r, e, r);
}
__device__ __forceinline__ float recip(float x) { return __frcp_rn(x); }

// diagonal symbol value for |k~|^2 = k2 (corner modes have k2 == 0 exactly)
template <typename T>
__device__ __forceinline__ T symbol_value(int kind, T a, T k2) {
  if (kind == SYM_PRESSURE) return (k2 == T(0)) ? T(0) : -recip(k2);
  if (kind == SYM_VELOCITY) return recip(T(1) + a * k2);
  if (kind == SYM_PROJECT) return (k2 == T(0)) ? T(0) : T(1);
  return T(1);
}

}  // namespace vd
