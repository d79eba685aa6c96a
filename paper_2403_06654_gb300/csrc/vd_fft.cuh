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
// buf[l * ls + idx * es].  Strided-axis tiles use (es, ls) = (W, 1), contiguous x lines use
// (1, n + pad); LINE_FAST selects the thread mapping that keeps shared-memory accesses of a
// warp on consecutive addresses for each layout.
#pragma once

#include "vd_common.cuh"

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

template <typename T, int S>
__device__ __forceinline__ void dft4(cpx<T>* u) {
  cpx<T> a = u[0] + u[2], b = u[0] - u[2];
  cpx<T> c = u[1] + u[3], d = mul_si<T, S>(u[1] - u[3]);
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
  dft4<T, S>(e);
  dft4<T, S>(o);
  // o_k *= W8^k, W8 = exp(S 2 pi i / 8)
  cpx<T> o1 = o[1], o3 = o[3];
  // W8^1 = (1 + S i)/sqrt 2 ; W8^2 = S i ; W8^3 = (-1 + S i)/sqrt 2
  o[1] = scal(o1 + mul_si<T, S>(o1), r2);
  o[2] = mul_si<T, S>(o[2]);
  o[3] = scal(mul_si<T, S>(o3) - o3, r2);
  u[0] = e[0] + o[0];
  u[4] = e[0] - o[0];
  u[1] = e[1] + o[1];
  u[5] = e[1] - o[1];
  u[2] = e[2] + o[2];
  u[6] = e[2] - o[2];
  u[3] = e[3] + o[3];
  u[7] = e[3] - o[3];
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
  } else {
    dft8<T, S>(u);
  }
}

// one Stockham stage over nlines lines
template <typename T, int S, int R, bool LINE_FAST>
__device__ __forceinline__ void stockham_stage(const cpx<T>* __restrict__ src, cpx<T>* __restrict__ dst,
                                               int es, int ls, int nlines, int n, int p,
                                               const cpx<T>* __restrict__ tw, int tid, int nthr) {
  const int nb = n / R;
  const int total = nb * nlines;
  const int tws = n / (p * R);
  for (int q = tid; q < total; q += nthr) {
    int line, i;
    if (LINE_FAST) {
      line = q % nlines;
      i = q / nlines;
    } else {
      i = q % nb;
      line = q / nb;
    }
    const int k = i % p;
    const cpx<T>* s = src + line * ls;
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
    cpx<T>* d = dst + line * ls + ((i - k) * R + k) * es;
#pragma unroll
    for (int r = 0; r < R; ++r) d[r * p * es] = u[r];
  }
}

// Full transform; input in a.  Returns the buffer holding the result.
// Must be called by all threads of the block; syncs before every stage and at the end.
template <typename T, int S, bool LINE_FAST>
__device__ cpx<T>* fft_pingpong(cpx<T>* a, cpx<T>* b, int es, int ls, int nlines, const FftPlan& pl,
                                const cpx<T>* tw, int tid, int nthr) {
  cpx<T>* src = a;
  cpx<T>* dst = b;
  int p = 1;
  for (int s = 0; s < pl.nst; ++s) {
    const int R = pl.rad[s];
    __syncthreads();
    switch (R) {
      case 2: stockham_stage<T, S, 2, LINE_FAST>(src, dst, es, ls, nlines, pl.n, p, tw, tid, nthr); break;
      case 3: stockham_stage<T, S, 3, LINE_FAST>(src, dst, es, ls, nlines, pl.n, p, tw, tid, nthr); break;
      case 4: stockham_stage<T, S, 4, LINE_FAST>(src, dst, es, ls, nlines, pl.n, p, tw, tid, nthr); break;
      case 5: stockham_stage<T, S, 5, LINE_FAST>(src, dst, es, ls, nlines, pl.n, p, tw, tid, nthr); break;
      default: stockham_stage<T, S, 8, LINE_FAST>(src, dst, es, ls, nlines, pl.n, p, tw, tid, nthr); break;
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
