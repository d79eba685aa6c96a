// Complex float pairs in packed two-float registers (sm_100 family): the real and imaginary
// parts of a complex float-pair value side by side, hi = (re.hi, im.hi) and lo = (re.lo, im.lo),
// so that one packed instruction (add / sub / mul / fma .rn.f32x2) does the float work of both
// parts.  Every operation is the complex float-pair operation of vd_dd.cuh / vd_fft.cuh applied
// to the two parts: the same IEEE operations in the same order on each lane (a negation is a
// multiply by -1, exact; a - b is a + (-b) as in vd_dd.cuh, using fl(x + (-y)) = fl(x - y); a
// complex product pairs the value and its swapped copy with twiddle entries laid out for the
// lanes, p_cmul), so results are bit-identical to the unpacked code.
#pragma once

#include <cuda_runtime.h>

#include "vd_common.cuh"
#include "vd_dd.cuh"

namespace vd {

typedef unsigned long long f2r;   // two floats: lane 0 (low half) = real part, lane 1 = imaginary

__device__ __forceinline__ f2r f2_pack(float a, float b) {
  f2r r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ float f2_l0(f2r r) {
  float a;
  asm("{\n\t.reg .f32 t;\n\tmov.b64 {%0, t}, %1;\n\t}" : "=f"(a) : "l"(r));
  return a;
}
__device__ __forceinline__ float f2_l1(f2r r) {
  float b;
  asm("{\n\t.reg .f32 t;\n\tmov.b64 {t, %0}, %1;\n\t}" : "=f"(b) : "l"(r));
  return b;
}
__device__ __forceinline__ f2r f2_add(f2r a, f2r b) {
  f2r d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2r f2_sub(f2r a, f2r b) {
  f2r d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2r f2_mul(f2r a, f2r b) {
  f2r d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2r f2_fma(f2r a, f2r b, f2r c) {   // a b + c, one rounding per lane
  f2r d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ f2r f2_neg(f2r a) { return f2_mul(a, f2_pack(-1.0f, -1.0f)); }
__device__ __forceinline__ f2r f2_swap(f2r a) { return f2_pack(f2_l1(a), f2_l0(a)); }

// a complex float pair, packed
struct pdd {
  f2r hi, lo;
};

__device__ __forceinline__ pdd pdd_of(cpx<dd> v) {
  return pdd{f2_pack(v.x.hi, v.y.hi), f2_pack(v.x.lo, v.y.lo)};
}
__device__ __forceinline__ cpx<dd> cpx_of(pdd v) {
  return mk<dd>(dd(f2_l0(v.hi), f2_l0(v.lo)), dd(f2_l1(v.hi), f2_l1(v.lo)));
}
// a real float pair in both lanes
__device__ __forceinline__ pdd pdd_bc(dd s) { return pdd{f2_pack(s.hi, s.hi), f2_pack(s.lo, s.lo)}; }

// error-free transformations, lane by lane
__device__ __forceinline__ pdd p_fast_two_sum(f2r a, f2r b) {
  const f2r s = f2_add(a, b);
  return pdd{s, f2_sub(b, f2_sub(s, a))};
}
__device__ __forceinline__ pdd p_two_sum(f2r a, f2r b) {
  const f2r s = f2_add(a, b);
  const f2r bb = f2_sub(s, a);
  return pdd{s, f2_add(f2_sub(a, f2_sub(s, bb)), f2_sub(b, bb))};
}
// two_sum(a, -b): s = a - b, bb = s - a, e = (a - (s - bb)) - (b + bb)
__device__ __forceinline__ pdd p_two_diff(f2r a, f2r b) {
  const f2r s = f2_sub(a, b);
  const f2r bb = f2_sub(s, a);
  return pdd{s, f2_sub(f2_sub(a, f2_sub(s, bb)), f2_add(b, bb))};
}

// complex a + b and a - b with the float-pair renormalisation (operator+ / operator- of dd)
__device__ __forceinline__ pdd operator+(pdd a, pdd b) {
  const pdd s = p_two_sum(a.hi, b.hi);
  return p_fast_two_sum(s.hi, f2_add(s.lo, f2_add(a.lo, b.lo)));
}
__device__ __forceinline__ pdd operator-(pdd a, pdd b) {
  const pdd s = p_two_diff(a.hi, b.hi);
  return p_fast_two_sum(s.hi, f2_add(s.lo, f2_sub(a.lo, b.lo)));
}
// the unnormalised sums of cadd_lazy / csub_lazy
__device__ __forceinline__ pdd p_add_lazy(pdd a, pdd b) {
  const pdd s = p_two_sum(a.hi, b.hi);
  return pdd{s.hi, f2_add(s.lo, f2_add(a.lo, b.lo))};
}
__device__ __forceinline__ pdd p_sub_lazy(pdd a, pdd b) {
  const pdd s = p_two_diff(a.hi, b.hi);
  return pdd{s.hi, f2_add(s.lo, f2_sub(a.lo, b.lo))};
}
// v * s for a real float pair s given in both lanes (scal of cpx<dd>)
__device__ __forceinline__ pdd p_scal(pdd v, pdd s) {
  const f2r p = f2_mul(v.hi, s.hi);
  f2r e = f2_fma(v.hi, s.hi, f2_neg(p));
  e = f2_fma(v.hi, s.lo, e);
  e = f2_fma(v.lo, s.hi, e);
  return p_fast_two_sum(p, e);
}
// complex conjugate and the exchange of the two parts
__device__ __forceinline__ pdd p_conj(pdd v) {
  const f2r sg = f2_pack(1.0f, -1.0f);
  return pdd{f2_mul(v.hi, sg), f2_mul(v.lo, sg)};
}
__device__ __forceinline__ pdd p_swap(pdd v) { return pdd{f2_swap(v.hi), f2_swap(v.lo)}; }
// multiply by S i: forward (S < 0) (re, im) -> (im, -re), inverse (-im, re)
template <int S>
__device__ __forceinline__ pdd p_mul_si(pdd v) {
  const f2r sg = (S < 0) ? f2_pack(1.0f, -1.0f) : f2_pack(-1.0f, 1.0f);
  return pdd{f2_mul(f2_swap(v.hi), sg), f2_mul(f2_swap(v.lo), sg)};
}
// Complex product with a twiddle w, as cmul (forward) or cmulc (inverse) of vd_dd.cuh, from
// the table entries wr = (w.re, w.re) and wi = (-w.im, w.im) (forward) or (w.im, -w.im)
// (inverse): lane 0 = a.re w.re + a.im (-+ w.im), lane 1 = a.im w.re + a.re (+- w.im), each a
// dd_sum_prod.  Lane 1 forms the two products in the other order; the exact two_sum of their
// high parts and the commutative sum of their error terms make it the same bits.
__device__ __forceinline__ pdd p_cmul(pdd a, pdd wr, pdd wi) {
  const f2r sh = f2_swap(a.hi), sl = f2_swap(a.lo);
  const f2r p = f2_mul(a.hi, wr.hi);
  f2r e = f2_fma(a.hi, wr.hi, f2_neg(p));
  e = f2_fma(a.hi, wr.lo, e);
  e = f2_fma(a.lo, wr.hi, e);
  const f2r q = f2_mul(sh, wi.hi);
  f2r f = f2_fma(sh, wi.hi, f2_neg(q));
  f = f2_fma(sh, wi.lo, f);
  f = f2_fma(sl, wi.hi, f);
  const pdd s = p_two_sum(p, q);
  return p_fast_two_sum(s.hi, f2_add(s.lo, f2_add(e, f)));
}
// the table entries of twiddle w for direction S
template <int S>
__device__ __forceinline__ void p_tw_entry(cpx<dd> w, pdd* wr, pdd* wi) {
  *wr = pdd{f2_pack(w.x.hi, w.x.hi), f2_pack(w.x.lo, w.x.lo)};
  if (S < 0) *wi = pdd{f2_pack(-w.y.hi, w.y.hi), f2_pack(-w.y.lo, w.y.lo)};
  else *wi = pdd{f2_pack(w.y.hi, -w.y.hi), f2_pack(w.y.lo, -w.y.lo)};
}

// ---------------------------------------------------------------------------------------
// codelets: the float-pair paths of dft2 / dft4 / dft8 (vd_fft.cuh), packed
// ---------------------------------------------------------------------------------------

template <int S>
__device__ __forceinline__ void p_dft2(pdd& a, pdd& b) {
  const pdd t = a - b;
  a = a + b;
  b = t;
}

template <int S, bool LAZY_OUT = false>
__device__ __forceinline__ void p_dft4(pdd* u) {
  const pdd a = p_add_lazy(u[0], u[2]);
  const pdd b = p_sub_lazy(u[0], u[2]);
  const pdd c = p_add_lazy(u[1], u[3]);
  const pdd d = p_mul_si<S>(p_sub_lazy(u[1], u[3]));
  if constexpr (LAZY_OUT) {
    u[0] = p_add_lazy(a, c);
    u[2] = p_sub_lazy(a, c);
    u[1] = p_add_lazy(b, d);
    u[3] = p_sub_lazy(b, d);
    return;
  }
  u[0] = a + c;
  u[2] = a - c;
  u[1] = b + d;
  u[3] = b - d;
}

template <int S>
__device__ __forceinline__ void p_dft8(pdd* u) {
  const pdd r2 = pdd_bc(dd(0.70710678118654752440084436210485));   // 1/sqrt(2)
  pdd e[4] = {u[0], u[2], u[4], u[6]};
  pdd o[4] = {u[1], u[3], u[5], u[7]};
  p_dft4<S, true>(e);
  p_dft4<S, true>(o);
  const pdd o1 = o[1], o3 = o[3];
  o[1] = p_scal(p_add_lazy(o1, p_mul_si<S>(o1)), r2);
  o[3] = p_scal(p_sub_lazy(p_mul_si<S>(o3), o3), r2);
  o[2] = p_mul_si<S>(o[2]);
  u[0] = e[0] + o[0];
  u[4] = e[0] - o[0];
  u[1] = e[1] + o[1];
  u[5] = e[1] - o[1];
  u[2] = e[2] + o[2];
  u[6] = e[2] - o[2];
  u[3] = e[3] + o[3];
  u[7] = e[3] - o[3];
}

template <int S, int R>
__device__ __forceinline__ void p_dftR(pdd* u) {
  if constexpr (R == 2) p_dft2<S>(u[0], u[1]);
  else if constexpr (R == 4) p_dft4<S>(u);
  else p_dft8<S>(u);
}

// The packed engine runs the stage sequence of a power-of-two length with the stage
// parameters as compile-time constants (strides, twiddle steps and butterfly counts become
// immediates): radix-8 stages, then one radix-4 or radix-2 stage for the remaining factor --
// the order of the plans, which p_plan_ok checks.
__host__ __device__ constexpr int p_log2(int n) { return n <= 1 ? 0 : 1 + p_log2(n / 2); }
__host__ __device__ constexpr int p_nst(int n) { return p_log2(n) / 3 + (p_log2(n) % 3 ? 1 : 0); }
__host__ __device__ constexpr int p_rad(int n, int s) {
  return s < p_log2(n) / 3 ? 8 : (p_log2(n) % 3 == 2 ? 4 : 2);
}

// plans the packed engine takes: lengths 64, 128, 256, 512 in the stage order above, with at
// most 8 elements of a line per thread (istep threads share a line)
__host__ __device__ inline bool p_plan_ok(const FftPlan& pl, int istep) {
  if (pl.n != 64 && pl.n != 128 && pl.n != 256 && pl.n != 512) return false;
  if (pl.n > 8 * istep || pl.nst != p_nst(pl.n)) return false;
  for (int s = 0; s < pl.nst; ++s)
    if (pl.rad[s] != p_rad(pl.n, s)) return false;
  return true;
}

// One Stockham stage of the packed engine (stockham_stage of vd_fft.cuh, radix 2 / 4 / 8) for
// a line of N elements with span P; a thread has at most 8 / R butterflies (N <= 8 istep).
// Element stride ES > 0 is a compile-time stride, 0 takes es.
// twr, twi: the twiddle table in the form p_cmul takes for this direction (p_tw_entry).
template <int S, int R, int N, int P, int ES>
__device__ __forceinline__ void p_stage(const pdd* __restrict__ src, pdd* __restrict__ dst, int es_rt, int lofs,
                                        int i0, int istep, const pdd* __restrict__ twr,
                                        const pdd* __restrict__ twi) {
  constexpr int NB = N / R, TWS = N / (P * R), MB = 8 / R;
  const int es = ES > 0 ? ES : es_rt;
#pragma unroll
  for (int b = 0; b < MB; ++b) {
    const int i = i0 + b * istep;
    if (i < NB) {
      const int k = i & (P - 1);
      const pdd* s = src + lofs + i * es;
      pdd u[R];
#pragma unroll
      for (int r = 0; r < R; ++r) u[r] = s[r * NB * es];
      if constexpr (P > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) u[r] = p_cmul(u[r], twr[r * k * TWS], twi[r * k * TWS]);
      }
      p_dftR<S, R>(u);
      pdd* d = dst + lofs + ((i - k) * R + k) * es;
#pragma unroll
      for (int r = 0; r < R; ++r) d[r * P * es] = u[r];
    }
  }
}

template <int S, int N, int ST, int P, int ES>
__device__ __forceinline__ pdd* p_stages(pdd* a, pdd* b, int es, int lofs, int i0, int istep, const pdd* twr,
                                         const pdd* twi) {
  if constexpr (ST < p_nst(N)) {
    constexpr int R = p_rad(N, ST);
    __syncthreads();
    p_stage<S, R, N, P, ES>(a, b, es, lofs, i0, istep, twr, twi);
    return p_stages<S, N, ST + 1, P * R, ES>(b, a, es, lofs, i0, istep, twr, twi);
  } else {
    return a;
  }
}

// full transform of every line of the block (fft_lines), packed, for a plan that p_plan_ok
// accepts; input in a, returns the buffer holding the result.  Must be called by all threads
// of the block (barriers before every stage and at the end).
template <int S, int ES = 0>
__device__ __forceinline__ pdd* p_fft_lines(pdd* a, pdd* b, int es, int lofs, int i0, int istep, const FftPlan& pl,
                                            const pdd* twr, const pdd* twi) {
  pdd* res;
  switch (pl.n) {
    case 64: res = p_stages<S, 64, 0, 1, ES>(a, b, es, lofs, i0, istep, twr, twi); break;
    case 128: res = p_stages<S, 128, 0, 1, ES>(a, b, es, lofs, i0, istep, twr, twi); break;
    case 256: res = p_stages<S, 256, 0, 1, ES>(a, b, es, lofs, i0, istep, twr, twi); break;
    default: res = p_stages<S, 512, 0, 1, ES>(a, b, es, lofs, i0, istep, twr, twi); break;
  }
  __syncthreads();
  return res;
}

}  // namespace vd
