// Transform pass kernels: strided-axis passes (y, z) and the fused contiguous x pass.
#include "vd_passes.cuh"
#include "vd_fft.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>
#include "vd_dd.cuh"
#include "vd_pdd.cuh"
#include "vd_prof.h"

#include <cmath>
#include <type_traits>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>

namespace vd {
static void ensure_smem(const void* func, size_t smem);
static int sm_count();
}

namespace vd {

// Element load / store of a pass.  The float-pair instantiation (T = dd) may read its input
// from, and write its output to, double fields (the Krylov vectors), converting on the fly.
// CV = false compiles the plain path only (programs without any double field): the
// conversion code is then absent instead of merely skipped.
template <typename T, bool CV = true>
__device__ __forceinline__ cpx<T> ld_el(const void* p, int conv, int go) {
  if constexpr (std::is_same<T, dd>::value && CV) {
    if (conv) {
      const cpx<double> v = reinterpret_cast<const cpx<double>*>(p)[go];
      return mk<T>(dd_from_double(v.x), dd_from_double(v.y));
    }
  }
  return reinterpret_cast<const cpx<T>*>(p)[go];
}
template <typename T, bool CV = true>
__device__ __forceinline__ void st_el(void* p, int conv, int go, cpx<T> v, bool first) {
  if constexpr (std::is_same<T, dd>::value && CV) {
    if (conv) {
      cpx<double>* q = reinterpret_cast<cpx<double>*>(p) + go;
      const cpx<double> d = mk<double>(dd_to_double(v.x), dd_to_double(v.y));
      *q = first ? d : (*q + d);
      return;
    }
  }
  cpx<T>* q = reinterpret_cast<cpx<T>*>(p) + go;
  *q = first ? v : (*q + v);
}

// kfac[axis] and a scale factor in the arithmetic type.  Float-pair and float values come
// converted from the host (hi = the double rounded to float), so float kernels issue no
// double -> float conversions: those run on the FP64 pipe, ~1/64 of the float rate on GB300.
template <typename T>
__device__ __forceinline__ T kfac_t(const GridDesc& g, int a) {
  if constexpr (std::is_same<T, dd>::value) return dd(g.kfac_dd[a][0], g.kfac_dd[a][1]);
  else if constexpr (std::is_same<T, float>::value) return g.kfac_f[a];
  else return g.kfac[a];
}
template <typename T>
__device__ __forceinline__ T scale_t(double s, float hi, float lo) {
  if constexpr (std::is_same<T, dd>::value) return dd(hi, lo);
  else if constexpr (std::is_same<T, float>::value) return hi;
  else return s;
}

// z * (wh + wl) rounded once to float: the product with the high part is split exactly by an
// FMA (Dekker's two-product), the low part's product is added to its error term before the
// final rounding
__device__ __forceinline__ float mul_pair(float z, float wh, float wl) {
  const float p = z * wh;
  const float e = fmaf(z, wh, -p);
  return p + fmaf(z, wl, e);
}

// Hint: bring [p, p + bytes) into L2 (p and bytes multiples of 16), in pieces of at most 32 KB.
__device__ __forceinline__ void prefetch_l2(const void* p, unsigned bytes) {
  const size_t ga = __cvta_generic_to_global(p);
  for (unsigned o = 0; o < bytes; o += 32768u) {
    const unsigned len = (bytes - o < 32768u) ? bytes - o : 32768u;
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(ga + o), "r"(len) : "memory");
  }
}

// Hint: bring the 128-byte line holding p into L2.
__device__ __forceinline__ void prefetch_line_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(__cvta_generic_to_global(p)));
}

constexpr int kThreads = 256;
template <typename T>
constexpr int kEPT = (sizeof(T) == 4) ? 16 : 8;   // tile elements per thread (float: 16; double, dd: 8)

static inline int tile_width(int n, int ept) {
  int w = 1;
  while (w < 64 && (2 * w) * n <= ept * kThreads) w *= 2;
  return w;
}
static inline int ilog2(int v) {
  int l = 0;
  while ((1 << (l + 1)) <= v) ++l;
  return l;
}
static inline int lines_per_cta(int m, int ept) {
  int l = 1;
  while (l < 64 && (2 * l) * m <= ept * kThreads / 2) l *= 2;
  return l;
}

// ---------------------------------------------------------------------------------------
// strided axis pass
// ---------------------------------------------------------------------------------------

// PK (float pairs, radices 2 / 4 / 8 only): the shared-memory transform runs on packed
// complex float pairs (vd_pdd.cuh), bit-identical to the unpacked engine; its twiddle table
// holds two entries per twiddle.
template <typename T, int S, bool CV, bool PK = false>
__global__ void __launch_bounds__(kThreads, (std::is_same<T, double>::value ? 2 : (std::is_same<T, dd>::value ? 4 : 3))) k_axis(const AxisProg P, const GridDesc g,
                                                   const cpx<T>* __restrict__ twg, int lw) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (P.done && *P.done) return;
  const int axis = P.axis;
  const FftPlan& pl = (axis == 2) ? g.pz : g.py;
  const int n = pl.n;
  const int W = 1 << lw;
  using E = typename std::conditional<PK, pdd, cpx<T>>::type;
  E* tw = reinterpret_cast<E*>(smem_raw);
  E* tw2 = tw + n;   // PK: the second table
  E* A = tw + (PK ? 2 : 1) * n;
  E* B = A + W * n;
  const int tid = threadIdx.x;
  for (int j = tid; j < n; j += kThreads) {
    if constexpr (PK) p_tw_entry<S>(twg[pl.tw_off + j], &tw[j], &tw2[j]);
    else tw[j] = twg[pl.tw_off + j];
  }

  // field offsets fit in 32 bits (ncplx < 2^31 is checked when the grid is created)
  int line_stride, inner_n, outer_stride;
  if (axis == 2) {
    line_stride = g.n1 * g.h0;
    inner_n = line_stride;
    outer_stride = 0;
  } else {
    line_stride = g.h0;
    inner_n = g.h0;
    outer_stride = g.n1 * g.h0;
  }
  const int tiles = (inner_n + W - 1) >> lw;
  const int o = blockIdx.x / tiles;
  const int col0 = (blockIdx.x - o * tiles) << lw;
  // this thread's line (column) and its first element / butterfly
  const int w = tid & (W - 1);
  const int ib = tid >> lw;
  const int istep = kThreads >> lw;
  const int col = col0 + w;
  const bool colok = col < inner_n;
  const int g0 = o * outer_stride + col + ib * line_stride;   // offset of element ib
  const int gstep = istep * line_stride;                      // offset step between the thread's elements
  const T* __restrict__ symarr = reinterpret_cast<const T*>(P.symarr);
  // |k~|^2 of the axes other than the pass axis (constant for the line)
  T kperp2;
  if (axis == 2) {
    const int kyi = col / g.h0;
    const int kxi = col - kyi * g.h0;
    const T kx = kfac_t<T>(g, 0) * (T)freq_tilde(kxi, g.n0);
    const T ky = kfac_t<T>(g, 1) * (T)freq_tilde(kyi, g.n1);
    kperp2 = kx * kx + ky * ky;
  } else {
    const T kx = kfac_t<T>(g, 0) * (T)freq_tilde(col, g.n0);
    kperp2 = kx * kx;
    if (g.ndim == 3) {
      const T kz = kfac_t<T>(g, 2) * (T)freq_tilde(o, g.n2);
      kperp2 += kz * kz;
    }
  }
  const T kfa = kfac_t<T>(g, axis);
  // real factor of a multiplier at line element i (global offset go)
  auto mult = [&](int flags, int i, int go, T base) -> T {
    const T ka = kfa * (T)freq_tilde(i, n);
    T c = base;
    if (flags & MUL_IK) c *= ka;
    if (flags & MUL_IK2) c *= -ka * ka;
    if (flags & MUL_SYM) c *= symarr[go];
    if (flags & MUL_NEGK2) c *= -(ka * ka + kperp2);
    return c;
  };

  // Each transform writes its result straight to out[dst]; a transform that accumulates
  // (first == 0) reads back the partial sum of the same elements, written earlier by this
  // very thread, so no synchronisation is needed and the partial stays in L2.
  const int nq = (n - ib + istep - 1) / istep;   // elements of this thread in its line
  for (int t = 0; t < P.nxf; ++t) {
    const Xf xf = P.xf[t];
    const void* src = P.in[xf.src];
    void* dst = P.out[xf.dst];
    const int cin = (P.conv_in >> xf.src) & 1, cout = (P.conv_out >> xf.dst) & 1;
    const T scale = scale_t<T>(xf.scale, xf.scale_hi, xf.scale_lo);
    if (xf.nofft) {
      if (colok) {
#pragma unroll 4
        for (int q = 0; q < nq; ++q) {
          const int i = ib + q * istep;
          const int go = g0 + q * gstep;
          cpx<T> v = scal(ld_el<T, CV>(src, cin, go), mult(xf.pre, i, go, scale));
          if (xf.pre & MUL_IK) v = mul_i(v);
          st_el<T, CV>(dst, cout, go, v, xf.first);
        }
      }
      continue;
    }
    __syncthreads();
#pragma unroll 4
    for (int q = 0; q < nq; ++q) {
      const int i = ib + q * istep;
      const int go = g0 + q * gstep;
      cpx<T> v = mk<T>(T(0), T(0));
      if (colok) v = ld_el<T, CV>(src, cin, go);
      if (xf.pre) {
        v = scal(v, mult(xf.pre, i, go, T(1)));
        if (xf.pre & MUL_IK) v = mul_i(v);
      }
      if constexpr (PK) A[i * W + w] = pdd_of(v);
      else A[i * W + w] = v;
    }
    // PK: the rows of the next transform's input tile are prefetched into L2 (one thread per
    // row: a row of the tile is W elements of 16 bytes) while this one is transformed
    if constexpr (PK) {
      if (w == 0 && t + 1 < P.nxf && !P.xf[t + 1].nofft) {
        const cpx<T>* nsrc = reinterpret_cast<const cpx<T>*>(P.in[P.xf[t + 1].src]);   // 16-byte elements
        for (int q = 0; q < nq; ++q) prefetch_line_l2(nsrc + g0 + q * gstep);
      }
    }
    E* res;
    if constexpr (PK) res = p_fft_lines<S>(A, B, W, w, ib, istep, pl, tw, tw2);
    else res = fft_lines<T, S>(A, B, W, w, ib, istep, pl, tw);
    if (colok) {
#pragma unroll 4
      for (int q = 0; q < nq; ++q) {
        const int i = ib + q * istep;
        const int go = g0 + q * gstep;
        cpx<T> v;
        if constexpr (PK) v = cpx_of(res[i * W + w]);
        else v = res[i * W + w];
        if (xf.post) {
          v = scal(v, mult(xf.post, i, go, scale));
          if (xf.post & MUL_IK) v = mul_i(v);
        } else {
          v = scal(v, scale);
        }
        st_el<T, CV>(dst, cout, go, v, xf.first);
      }
    }
  }
}

// ---------------------------------------------------------------------------------------
// strided axis pass, register-resident four-step transform for n = N1 * N2 (N1 = C * N2)
//
// With n = N2 n1 + n2 and k = k1 + N1 k2:
//   X[k1 + N1 k2] = sum_{n2} W_{N2}^{n2 k2} W_n^{n2 k1} sum_{n1} x[N2 n1 + n2] W_{N1}^{n1 k1}.
// Thread n2 of a line holds x[N2 n1 + n2] (the rows it loads), transforms over n1 in
// registers, multiplies by W_n^{n2 k1}, and one shared-memory transpose hands column k1 to
// thread k1 mod N2, which transforms over n2 and stores rows k1 + N1 k2.  16 lines (columns)
// per block, line stride n + 1 in shared memory (conflict-free transposes).  Length 256 runs
// three blocks per SM (80 registers, a few hundred bytes of spills held in L1): measured
// faster than two (128 registers) and four (64 registers, spills reaching L2).
// ---------------------------------------------------------------------------------------

constexpr int kRLines = 16;
constexpr int kTmaMaxIn = 4;   // inputs a TMA-staged program may read
constexpr int kPairCols = 18;  // columns of a y-pass box (16 + 2: a 16-byte aligned start for odd rows)

// The common multipliers (none, or i k~ along the axis) with a scale of one, in loops of their
// own, so that the flag tests and the wavenumber arithmetic of the general case stay out of the
// unrolled element loops.  katab[i] = k~ of index i along the axis, the same float product the
// general case forms; x * 1 is exact, so both paths give the same bits.
template <typename T, int N1, int N2>
__device__ __forceinline__ void pre_ik(cpx<T>* u, int t, const T* katab) {
#pragma unroll
  for (int j = 0; j < N1; ++j) u[j] = mul_i(scal(u[j], katab[N2 * j + t]));
}

// row k1 + N1 k2 of a line <- v[k2] (times i k~ if IK), added to what the row holds unless FIRST
// (partial sums read in batches of 4 before their stores, so that their latencies overlap)
template <typename T, int N1, int N2, bool IK, bool FIRST>
__device__ __forceinline__ void store_rows(cpx<T>* __restrict__ q, int gbase, int ls, int k1, const cpx<T>* v,
                                           const T* katab) {
  constexpr int PB = N2 < 4 ? N2 : 4;
#pragma unroll
  for (int k0 = 0; k0 < N2; k0 += PB) {
    cpx<T> prev[PB];
    if constexpr (!FIRST) {
#pragma unroll
      for (int b = 0; b < PB; ++b) prev[b] = q[gbase + (k1 + N1 * (k0 + b)) * ls];
    }
#pragma unroll
    for (int b = 0; b < PB; ++b) {
      const int i = k1 + N1 * (k0 + b);
      cpx<T> vv = v[k0 + b];
      if constexpr (IK) vv = mul_i(scal(vv, katab[i]));
      if constexpr (FIRST) q[gbase + i * ls] = vv;
      else q[gbase + i * ls] = prev[b] + vv;
    }
  }
}

// the store of one output line: the common cases, or false for the general one
template <typename T, int N1, int N2>
__device__ __forceinline__ bool store_rows_common(const Xf& xf, T scale, cpx<T>* q, int gbase, int ls, int k1,
                                                  const cpx<T>* v, const T* katab) {
  if (scale != T(1) || (xf.post != 0 && xf.post != MUL_IK)) return false;
  if (xf.post == 0) {
    if (xf.first) store_rows<T, N1, N2, false, true>(q, gbase, ls, k1, v, katab);
    else store_rows<T, N1, N2, false, false>(q, gbase, ls, k1, v, katab);
  } else {
    if (xf.first) store_rows<T, N1, N2, true, true>(q, gbase, ls, k1, v, katab);
    else store_rows<T, N1, N2, true, false>(q, gbase, ls, k1, v, katab);
  }
  return true;
}

// Twiddles W_m^{t k1} (k1 in [1, M1)) of one thread's first four-step layer.  Float: as the
// product W_m^{4 t a} W_m^{t b} (k1 = 4 a + b) of six values read once per kernel (one float
// complex product, within ~1.5 ulp of the table), so that the x pass does not read a twiddle
// from shared memory per element; other types: the table.
template <typename T, int M1>
struct StepTw {
  const cpx<T>* tw;
  int t;
  __device__ __forceinline__ StepTw(const cpx<T>* tab, int tt) : tw(tab), t(tt) {}
  __device__ __forceinline__ cpx<T> operator()(int k1) const { return tw[t * k1]; }
};
template <int M1>
struct StepTw<float, M1> {
  cpx<float> a[M1 / 4], b[4];   // a[i] = W^{4 t i}, b[i] = W^{t i}
  __device__ __forceinline__ StepTw(const cpx<float>* tab, int t) {
#pragma unroll
    for (int i = 0; i < 4; ++i) b[i] = tab[t * i];
#pragma unroll
    for (int i = 0; i < M1 / 4; ++i) a[i] = tab[4 * t * i];
  }
  __device__ __forceinline__ cpx<float> operator()(int k1) const {
    const int i = k1 >> 2, j = k1 & 3;
    if (i == 0) return b[j];
    if (j == 0) return a[i];
    return cmul(a[i], b[j]);
  }
};

template <typename T, int S, int N1, int N2>
__global__ void __launch_bounds__(kRLines * N2, (N2 == 16 ? 3 : 2)) k_axis_r(const AxisProg P, const GridDesc g,
                                                        const cpx<T>* __restrict__ twg) {
  static_assert(std::is_same<T, float>::value, "register four-step pass: float storage only");
  constexpr int N = N1 * N2;
  constexpr int C = N1 / N2;
  constexpr int LS = N + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (P.done && *P.done) return;
  const int axis = P.axis;
  const FftPlan& pl = (axis == 2) ? g.pz : g.py;
  cpx<T>* tw = reinterpret_cast<cpx<T>*>(smem_raw);
  cpx<T>* Y = tw + N;
  T* katab = reinterpret_cast<T*>(Y + kRLines * LS);   // k~ of every index along the axis
  const int tid = threadIdx.x;
  const T kfa = kfac_t<T>(g, axis);
  for (int j = tid; j < N; j += kRLines * N2) {
    tw[j] = twg[pl.tw_off + j];
    katab[j] = kfa * (T)freq_tilde(j, N);
  }
  __syncthreads();   // the tables are read by every thread before the first transpose

  // lines: z pass, the columns of the flattened (y, x) plane; y pass, the x columns of each z
  // plane (tiles of 16 columns, the last one of a plane ragged: numbering the lines across
  // plane boundaries instead, so that no tile is ragged, measured slower)
  int line_stride, inner_n, outer_stride;
  if (axis == 2) {
    line_stride = g.n1 * g.h0;
    inner_n = line_stride;
    outer_stride = 0;
  } else {
    line_stride = g.h0;
    inner_n = g.h0;
    outer_stride = g.n1 * g.h0;
  }
  const int tiles = (inner_n + kRLines - 1) / kRLines;
  const int o = blockIdx.x / tiles;
  const int col0 = (blockIdx.x - o * tiles) * kRLines;
  const int w = tid % kRLines;
  const int t = tid / kRLines;   // n2 in the first step
  const int col = col0 + w;
  const bool colok = col < inner_n;
  const int gbase = o * outer_stride + col;
  const T* __restrict__ symarr = reinterpret_cast<const T*>(P.symarr);
  T kperp2;
  if (axis == 2) {
    const int kyi = col / g.h0;
    const int kxi = col - kyi * g.h0;
    const T kx = kfac_t<T>(g, 0) * (T)freq_tilde(kxi, g.n0);
    const T ky = kfac_t<T>(g, 1) * (T)freq_tilde(kyi, g.n1);
    kperp2 = kx * kx + ky * ky;
  } else {
    const T kx = kfac_t<T>(g, 0) * (T)freq_tilde(col, g.n0);
    kperp2 = kx * kx;
    if (g.ndim == 3) {
      const T kz = kfac_t<T>(g, 2) * (T)freq_tilde(o, g.n2);
      kperp2 += kz * kz;
    }
  }
  auto mult = [&](int flags, int i, int go, T base) -> T {
    const T ka = kfa * (T)freq_tilde(i, N);
    T c = base;
    if (flags & MUL_IK) c *= ka;
    if (flags & MUL_IK2) c *= -ka * ka;
    if (flags & MUL_SYM) c *= symarr[go];
    if (flags & MUL_NEGK2) c *= -(ka * ka + kperp2);
    return c;
  };
  cpx<T>* Yl = Y + w * LS;

  for (int x = 0; x < P.nxf; ++x) {
    const Xf xf = P.xf[x];
    const void* src = P.in[xf.src];
    void* dst = P.out[xf.dst];
    const int cin = (P.conv_in >> xf.src) & 1, cout = (P.conv_out >> xf.dst) & 1;
    const T scale = scale_t<T>(xf.scale, xf.scale_hi, xf.scale_lo);
    if (xf.nofft) {
      if (colok) {
#pragma unroll
        for (int j = 0; j < N1; ++j) {
          const int i = N2 * j + t;
          const int go = gbase + i * line_stride;
          cpx<T> v = scal(ld_el<T>(src, cin, go), mult(xf.pre, i, go, scale));
          if (xf.pre & MUL_IK) v = mul_i(v);
          st_el<T>(dst, cout, go, v, xf.first);
        }
      }
      continue;
    }
    cpx<T> u[N1];
#pragma unroll
    for (int j = 0; j < N1; ++j) {
      const int i = N2 * j + t;
      u[j] = colok ? ld_el<T>(src, cin, gbase + i * line_stride) : mk<T>(T(0), T(0));
    }
    if (xf.pre == MUL_IK) {
      pre_ik<T, N1, N2>(u, t, katab);
    } else if (xf.pre && colok) {   // (lines past the end read no symbol)
#pragma unroll
      for (int j = 0; j < N1; ++j) {
        const int i = N2 * j + t;
        u[j] = scal(u[j], mult(xf.pre, i, gbase + i * line_stride, T(1)));
        if (xf.pre & MUL_IK) u[j] = mul_i(u[j]);
      }
    }
    dftR<T, S, N1>(u);
#pragma unroll
    for (int k1 = 1; k1 < N1; ++k1) {
      const cpx<T> wv = tw[t * k1];
      u[k1] = (S < 0) ? cmul(u[k1], wv) : cmulc(u[k1], wv);
    }
    __syncthreads();   // the previous transform has finished reading Y
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) Yl[t * N1 + k1] = u[k1];
    __syncthreads();
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const int k1 = t + N2 * c;
      cpx<T> v[N2];
#pragma unroll
      for (int n2 = 0; n2 < N2; ++n2) v[n2] = Yl[n2 * N1 + k1];
      dftR<T, S, N2>(v);
      if (colok && !store_rows_common<T, N1, N2>(xf, scale, reinterpret_cast<cpx<T>*>(dst), gbase, line_stride, k1,
                                                  v, katab)) {
        // a transform that accumulates reads all of its partial sums before its first store,
        // so their latencies overlap (the compiler cannot move a load of dst above a store to
        // dst); the partials were written by this thread, so the order is unchanged
        cpx<T>* q = reinterpret_cast<cpx<T>*>(dst);
        constexpr int PB = N2 < 4 ? N2 : 4;   // partial sums read in batches of PB (fewer spills than 8)
#pragma unroll
        for (int k0 = 0; k0 < N2; k0 += PB) {
          cpx<T> prev[PB];
          if (!xf.first) {
#pragma unroll
            for (int b = 0; b < PB; ++b) prev[b] = q[gbase + (k1 + N1 * (k0 + b)) * line_stride];
          }
#pragma unroll
          for (int b = 0; b < PB; ++b) {
            const int i = k1 + N1 * (k0 + b);
            const int go = gbase + i * line_stride;
            cpx<T> vv = v[k0 + b];
            if (xf.post) {
              vv = scal(vv, mult(xf.post, i, go, scale));
              if (xf.post & MUL_IK) vv = mul_i(vv);
            } else {
              vv = scal(vv, scale);
            }
            q[go] = xf.first ? vv : (prev[b] + vv);
          }
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------------------
// y and z passes, register four-step transform with TMA-staged input (float, n = 128 / 256)
//
// The same arithmetic as k_axis_r, in a persistent grid: each block walks its tiles (16
// adjacent columns, i.e. 16 lines) and, for every tile, the transforms of the program.  The
// input of the next (tile, transform) item is fetched by the tensor memory accelerator
// (cp.async.bulk.tensor, one box of N rows x 128 bytes) into a shared-memory buffer while the
// current item is transformed and stored, so loads stay in flight without registers.
// A z tile is a box of the field viewed as a 2D tensor [n2][2 n1 h0] of floats: its rows
// (z planes) are n1 h0 8 bytes apart, a multiple of 16 for even n1.  A y row is 8 h0 bytes, not
// a multiple of 16 when h0 is odd (n0 a multiple of 4), so a y tile is fetched as two boxes of
// the plane viewed as n1/2 "pair rows" (y rows 2r and 2r+1 back to back, 16 h0 bytes): the even
// rows from the pair row's column col0, the odd rows from column h0 + col0 - 1 (one column early
// when h0 is odd, so that the box starts on a 16-byte boundary; 18 columns wide).  A tile starts
// at a multiple of 128 bytes.  Columns past the end of a row or plane arrive as zeros (box fill)
// or belong to the neighbouring row; they are neither transformed into anything stored nor
// written.
// Every wait on the transfer barrier is bounded; a block that gives up raises the grid's error
// word (reported by the solve as VD_ERR_TIMEOUT), waits (bounded) for its own transfer in
// flight and returns.
// ---------------------------------------------------------------------------------------

struct TmaMaps {
  CUtensorMap m[kTmaMaxIn];
};

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait for the phase `parity` of the barrier; false if it did not complete
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity) {
  for (int i = 0; i < (1 << 22); ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
          smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
      : "memory");
}

template <int S, int N1, int N2, int AX>
__global__ void __launch_bounds__(kRLines * N2, (N2 == 16 ? 3 : 6))
    k_axis_tma(const AxisProg P, const GridDesc g, const cpx<float>* __restrict__ twg, const __grid_constant__ TmaMaps maps) {
  using T = float;
  constexpr int N = N1 * N2;
  constexpr int C = N1 / N2;
  constexpr int LS = N + 1;
  constexpr int NT = kRLines * N2;
  // staged tile: z pass, one box of N rows x 16 columns; y pass, two boxes of N/2 pair rows x 18
  // columns (even and odd y rows, see below)
  constexpr unsigned kBoxBytes = (unsigned)(N * (AX == 2 ? kRLines : kPairCols) * sizeof(cpx<T>));
  extern __shared__ __align__(1024) unsigned char smem_tma[];
  unsigned char* smem_raw = smem_tma;
  if (P.done && *P.done) return;
  constexpr int axis = AX;   // 1 = y, 2 = z (compiled apart: the z form keeps its register budget)
  const FftPlan& pl = (axis == 2) ? g.pz : g.py;
  cpx<T>* buf = reinterpret_cast<cpx<T>*>(smem_raw);                       // the staged tile
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + kBoxBytes);
  cpx<T>* tw = reinterpret_cast<cpx<T>*>(smem_raw + kBoxBytes + 16);
  cpx<T>* Y = tw + N;
  T* katab = reinterpret_cast<T*>(Y + kRLines * LS);   // k~ of every index along the axis
  const int tid = threadIdx.x;
  const T kfa = kfac_t<T>(g, axis);
  for (int j = tid; j < N; j += NT) {
    tw[j] = twg[pl.tw_off + j];
    katab[j] = kfa * (T)freq_tilde(j, N);
  }
  if (tid == 0) mbar_init(bar, 1);
  __syncthreads();

  // z pass: lines are the columns of the flattened (y, x) plane (one "plane" of tiles);
  // y pass: lines are the x columns of each z plane o
  const int line_stride = (axis == 2) ? g.n1 * g.h0 : g.h0;
  const int inner_n = line_stride;
  const int outer_stride = (axis == 2) ? 0 : g.n1 * g.h0;
  const int tpp = (inner_n + kRLines - 1) / kRLines;   // tiles per plane
  const int tiles = tpp * ((axis == 2) ? 1 : g.n2);
  const int w = tid % kRLines;
  const int t = tid / kRLines;
  const int nx = P.nxf;
  // items of this block: (tile, transform), tiles blockIdx.x, blockIdx.x + gridDim.x, ...
  const int my_tiles = (blockIdx.x < tiles) ? (tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const int nitems = my_tiles * nx;
  if (nitems == 0) return;
  auto issue = [&](int item) {
    const int tile = (int)blockIdx.x + (item / nx) * (int)gridDim.x;
    const int x = item % nx;
    const int o = tile / tpp;
    const int col0 = (tile - o * tpp) * kRLines;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(bar, kBoxBytes);
    if (axis == 2) {
      tma_load_2d(buf, &maps.m[P.xf[x].src], 2 * col0, 0, bar);
    } else {
      // even y rows: columns col0.. of the first half of each pair row; odd y rows: from column
      // h0 - (h0 & 1) + col0 of the pair row, one column early when h0 is odd (16-byte start)
      tma_load_3d(buf, &maps.m[P.xf[x].src], 2 * col0, 0, o, bar);
      tma_load_3d(buf + (N / 2) * kPairCols, &maps.m[P.xf[x].src], 2 * (g.h0 - (g.h0 & 1) + col0), 0, o, bar);
    }
  };
  if (tid == 0) issue(0);
  const T* __restrict__ symarr = reinterpret_cast<const T*>(P.symarr);
  cpx<T>* Yl = Y + w * LS;
  // y pass: this thread's rows all have the parity of t (N2 is even): even rows in the first
  // box, odd rows in the second, whose column 0 is the row's column -1 when h0 is odd
  const cpx<T>* ybase = (t & 1) ? buf + (N / 2) * kPairCols + (g.h0 & 1) : buf;

  for (int it = 0; it < nitems; ++it) {
    const int tile = (int)blockIdx.x + (it / nx) * (int)gridDim.x;
    const Xf xf = P.xf[it % nx];
    const int o = tile / tpp;
    const int col = (tile - o * tpp) * kRLines + w;
    const bool colok = col < inner_n;
    const int gbase = o * outer_stride + col;
    T kperp2 = T(0);   // the perpendicular |k~|^2 of this line, for the multipliers that need it
    if ((xf.pre | xf.post) & MUL_NEGK2) {
      if (axis == 2) {
        const int kyi = col / g.h0;
        const int kxi = col - kyi * g.h0;
        const T kx = kfac_t<T>(g, 0) * (T)freq_tilde(kxi, g.n0);
        const T ky = kfac_t<T>(g, 1) * (T)freq_tilde(kyi, g.n1);
        kperp2 = kx * kx + ky * ky;
      } else {
        const T kx = kfac_t<T>(g, 0) * (T)freq_tilde(col, g.n0);
        kperp2 = kx * kx;
        if (g.ndim == 3) {
          const T kz = kfac_t<T>(g, 2) * (T)freq_tilde(o, g.n2);
          kperp2 += kz * kz;
        }
      }
    }
    auto mult = [&](int flags, int i, int go, T base) -> T {
      const T ka = kfa * (T)freq_tilde(i, N);
      T c = base;
      if (flags & MUL_IK) c *= ka;
      if (flags & MUL_IK2) c *= -ka * ka;
      if (flags & MUL_SYM) c *= symarr[go];
      if (flags & MUL_NEGK2) c *= -(ka * ka + kperp2);
      return c;
    };
    const bool ok = mbar_wait_bounded(bar, (unsigned)(it & 1));
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        if (g.dev_err) atomicExch(g.dev_err, 1);
        mbar_wait_bounded(bar, (unsigned)(it & 1));   // the transfer in flight, if it ever lands
      }
      __syncthreads();
      return;
    }
    void* dst = P.out[xf.dst];
    const T scale = scale_t<T>(xf.scale, xf.scale_hi, xf.scale_lo);
    cpx<T> u[N1];
#pragma unroll
    for (int j = 0; j < N1; ++j) {
      const int i = N2 * j + t;
      u[j] = (AX == 2) ? buf[i * kRLines + w] : ybase[(i >> 1) * kPairCols + w];
    }
    if (xf.pre == MUL_IK) {
      pre_ik<T, N1, N2>(u, t, katab);
    } else if (xf.pre && colok) {   // (columns past the end read no symbol)
#pragma unroll
      for (int j = 0; j < N1; ++j) {
        const int i = N2 * j + t;
        u[j] = scal(u[j], mult(xf.pre, i, gbase + i * line_stride, T(1)));
        if (xf.pre & MUL_IK) u[j] = mul_i(u[j]);
      }
    }
    // every thread has read the staged tile, and the previous item's transpose reads are done:
    // the buffer takes the next item's input while this one is transformed and stored
    __syncthreads();
    if (tid == 0 && it + 1 < nitems) issue(it + 1);
    dftR<T, S, N1>(u);
#pragma unroll
    for (int k1 = 1; k1 < N1; ++k1) {
      const cpx<T> wv = tw[t * k1];
      u[k1] = (S < 0) ? cmul(u[k1], wv) : cmulc(u[k1], wv);
    }
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) Yl[t * N1 + k1] = u[k1];
    __syncthreads();
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const int k1 = t + N2 * c;
      cpx<T> v[N2];
#pragma unroll
      for (int n2 = 0; n2 < N2; ++n2) v[n2] = Yl[n2 * N1 + k1];
      dftR<T, S, N2>(v);
      if (colok && !store_rows_common<T, N1, N2>(xf, scale, reinterpret_cast<cpx<T>*>(dst), gbase, line_stride, k1,
                                                  v, katab)) {
        cpx<T>* q = reinterpret_cast<cpx<T>*>(dst);
        constexpr int PB = N2 < 4 ? N2 : 4;
#pragma unroll
        for (int k0 = 0; k0 < N2; k0 += PB) {
          cpx<T> prev[PB];
          if (!xf.first) {
#pragma unroll
            for (int b = 0; b < PB; ++b) prev[b] = q[gbase + (k1 + N1 * (k0 + b)) * line_stride];
          }
#pragma unroll
          for (int b = 0; b < PB; ++b) {
            const int i = k1 + N1 * (k0 + b);
            const int go = gbase + i * line_stride;
            cpx<T> vv = v[k0 + b];
            if (xf.post) {
              vv = scal(vv, mult(xf.post, i, go, scale));
              if (xf.post & MUL_IK) vv = mul_i(vv);
            } else {
              vv = scal(vv, scale);
            }
            q[go] = xf.first ? vv : (prev[b] + vv);
          }
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------------------
// contiguous x pass (real <-> half spectrum through a complex FFT of length n0/2)
// ---------------------------------------------------------------------------------------

// float pairs: MINB blocks per SM, 3 (80 registers, no spills) where shared memory admits no
// more (16 lines per block take 70-77 KB), 4 (64 registers) for smaller blocks.
// PK (float pairs, radices 2 / 4 / 8 only): the transforms and the (un)packing of the real
// transform run on packed complex float pairs (vd_pdd.cuh), bit-identical to the unpacked
// code, with packed twiddle tables for both directions and the packing twiddles W_{n0}^k.
template <typename T, bool CV, bool PK = false, int MINB = (std::is_same<T, dd>::value ? 3 : 1)>
__global__ void __launch_bounds__(kThreads, MINB) k_xpass(const XProg P, const GridDesc g,
                                                    const cpx<T>* __restrict__ twg, int llpc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (P.done && *P.done) return;
  const int m = g.n0 / 2;
  const int h0 = g.h0;
  const int ls = m + 1;
  const int LPC = 1 << llpc;
  using E = typename std::conditional<PK, pdd, cpx<T>>::type;
  // unpacked: W_m^j (m), W_{n0}^k (m + 1, padded to m + 2: 16-byte alignment), two line buffers
  // PK: wr, wi forward, wi inverse of W_m^j (m each), wr, wi forward of W_{n0}^k (m + 1 each),
  // two line buffers
  cpx<T>* twm = reinterpret_cast<cpx<T>*>(smem_raw);
  cpx<T>* pk = twm + m;
  E* twx = reinterpret_cast<E*>(smem_raw);
  E* pkx = twx + 3 * m;
  E* A = PK ? pkx + 2 * (m + 1) : reinterpret_cast<E*>(pk + (m + 2));
  E* B = A + LPC * ls;
  const int tid = threadIdx.x;
  for (int j = tid; j < m; j += kThreads) {
    if constexpr (PK) {
      const cpx<T> w = twg[g.px.tw_off + j];
      p_tw_entry<-1>(w, &twx[j], &twx[m + j]);
      pdd wr;
      p_tw_entry<+1>(w, &wr, &twx[2 * m + j]);
    } else {
      twm[j] = twg[g.px.tw_off + j];
    }
  }
  for (int j = tid; j <= m; j += kThreads) {
    if constexpr (PK) p_tw_entry<-1>(twg[g.pk_off + j], &pkx[j], &pkx[m + 1 + j]);
    else pk[j] = twg[g.pk_off + j];
  }

  const long long nlines = (long long)g.n1 * g.n2;
  const long long line0 = (long long)blockIdx.x * LPC;
  const int nl = (int)min((long long)LPC, nlines - line0);
  // this thread's line and its position in the line
  const int ltpl = 8 - llpc;   // log2(threads per line), kThreads = 256
  const int TPL = 1 << ltpl;
  const int line = tid >> ltpl;
  const int t0 = tid & (TPL - 1);
  const bool lok = line < nl;
  const int lofs = line * ls;
  const T kfx = kfac_t<T>(g, 0);
  const T scale = scale_t<T>(P.scale, P.scale_hi, P.scale_lo);
  const T* __restrict__ symarr = reinterpret_cast<const T*>(P.symarr) + (line0 + line) * h0;
  // float pairs: the block's lines of a component are one contiguous chunk (16 bytes per
  // element, float pairs and doubles alike); the weights and each next component's input are
  // prefetched into L2 while the current component is transformed
  constexpr bool kPrefetch = std::is_same<T, dd>::value;
  if (kPrefetch && tid == 0 && P.mode == 0 && P.wfield)
    prefetch_l2(reinterpret_cast<const cpx<T>*>(P.wfield) + line0 * m, (unsigned)(nl * m) * 16u);
  // the transforms and element conversions of the engine in use
  auto fft_fwd = [&](E* a, E* b) -> E* {
    if constexpr (PK) return p_fft_lines<-1, 1>(a, b, 1, lofs, t0, TPL, g.px, twx, twx + m);
    else return fft_lines<T, -1>(a, b, 1, lofs, t0, TPL, g.px, twm);
  };
  auto fft_inv = [&](E* a, E* b) -> E* {
    if constexpr (PK) return p_fft_lines<+1, 1>(a, b, 1, lofs, t0, TPL, g.px, twx, twx + 2 * m);
    else return fft_lines<T, +1>(a, b, 1, lofs, t0, TPL, g.px, twm);
  };
  auto to_e = [](cpx<T> v) -> E {
    if constexpr (PK) return pdd_of(v);
    else return v;
  };

  // c = -1: the inverse-only transform of component 0 into aux_out (mode 0 programs only)
  for (int c = P.aux_out ? -1 : 0; c < P.ncomp; ++c) {
    const bool aux = c < 0;
    const int ci = aux ? 0 : c;
    const int mode = aux ? 2 : P.mode;
    E* res;
    __syncthreads();
    if (kPrefetch && tid == 0 && c + 1 < P.ncomp) {
      const int per = (P.mode == 1) ? m : h0;   // elements per line of the next input
      prefetch_l2(reinterpret_cast<const cpx<T>*>(P.in[c + 1]) + line0 * per, (unsigned)(nl * per) * 16u);
    }
    if (mode == 1) {
      const int cin = (P.conv_in >> c) & 1;
      const int rbase = (int)((line0 + line) * m);
      if (lok) {
#pragma unroll 4
        for (int j = t0; j < m; j += TPL) A[lofs + j] = to_e(ld_el<T, CV>(P.in[c], cin, rbase + j));
      }
      res = fft_fwd(A, B);
    } else {
      const int cin = (P.conv_in >> ci) & 1;
      const int lbase = (int)((line0 + line) * h0);
      const int pre = aux ? 0 : P.pre[ci];
      if (lok) {
#pragma unroll 4
        for (int k = t0; k < h0; k += TPL) {
          cpx<T> v = ld_el<T, CV>(P.in[ci], cin, lbase + k);
          if (pre) {
            const T kx = kfx * (T)freq_tilde(k, g.n0);
            T cc = T(1);
            if (pre & MUL_IK) cc *= kx;
            if (pre & MUL_SYM) cc *= symarr[k];
            if (pre & (MUL_NEGK2 | MUL_IK2)) cc *= -kx * kx;
            v = scal(v, cc);
            if (pre & MUL_IK) v = mul_i(v);
          }
          B[lofs + k] = to_e(v);
        }
      }
      __syncthreads();
      // pack the half spectrum into a length-m complex spectrum (inverse real transform)
      if (lok) {
        for (int k = t0; k < m; k += TPL) {
          if constexpr (PK) {
            // (X + conj Xr) + i cmulc(X - conj Xr, w), with cmulc(t, w) = conj cmul(conj t, w)
            // bit for bit, conj t = conj X - Xr and i conj C = (C.im, C.re)
            const pdd X = B[lofs + k], Xr = B[lofs + (m - k)];
            const pdd C = p_cmul(p_conj(X) - Xr, pkx[k], pkx[m + 1 + k]);
            A[lofs + k] = (X + p_conj(Xr)) + p_swap(C);
          } else {
            const cpx<T> X = B[lofs + k];
            const cpx<T> Xc = conjg(B[lofs + (m - k)]);
            A[lofs + k] = (X + Xc) + mul_i(cmulc(X - Xc, pk[k]));
          }
        }
      }
      res = fft_inv(A, B);
      if (mode == 2) {
        void* o = aux ? P.aux_out : P.out[c];
        const int cout = aux ? P.aux_conv : ((P.conv_out >> c) & 1);
        const T sc = aux ? scale_t<T>(P.aux_scale, P.aux_scale_hi, P.aux_scale_lo) : scale;
        const int rbase = (int)((line0 + line) * m);
        if (lok)
          for (int j = t0; j < m; j += TPL) {
            if constexpr (PK) st_el<T, CV>(o, cout, rbase + j, cpx_of(p_scal(res[lofs + j], pdd_bc(sc))), true);
            else st_el<T, CV>(o, cout, rbase + j, scal(res[lofs + j], sc), true);
          }
        continue;
      }
      if (P.wfield && lok) {
        bool done_pair = false;
        if constexpr (PK) {
          // lane by lane the float-pair products z.x wv.x and z.y wv.y
          const cpx<T>* __restrict__ wf = reinterpret_cast<const cpx<T>*>(P.wfield) + (line0 + line) * m;
#pragma unroll 4
          for (int j = t0; j < m; j += TPL) res[lofs + j] = p_scal(res[lofs + j], pdd_of(wf[j]));
          done_pair = true;
        } else if constexpr (std::is_same<T, float>::value) {
          if (P.wf_dd) {
            const float4* __restrict__ wf4 = reinterpret_cast<const float4*>(P.wfield) + (line0 + line) * m;
#pragma unroll 4
            for (int j = t0; j < m; j += TPL) {
              const cpx<T> z = res[lofs + j];
              const float4 w = wf4[j];
              res[lofs + j] = mk<T>(mul_pair(z.x, w.x, w.y), mul_pair(z.y, w.z, w.w));
            }
            done_pair = true;
          }
        }
        if constexpr (!PK) {
          if (!done_pair) {
            const cpx<T>* __restrict__ wf = reinterpret_cast<const cpx<T>*>(P.wfield) + (line0 + line) * m;
#pragma unroll 4
            for (int j = t0; j < m; j += TPL) {
              const cpx<T> z = res[lofs + j];
              const cpx<T> wv = wf[j];
              res[lofs + j] = mk<T>(z.x * wv.x, z.y * wv.y);
            }
          }
        }
      }
      E* other = (res == A) ? B : A;
      res = fft_fwd(res, other);
    }
    // unpack the length-m spectrum into the half spectrum of the real line
    const int cout = (P.conv_out >> c) & 1;
    const int obase = (int)((line0 + line) * h0);
    const int post = P.post[c];
    if (lok) {
      for (int k = t0; k < h0; k += TPL) {
        T cc = scale;
        const T kx = kfx * (T)freq_tilde(k, g.n0);
        if (post & MUL_IK) cc *= kx;
        if (post & MUL_SYM) cc *= symarr[k];
        if (post & (MUL_NEGK2 | MUL_IK2)) cc *= -kx * kx;
        if constexpr (PK) {
          // (Z + Zc) - i cmul(Z - Zc, w), Zc = conj of the mirrored entry
          const pdd Z = res[lofs + (k == m ? 0 : k)];
          const pdd Zc = p_conj(res[lofs + (k == 0 ? 0 : m - k)]);
          const pdd C = p_cmul(Z - Zc, pkx[k], pkx[m + 1 + k]);
          pdd X = p_scal((Z + Zc) - p_mul_si<+1>(C), pdd_bc(cc));
          if (post & MUL_IK) X = p_mul_si<+1>(X);
          st_el<T, CV>(P.out[c], cout, obase + k, cpx_of(X), true);
        } else {
          const cpx<T> Z = res[lofs + (k == m ? 0 : k)];
          const cpx<T> Zc = conjg(res[lofs + (k == 0 ? 0 : m - k)]);
          cpx<T> X = (Z + Zc) - mul_i(cmul(Z - Zc, pk[k]));
          X = scal(X, cc);
          if (post & MUL_IK) X = mul_i(X);
          st_el<T, CV>(P.out[c], cout, obase + k, X, true);
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------------------
// contiguous x pass, register-resident four-step transforms (m = n0/2 = M1 * M2, M1 = C M2)
//
// Each line is handled by M2 threads; thread t holds z[M2 q + t], q in [0, M1) (the
// four-step input distribution).  A four-step transform leaves thread t with outputs
// k1 + M1 k2 for k1 = t + M2 c, which is z[M2 (c + C k2) + t] -- the same distribution -- so
// the inverse transform, the multiply by the weights and the forward transform chain in
// registers.  Shared memory holds one line buffer per line: the spectral line for the
// (un)packing of the real transform and the column transposes (row stride M1 + 1; line
// stride LS chosen so the transposes are free of bank conflicts).
// ---------------------------------------------------------------------------------------

// cos and sin of pi q / M1 (M1 = 8 or 16), q in [0, M1): a switch on a constant index after
// unrolling, so the values become immediates
template <int M1>
__device__ __forceinline__ float cospi_q(int q) {
  if constexpr (M1 == 8) {
    switch (q) {
      case 0: return 1.0f;
      case 1: return 0.923879533f;
      case 2: return 0.707106781f;
      case 3: return 0.382683432f;
      case 4: return 0.0f;
      case 5: return -0.382683432f;
      case 6: return -0.707106781f;
      default: return -0.923879533f;
    }
  } else {
    switch (q) {
      case 0: return 1.0f;
      case 1: return 0.980785280f;
      case 2: return 0.923879533f;
      case 3: return 0.831469612f;
      case 4: return 0.707106781f;
      case 5: return 0.555570233f;
      case 6: return 0.382683432f;
      case 7: return 0.195090322f;
      case 8: return 0.0f;
      case 9: return -0.195090322f;
      case 10: return -0.382683432f;
      case 11: return -0.555570233f;
      case 12: return -0.707106781f;
      case 13: return -0.831469612f;
      case 14: return -0.923879533f;
      default: return -0.980785280f;
    }
  }
}
template <int M1>
__device__ __forceinline__ float sinpi_q(int q) {
  return (q == 0) ? 0.0f : cospi_q<M1>((q + M1 / 2) % M1) * ((q + M1 / 2 >= M1) ? -1.0f : 1.0f) * -1.0f;
}

// Packing twiddle W_{n0}^k of the float register x passes for k = M2 q + t (n0 = 2 M1 M2):
// W_{n0}^{M2 q} = exp(-i pi q / M1) from compile-time constants times this thread's W_{n0}^t
// (one float complex product, within ~1 ulp of the table value) instead of a shared-memory
// read per element: the x pass is limited by its shared-memory instruction rate.
template <int M1>
__device__ __forceinline__ cpx<float> pk_q(int q, cpx<float> wt) {
  const float c = cospi_q<M1>(q), s = sinpi_q<M1>(q);   // W_{n0}^{M2 q} = c - i s
  return mk<float>(c * wt.x + s * wt.y, c * wt.y - s * wt.x);
}

template <typename T, int M1, int M2>
struct XR {
  static constexpr int M = M1 * M2;
  static constexpr int C = M1 / M2;
  static constexpr int LINES = 256 / M2;
  static constexpr int RS = M1 + 1;                      // row stride of the transpose
  static constexpr int LS0 = (M2 * RS > M + 1) ? M2 * RS : M + 1;
  static constexpr int LS = (sizeof(T) == 4) ? ((LS0 + 7) / 16 * 16 + 8) : LS0;   // float: LS = 8 mod 16
};

// one four-step transform of length M1*M2 on registers u[M1] (input z[M2 q + t] in u[q]);
// on return u[c + C k2] = output[t + M2 c + M1 k2].  Yl: this line's buffer.
template <typename T, int S, int M1, int M2>
__device__ __forceinline__ void fourstep(cpx<T> (&u)[M1], cpx<T>* Yl, const StepTw<T, M1>& tw, int t) {
  constexpr int RS = M1 + 1;
  constexpr int C = M1 / M2;
  dftR<T, S, M1>(u);
#pragma unroll
  for (int k1 = 1; k1 < M1; ++k1) {
    const cpx<T> w = tw(k1);
    u[k1] = (S < 0) ? cmul(u[k1], w) : cmulc(u[k1], w);
  }
  __syncthreads();
#pragma unroll
  for (int k1 = 0; k1 < M1; ++k1) Yl[t * RS + k1] = u[k1];
  __syncthreads();
#pragma unroll
  for (int c = 0; c < C; ++c) {
    cpx<T> v[M2];
#pragma unroll
    for (int n2 = 0; n2 < M2; ++n2) v[n2] = Yl[n2 * RS + t + M2 * c];
    dftR<T, S, M2>(v);
#pragma unroll
    for (int k2 = 0; k2 < M2; ++k2) u[c + C * k2] = v[k2];
  }
}

template <typename T, int M1, int M2>
__global__ void __launch_bounds__(256, (sizeof(T) == 4 ? 4 : 1)) k_xpass_r(const XProg P, const GridDesc g,
                                                                          const cpx<T>* __restrict__ twg) {
  using X = XR<T, M1, M2>;
  constexpr int M = X::M, LINES = X::LINES, LS = X::LS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (P.done && *P.done) return;
  const int h0 = g.h0;
  cpx<T>* twm = reinterpret_cast<cpx<T>*>(smem_raw);
  cpx<T>* pk = twm + M;
  cpx<T>* buf = pk + (M + 2);
  const int tid = threadIdx.x;
  for (int j = tid; j < M; j += 256) twm[j] = twg[g.px.tw_off + j];
  for (int j = tid; j <= M; j += 256) pk[j] = twg[g.pk_off + j];
  const long long nlines = (long long)g.n1 * g.n2;
  const long long line0 = (long long)blockIdx.x * LINES;
  const int line = tid / M2;
  const int t = tid % M2;
  const bool lok = line0 + line < nlines;
  cpx<T>* Yl = buf + line * LS;
  const T kfx = kfac_t<T>(g, 0);
  const T scale = scale_t<T>(P.scale, P.scale_hi, P.scale_lo);
  const int lb = (int)((line0 + line) * h0);      // spectral line base
  const int rb = (int)((line0 + line) * M);       // real line base (complex pairs)
  const T* __restrict__ symarr = reinterpret_cast<const T*>(P.symarr);
  auto premul = [&](int flags, int k, cpx<T> v) -> cpx<T> {
    if (!flags) return v;
    const T kx = kfx * (T)freq_tilde(k, g.n0);
    T cc = T(1);
    if (flags & MUL_IK) cc *= kx;
    if (flags & MUL_SYM) cc *= symarr[lb + k];
    if (flags & (MUL_NEGK2 | MUL_IK2)) cc *= -kx * kx;
    v = scal(v, cc);
    if (flags & MUL_IK) v = mul_i(v);
    return v;
  };

  __syncthreads();   // the tables are complete
  const StepTw<T, M1> stw(twm, t);
  for (int c = 0; c < P.ncomp; ++c) {
    const int cin = (P.conv_in >> c) & 1, cout = (P.conv_out >> c) & 1;
    cpx<T> u[M1];
    __syncthreads();
    if (P.mode == 1) {
#pragma unroll
      for (int q = 0; q < M1; ++q) u[q] = lok ? ld_el<T>(P.in[c], cin, rb + M2 * q + t) : mk<T>(T(0), T(0));
    } else {
      // stage the half spectrum (h0 = M + 1 entries: k = t + M2 q, and k = M for thread 0),
      // all loads of the thread issued before the first store, then pack it into the
      // length-m complex spectrum
      if (lok) {
        cpx<T> hv[M1];
#pragma unroll
        for (int q = 0; q < M1; ++q) hv[q] = ld_el<T>(P.in[c], cin, lb + t + M2 * q);
        const cpx<T> hn = (t == 0) ? ld_el<T>(P.in[c], cin, lb + M) : mk<T>(T(0), T(0));
#pragma unroll
        for (int q = 0; q < M1; ++q) Yl[t + M2 * q] = premul(P.pre[c], t + M2 * q, hv[q]);
        if (t == 0) Yl[M] = premul(P.pre[c], M, hn);
      }
      __syncthreads();
#pragma unroll
      for (int q = 0; q < M1; ++q) {
        const int j = M2 * q + t;
        const cpx<T> Xv = Yl[j];
        const cpx<T> Xc = conjg(Yl[M - j]);
        cpx<T> w;
        if constexpr (std::is_same<T, float>::value) w = pk_q<M1>(q, pk[t]);
        else w = pk[j];
        u[q] = (Xv + Xc) + mul_i(cmulc(Xv - Xc, w));
      }
      fourstep<T, +1, M1, M2>(u, Yl, stw, t);
      if (P.mode == 2) {
        if (lok) {
#pragma unroll
          for (int q = 0; q < M1; ++q) st_el<T>(P.out[c], cout, rb + M2 * q + t, scal(u[q], scale), true);
        }
        continue;
      }
      if (P.wfield && lok) {
        if (P.wf_dd) {
          // the float pairs of the two reals of u[q]: one 16-byte load
          const float4* __restrict__ wf4 = reinterpret_cast<const float4*>(P.wfield) + rb;
#pragma unroll
          for (int q = 0; q < M1; ++q) {
            const float4 w = wf4[M2 * q + t];
            u[q] = mk<T>(mul_pair(u[q].x, w.x, w.y), mul_pair(u[q].y, w.z, w.w));
          }
        } else {
          const cpx<T>* __restrict__ wf = reinterpret_cast<const cpx<T>*>(P.wfield) + rb;
#pragma unroll
          for (int q = 0; q < M1; ++q) {
            const cpx<T> wv = wf[M2 * q + t];
            u[q] = mk<T>(u[q].x * wv.x, u[q].y * wv.y);
          }
        }
      }
    }
    fourstep<T, -1, M1, M2>(u, Yl, stw, t);
    // unpack the length-m spectrum into the half spectrum
    __syncthreads();
#pragma unroll
    for (int q = 0; q < M1; ++q) Yl[M2 * q + t] = u[q];
    __syncthreads();
    if (lok) {
      const int post = P.post[c];
      // entries k = t + M2 q (q < M1) and, for thread 0, k = M: a fixed count, unrolled
      auto unpack = [&](int k, cpx<T> w) {
        const cpx<T> Z = Yl[k == M ? 0 : k];
        const cpx<T> Zc = conjg(Yl[k == 0 ? 0 : M - k]);
        cpx<T> Xv = (Z + Zc) - mul_i(cmul(Z - Zc, w));
        T cc = scale;
        if (post) {
          const T kx = kfx * (T)freq_tilde(k, g.n0);
          if (post & MUL_IK) cc *= kx;
          if (post & MUL_SYM) cc *= symarr[lb + k];
          if (post & (MUL_NEGK2 | MUL_IK2)) cc *= -kx * kx;
        }
        Xv = scal(Xv, cc);
        if (post & MUL_IK) Xv = mul_i(Xv);
        st_el<T>(P.out[c], cout, lb + k, Xv, true);
      };
#pragma unroll
      for (int q = 0; q < M1; ++q) {
        if constexpr (std::is_same<T, float>::value) unpack(t + M2 * q, pk_q<M1>(q, pk[t]));
        else unpack(t + M2 * q, pk[t + M2 * q]);
      }
      if (t == 0) unpack(M, pk[M]);
    }
  }
}

// ---------------------------------------------------------------------------------------
// fused x pass (mode 0), register four-step transforms with TMA-staged input lines (float)
//
// The arithmetic of k_xpass_r in a persistent grid over (group of LINES lines, component)
// items.  A group's half-spectrum lines are contiguous in memory (LINES x pitch complex
// values; 16-byte aligned for an even group size), so the tensor memory accelerator fetches
// the next item's lines with one bulk copy (cp.async.bulk) into a shared-memory stage while
// the current item is transformed, weighted and stored.  Packing reads the stage directly.
// Bounded waits as in k_axis_tma.
// ---------------------------------------------------------------------------------------

__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}

template <int M1, int M2>
__global__ void __launch_bounds__(256, 3) k_xpass_tma(const XProg P, const GridDesc g, const cpx<float>* __restrict__ twg) {
  using T = float;
  using X = XR<T, M1, M2>;
  constexpr int M = X::M, LINES = X::LINES, LS = X::LS;
  extern __shared__ __align__(1024) unsigned char smem_tma[];
  unsigned char* smem_raw = smem_tma;
  if (P.done && *P.done) return;
  const int h0 = g.h0;
  const int pitch = h0;
  const unsigned stage_bytes = (unsigned)(LINES * pitch * sizeof(cpx<T>));   // multiple of 16 (LINES even)
  cpx<T>* stage = reinterpret_cast<cpx<T>*>(smem_raw);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + stage_bytes);
  cpx<T>* twm = reinterpret_cast<cpx<T>*>(smem_raw + stage_bytes + 16);
  cpx<T>* pk = twm + M;
  cpx<T>* buf = pk + (M + 2);
  const int tid = threadIdx.x;
  for (int j = tid; j < M; j += 256) twm[j] = twg[g.px.tw_off + j];
  for (int j = tid; j <= M; j += 256) pk[j] = twg[g.pk_off + j];
  if (tid == 0) mbar_init(bar, 1);
  __syncthreads();
  const long long nlines = (long long)g.n1 * g.n2;
  const int groups = (int)((nlines + LINES - 1) / LINES);
  const int nc = P.ncomp;
  const int my_groups = ((int)blockIdx.x < groups) ? (groups - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const int nitems = my_groups * nc;
  if (nitems == 0) return;
  auto issue = [&](int item) {
    const long long line0 = (long long)((int)blockIdx.x + (item / nc) * (int)gridDim.x) * LINES;
    const int c = item % nc;
    const int nl = (int)min((long long)LINES, nlines - line0);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    const unsigned bytes = (unsigned)(nl * pitch * sizeof(cpx<T>));
    mbar_expect_tx(bar, bytes);
    bulk_load(stage, reinterpret_cast<const cpx<T>*>(P.in[c]) + line0 * pitch, bytes, bar);
  };
  if (tid == 0) issue(0);
  const int line = tid / M2;
  const int t = tid % M2;
  const StepTw<T, M1> stw(twm, t);   // (the tables were completed before the first barrier)
  cpx<T>* Yl = buf + line * LS;
  const cpx<T>* Sl = stage + line * pitch;
  const T kfx = kfac_t<T>(g, 0);
  const T scale = scale_t<T>(P.scale, P.scale_hi, P.scale_lo);

  for (int it = 0; it < nitems; ++it) {
    const long long line0 = (long long)((int)blockIdx.x + (it / nc) * (int)gridDim.x) * LINES;
    const int c = it % nc;
    const bool lok = line0 + line < nlines;
    const int lb = (int)((line0 + line) * pitch);
    const int rb = (int)((line0 + line) * M);
    const T* __restrict__ symarr = reinterpret_cast<const T*>(P.symarr) + (line0 + line) * h0;
    const int pre = P.pre[c], post = P.post[c];
    auto premul = [&](int k, cpx<T> v) -> cpx<T> {
      if (!pre) return v;
      const T kx = kfx * (T)freq_tilde(k, g.n0);
      T cc = T(1);
      if (pre & MUL_IK) cc *= kx;
      if (pre & MUL_SYM) cc *= symarr[k];
      if (pre & (MUL_NEGK2 | MUL_IK2)) cc *= -kx * kx;
      v = scal(v, cc);
      if (pre & MUL_IK) v = mul_i(v);
      return v;
    };
    const bool ok = mbar_wait_bounded(bar, (unsigned)(it & 1));
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        if (g.dev_err) atomicExch(g.dev_err, 1);
        mbar_wait_bounded(bar, (unsigned)(it & 1));
      }
      __syncthreads();
      return;
    }
    cpx<T> u[M1];
#pragma unroll
    for (int q = 0; q < M1; ++q) {
      const int j = M2 * q + t;
      const cpx<T> Xv = premul(j, Sl[j]);
      const cpx<T> Xc = conjg(premul(M - j, Sl[M - j]));
      u[q] = (Xv + Xc) + mul_i(cmulc(Xv - Xc, pk_q<M1>(q, pk[t])));
    }
    // the stage is consumed: it takes the next item's lines while this one is transformed
    __syncthreads();
    if (tid == 0 && it + 1 < nitems) issue(it + 1);
    fourstep<T, +1, M1, M2>(u, Yl, stw, t);
    if (P.wfield && lok) {
      if (P.wf_dd) {
        const float4* __restrict__ wf4 = reinterpret_cast<const float4*>(P.wfield) + rb;
#pragma unroll
        for (int q = 0; q < M1; ++q) {
          const float4 w = wf4[M2 * q + t];
          u[q] = mk<T>(mul_pair(u[q].x, w.x, w.y), mul_pair(u[q].y, w.z, w.w));
        }
      } else {
        const cpx<T>* __restrict__ wf = reinterpret_cast<const cpx<T>*>(P.wfield) + rb;
#pragma unroll
        for (int q = 0; q < M1; ++q) {
          const cpx<T> wv = wf[M2 * q + t];
          u[q] = mk<T>(u[q].x * wv.x, u[q].y * wv.y);
        }
      }
    }
    fourstep<T, -1, M1, M2>(u, Yl, stw, t);
    __syncthreads();
#pragma unroll
    for (int q = 0; q < M1; ++q) Yl[M2 * q + t] = u[q];
    __syncthreads();
    if (lok) {
      auto unpack = [&](int k, cpx<T> w) {
        const cpx<T> Z = Yl[k == M ? 0 : k];
        const cpx<T> Zc = conjg(Yl[k == 0 ? 0 : M - k]);
        cpx<T> Xv = (Z + Zc) - mul_i(cmul(Z - Zc, w));
        T cc = scale;
        if (post) {
          const T kx = kfx * (T)freq_tilde(k, g.n0);
          if (post & MUL_IK) cc *= kx;
          if (post & MUL_SYM) cc *= symarr[k];
          if (post & (MUL_NEGK2 | MUL_IK2)) cc *= -kx * kx;
        }
        Xv = scal(Xv, cc);
        if (post & MUL_IK) Xv = mul_i(Xv);
        reinterpret_cast<cpx<T>*>(P.out[c])[lb + k] = Xv;
      };
#pragma unroll
      for (int q = 0; q < M1; ++q) unpack(t + M2 * q, pk_q<M1>(q, pk[t]));
      if (t == 0) unpack(M, pk[M]);
    }
  }
}

// the staged x pass takes fused float programs with aligned fields and a whole-line stage
static bool xpass_tma_ok(const XProg& P, const GridDesc& g, int lines) {
  if (P.mode != 0 || P.aux_out || P.conv_in || P.conv_out || g.n1 * g.n2 < 2) return false;
  const int pitch = g.h0;
  if (((long long)lines * pitch * (long long)sizeof(cpx<float>)) % 16) return false;
  for (int c = 0; c < P.ncomp; ++c)
    if (reinterpret_cast<uintptr_t>(P.in[c]) & 15u) return false;
  return true;
}

template <int M1, int M2>
static bool launch_xpass_tma(const XProg& P, const GridDesc& g, const cpx<float>* tw, cudaStream_t st) {
  using X = XR<float, M1, M2>;
  if (!xpass_tma_ok(P, g, X::LINES)) return false;
  const int pitch = g.h0;
  const long long nlines = (long long)g.n1 * g.n2;
  const long long groups = (nlines + X::LINES - 1) / X::LINES;
  const long long blocks = std::min<long long>(groups, 3LL * sm_count());
  const size_t smem = sizeof(cpx<float>) * (size_t)(X::LINES * pitch) + 16 +
                      sizeof(cpx<float>) * (size_t)(X::M + (X::M + 2) + X::LINES * X::LS);
  ensure_smem(reinterpret_cast<const void*>(k_xpass_tma<M1, M2>), smem);
  k_xpass_tma<M1, M2><<<(unsigned)blocks, 256, smem, st>>>(P, g, tw);
  return true;
}

template <typename T, int M1, int M2>
static void launch_xpass_r(const XProg& P, const GridDesc& g, const cpx<T>* tw, cudaStream_t st) {
  using X = XR<T, M1, M2>;
  const long long nlines = (long long)g.n1 * g.n2;
  const long long blocks = (nlines + X::LINES - 1) / X::LINES;
  const size_t smem = sizeof(cpx<T>) * (size_t)(X::M + (X::M + 2) + X::LINES * X::LS);
  ensure_smem(reinterpret_cast<const void*>(k_xpass_r<T, M1, M2>), smem);
  k_xpass_r<T, M1, M2><<<(unsigned)blocks, 256, smem, st>>>(P, g, tw);
}

// ---------------------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------------------

// ---------------------------------------------------------------------------------------
// launch-shape table, filled by the autotuner (vd_autotune) and consulted by every launch:
// choice 0 = register-resident four-step kernel, > 0 = lines per block of the Stockham
// engine; absent = the built-in heuristic.  Optionally persisted in the file named by the
// environment variable VD_TUNE_FILE (one entry per line: kind type length axis dir choice).
// ---------------------------------------------------------------------------------------

template <typename T>
constexpr int type_code() {
  return std::is_same<T, dd>::value ? 2 : (sizeof(T) == 4 ? 1 : 0);
}

static std::mutex g_tune_mu;
static std::map<long long, int> g_tune;
static bool g_tune_loaded = false;

static long long tune_key(int kind, int type, int n, int axis, int dir) {
  return ((long long)kind << 48) | ((long long)type << 40) | ((long long)(axis & 0xff) << 32) |
         ((long long)((dir + 4) & 0xff) << 24) | (long long)(n & 0xffffff);
}

static void tune_load_locked() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char* path = std::getenv("VD_TUNE_FILE");
  if (!path) return;
  FILE* f = std::fopen(path, "r");
  if (!f) return;
  int kind, type, n, axis, dir, choice;
  while (std::fscanf(f, "%d %d %d %d %d %d", &kind, &type, &n, &axis, &dir, &choice) == 6)
    g_tune[tune_key(kind, type, n, axis, dir)] = choice;
  std::fclose(f);
}

int tune_get(int kind, int type, int n, int axis, int dir) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  tune_load_locked();
  auto it = g_tune.find(tune_key(kind, type, n, axis, dir));
  return it == g_tune.end() ? -1 : it->second;
}

void tune_set(int kind, int type, int n, int axis, int dir, int choice) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  tune_load_locked();
  if (choice < 0) g_tune.erase(tune_key(kind, type, n, axis, dir));
  else g_tune[tune_key(kind, type, n, axis, dir)] = choice;
}

int default_shape(int kind, int type, int n, int axis) {
  const int ept = (type == 1) ? 16 : 8;
  // float z passes of length 128/256: the TMA-staged kernel (its gain is largest on the
  // multi-transform programs of the operators, which the tuner's single transform understates)
  if (kind == 0 && type == 1 && axis == 2 && (n == 128 || n == 256)) return kChoiceStaged;
  if (kind == 0) return (type == 1 && (n == 128 || n == 256)) ? 0 : tile_width(n, ept);
  return (type == 1 && (n == 64 || n == 128 || n == 256)) ? 0 : lines_per_cta(n, ept);
}

int tune_table(int* out, int max) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  tune_load_locked();
  int k = 0;
  for (const auto& kv : g_tune) {
    if (out && k < max) {
      const long long key = kv.first;
      int* e = out + 6 * k;
      e[0] = (int)(key >> 48);
      e[1] = (int)((key >> 40) & 0xff);
      e[2] = (int)(key & 0xffffff);
      e[3] = (int)((key >> 32) & 0xff);
      e[4] = (int)((key >> 24) & 0xff) - 4;
      e[5] = kv.second;
    }
    ++k;
  }
  return k;
}

void tune_save() {
  const char* path = std::getenv("VD_TUNE_FILE");
  if (!path) return;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  FILE* f = std::fopen(path, "w");
  if (!f) return;
  for (const auto& kv : g_tune) {
    const long long key = kv.first;
    std::fprintf(f, "%d %d %d %d %d %d\n", (int)(key >> 48), (int)((key >> 40) & 0xff), (int)(key & 0xffffff),
                 (int)((key >> 32) & 0xff), (int)((key >> 24) & 0xff) - 4, kv.second);
  }
  std::fclose(f);
}

// Opt a kernel into more than 48 KB of dynamic shared memory.  The limit only grows, under a
// lock: launches from several host threads (server slots) must never lower it below the
// size another thread is about to launch with.
static void ensure_smem(const void* func, size_t smem) {
  if (smem <= 48 * 1024) return;
  static std::mutex mu;
  static std::map<const void*, size_t> set;
  std::lock_guard<std::mutex> lk(mu);
  size_t& cur = set[func];
  if (smem > cur) {
    cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cur = smem;
  }
}

template <typename T>
size_t axis_smem_bytes(const GridDesc& g, int axis) {
  const int n = (axis == 2) ? g.pz.n : g.py.n;
  const int W = tile_width(n, kEPT<T>);
  return sizeof(cpx<T>) * (size_t)(n + 2 * W * n);
}

template <typename T>
size_t xpass_smem_bytes(const GridDesc& g) {
  const int m = g.n0 / 2;
  const int L = lines_per_cta(m, kEPT<T>);
  return sizeof(cpx<T>) * (size_t)(m + (m + 2) + 2 * L * (m + 1));
}

template <typename T, int S, bool CV, bool PK>
static void launch_k_axis(const AxisProg& P, const GridDesc& g, const cpx<T>* tw, int W, long long blocks,
                          size_t smem, cudaStream_t st) {
  ensure_smem(reinterpret_cast<const void*>(k_axis<T, S, CV, PK>), smem);
  k_axis<T, S, CV, PK><<<(unsigned)blocks, kThreads, smem, st>>>(P, g, tw, ilog2(W));
}

template <typename T, int S, int N1, int N2>
static void launch_axis_r(const AxisProg& P, const GridDesc& g, const cpx<T>* tw, long long inner_n,
                          long long outer_n, cudaStream_t st) {
  const long long blocks = outer_n * ((inner_n + kRLines - 1) / kRLines);
  const size_t smem = sizeof(cpx<T>) * (size_t)(N1 * N2 + kRLines * (N1 * N2 + 1)) + sizeof(T) * (size_t)(N1 * N2);
  ensure_smem(reinterpret_cast<const void*>(k_axis_r<T, S, N1, N2>), smem);
  k_axis_r<T, S, N1, N2><<<(unsigned)blocks, kRLines * N2, smem, st>>>(P, g, tw);
}

static void split_scale(double s, float* hi, float* lo) {
  *hi = (float)s;
  *lo = (float)(s - (double)*hi);
}

// tensor-map encoder of the driver, looked up once through the runtime (no libcuda link)
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

// map of a half-spectrum field for the tiles of an axis pass: z pass, 2D [n2][2 n1 h0] floats;
// y pass, 3D [n2][n1][2 h0] (rows 8 h0 bytes apart: even h0 only); box 16 columns x N rows
static bool encode_tiles(CUtensorMap* m, const void* base, const GridDesc& g, int axis, int N) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc || (reinterpret_cast<uintptr_t>(base) & 15u)) return false;
  const cuuint64_t row = (cuuint64_t)g.h0 * sizeof(cpx<float>);
  if (axis == 2) {
    const cuuint64_t inner = (cuuint64_t)g.n1 * (cuuint64_t)g.h0;
    cuuint64_t dims[2] = {2 * inner, (cuuint64_t)g.n2};
    cuuint64_t strides[1] = {inner * sizeof(cpx<float>)};
    cuuint32_t box[2] = {2 * kRLines, (cuuint32_t)N};
    cuuint32_t es[2] = {1, 1};
    if (strides[0] % 16) return false;
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
  }
  // y pass: each z plane viewed as n1/2 pair rows (y rows 2r and 2r+1 back to back, 16 h0 bytes:
  // 16-byte aligned whatever the parity of h0), boxes of 18 columns x N/2 pair rows
  cuuint64_t dims[3] = {4 * (cuuint64_t)g.h0, (cuuint64_t)(g.n1 / 2), (cuuint64_t)g.n2};
  cuuint64_t strides[2] = {2 * row, row * (cuuint64_t)g.n1};
  cuuint32_t box[3] = {2 * kPairCols, (cuuint32_t)(N / 2), 1};
  cuuint32_t es[3] = {1, 1, 1};
  if ((g.n1 & 1) || strides[0] % 16 || strides[1] % 16) return false;
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(base), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

static int sm_count() {
  static int cached[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return 152;
  if (!cached[dev]) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    cached[dev] = v > 0 ? v : 152;
  }
  return cached[dev];
}

// The TMA-staged kernel takes programs whose transforms all run an FFT and read in[0..3].  It
// fetches the input of the next (tile, transform) item while the current one stores, so no
// transform may read a field that an earlier transform of the program writes.
static bool tma_program_ok(const AxisProg& P, const GridDesc& g) {
  if (P.conv_in || P.conv_out || P.nxf <= 0) return false;
  if (P.axis == 1 && (g.n1 & 1)) return false;
  for (int t = 0; t < P.nxf; ++t)
    if (P.xf[t].nofft || P.xf[t].src >= kTmaMaxIn) return false;
  for (int b = 1; b < P.nxf; ++b)
    for (int a = 0; a < b; ++a)
      if (P.in[P.xf[b].src] == P.out[P.xf[a].dst]) return false;
  return true;
}

template <int S, int N1, int N2, int AX>
static bool launch_axis_tma(const AxisProg& P, const GridDesc& g, const cpx<float>* tw, cudaStream_t st) {
  constexpr int N = N1 * N2;
  TmaMaps maps;
  std::memset(&maps, 0, sizeof maps);
  unsigned used = 0;
  for (int t = 0; t < P.nxf; ++t) used |= 1u << P.xf[t].src;
  for (int k = 0; k < kTmaMaxIn; ++k)
    if ((used >> k) & 1u)
      if (!encode_tiles(&maps.m[k], P.in[k], g, P.axis, N)) return false;
  const long long cols = (P.axis == 2) ? (long long)g.n1 * g.h0 : g.h0;
  const long long tiles = ((cols + kRLines - 1) / kRLines) * (P.axis == 2 ? 1 : g.n2);
  const int per_sm = (N2 == 16) ? 3 : 6;
  const long long blocks = std::min<long long>(tiles, (long long)per_sm * sm_count());
  const size_t stage = sizeof(cpx<float>) * (size_t)(N * (AX == 2 ? kRLines : kPairCols));
  const size_t smem = stage + 16 + sizeof(cpx<float>) * (size_t)(N + kRLines * (N + 1)) + sizeof(float) * (size_t)N;
  ensure_smem(reinterpret_cast<const void*>(k_axis_tma<S, N1, N2, AX>), smem);
  k_axis_tma<S, N1, N2, AX><<<(unsigned)blocks, kRLines * N2, smem, st>>>(P, g, tw, maps);
  return true;
}

template <typename T>
void launch_axis(const AxisProg& P0, int dir, const GridDesc& g, const void* tw, cudaStream_t st) {
  AxisProg P = P0;
  for (int t = 0; t < P.nxf; ++t) split_scale(P.xf[t].scale, &P.xf[t].scale_hi, &P.xf[t].scale_lo);
  const int n = (P.axis == 2) ? g.pz.n : g.py.n;
  int choice = tune_get(0, type_code<T>(), n, P.axis, dir);
  const bool reg_ok = std::is_same<T, float>::value && (n == 256 || n == 128);
  if (choice < 0) choice = default_shape(0, type_code<T>(), n, P.axis);
  if (choice == kChoiceStaged && !(reg_ok && tma_program_ok(P, g))) choice = 0;   // not applicable: register kernel
  const int W = (choice > 0 && choice <= 64) ? choice : tile_width(n, kEPT<T>);
  long long inner_n, outer_n;
  if (P.axis == 2) {
    inner_n = (long long)g.n1 * g.h0;
    outer_n = 1;
  } else {
    inner_n = g.h0;
    outer_n = g.n2;
  }
  const long long blocks = outer_n * ((inner_n + W - 1) / W);
  const size_t smem = sizeof(cpx<T>) * (size_t)(n + 2 * W * n);
  const cpx<T>* twp = reinterpret_cast<const cpx<T>*>(tw);
  // algorithmic traffic: every distinct input and output field once, the symbol array once
  unsigned inmask = 0, outmask = 0;
  int nfft = 0;
  bool sym = false;
  for (int t = 0; t < P.nxf; ++t) {
    inmask |= 1u << P.xf[t].src;
    outmask |= 1u << P.xf[t].dst;
    nfft += P.xf[t].nofft ? 0 : 1;
    sym = sym || ((P.xf[t].pre | P.xf[t].post) & MUL_SYM);
  }
  const double fb = (double)g.ncplx * sizeof(cpx<T>);
  const double bytes = (__builtin_popcount(inmask) + __builtin_popcount(outmask)) * fb + (sym ? g.ncplx * sizeof(T) : 0);
  const double flops = (double)nfft * (double)g.ncplx * 5.0 * std::log2((double)n);
  ProfScope ps(std::is_same<T, dd>::value ? PC_AXISDD : (sizeof(T) == 8 ? PC_AXIS64 : PC_AXIS32), st, bytes,
               flops);
  if constexpr (std::is_same<T, float>::value) {
    const cpx<float>* twf = reinterpret_cast<const cpx<float>*>(tw);
    if (choice == kChoiceStaged) {
      bool ok;
      if (P.axis == 2) {
        if (n == 256) ok = (dir < 0) ? launch_axis_tma<-1, 16, 16, 2>(P, g, twf, st) : launch_axis_tma<+1, 16, 16, 2>(P, g, twf, st);
        else ok = (dir < 0) ? launch_axis_tma<-1, 16, 8, 2>(P, g, twf, st) : launch_axis_tma<+1, 16, 8, 2>(P, g, twf, st);
      } else {
        if (n == 256) ok = (dir < 0) ? launch_axis_tma<-1, 16, 16, 1>(P, g, twf, st) : launch_axis_tma<+1, 16, 16, 1>(P, g, twf, st);
        else ok = (dir < 0) ? launch_axis_tma<-1, 16, 8, 1>(P, g, twf, st) : launch_axis_tma<+1, 16, 8, 1>(P, g, twf, st);
      }
      if (ok) return;
      choice = 0;   // no tensor map (encoder unavailable or unaligned field): the register kernel
    }
    // register-resident four-step kernel for the common lengths (unless tuned otherwise)
    if (reg_ok && choice <= 0) {
      if (n == 256) {
        if (dir < 0) launch_axis_r<T, -1, 16, 16>(P, g, twp, inner_n, outer_n, st);
        else launch_axis_r<T, +1, 16, 16>(P, g, twp, inner_n, outer_n, st);
      } else {
        if (dir < 0) launch_axis_r<T, -1, 16, 8>(P, g, twp, inner_n, outer_n, st);
        else launch_axis_r<T, +1, 16, 8>(P, g, twp, inner_n, outer_n, st);
      }
      return;
    }
  }
  const bool cv = (P.conv_in | P.conv_out) != 0;
  if constexpr (std::is_same<T, dd>::value) {
    if (choice != kChoiceUnpacked && p_plan_ok(P.axis == 2 ? g.pz : g.py, kThreads / W)) {
      const size_t psmem = smem + sizeof(pdd) * (size_t)n;   // the second twiddle table
      if (dir < 0 && cv) launch_k_axis<T, -1, true, true>(P, g, twp, W, blocks, psmem, st);
      else if (dir < 0) launch_k_axis<T, -1, false, true>(P, g, twp, W, blocks, psmem, st);
      else if (cv) launch_k_axis<T, +1, true, true>(P, g, twp, W, blocks, psmem, st);
      else launch_k_axis<T, +1, false, true>(P, g, twp, W, blocks, psmem, st);
      return;
    }
  }
  if (dir < 0 && cv) launch_k_axis<T, -1, true, false>(P, g, twp, W, blocks, smem, st);
  else if (dir < 0) launch_k_axis<T, -1, false, false>(P, g, twp, W, blocks, smem, st);
  else if (cv) launch_k_axis<T, +1, true, false>(P, g, twp, W, blocks, smem, st);
  else launch_k_axis<T, +1, false, false>(P, g, twp, W, blocks, smem, st);
}

template <typename T, bool CV, bool PK, int MINB = (std::is_same<T, dd>::value ? 3 : 1)>
static void launch_k_xpass(const XProg& P, const GridDesc& g, const cpx<T>* tw, int L, long long blocks, size_t smem,
                           cudaStream_t st) {
  ensure_smem(reinterpret_cast<const void*>(k_xpass<T, CV, PK, MINB>), smem);
  k_xpass<T, CV, PK, MINB><<<(unsigned)blocks, kThreads, smem, st>>>(P, g, tw, ilog2(L));
}

template <typename T>
void launch_xpass(const XProg& P0, const GridDesc& g, const void* tw, cudaStream_t st) {
  if (P0.aux_out && (P0.mode != 0 || !std::is_same<T, dd>::value)) {
    // the extra inverse output is fused into the float-pair engine only: elsewhere it is a
    // separate mode-2 pass over in[0], run before the program (which may work in place)
    XProg A{};
    A.ncomp = 1;
    A.mode = 2;
    A.in[0] = P0.in[0];
    A.conv_in = P0.conv_in & 1;
    A.out[0] = P0.aux_out;
    A.conv_out = P0.aux_conv;
    A.scale = P0.aux_scale;
    A.done = P0.done;
    launch_xpass<T>(A, g, tw, st);
    XProg B = P0;
    B.aux_out = nullptr;
    launch_xpass<T>(B, g, tw, st);
    return;
  }
  XProg P = P0;
  split_scale(P.scale, &P.scale_hi, &P.scale_lo);
  split_scale(P.aux_scale, &P.aux_scale_hi, &P.aux_scale_lo);
  const int m = g.n0 / 2;
  int choice = tune_get(1, type_code<T>(), m, 0, P.mode);
  const int L = (choice > 0 && choice <= 64) ? choice : lines_per_cta(m, kEPT<T>);
  const long long nlines = (long long)g.n1 * g.n2;
  const long long blocks = (nlines + L - 1) / L;
  const size_t smem = sizeof(cpx<T>) * (size_t)(m + (m + 2) + 2 * L * (m + 1));
  const bool cv = (P.conv_in | P.conv_out | (P.aux_out ? P.aux_conv : 0)) != 0;
  const double fc = (double)g.ncplx * sizeof(cpx<T>), fr = (double)g.nreal * sizeof(T);
  double bytes = 0, flops = 0;
  const double real_fft = (double)g.nreal * 2.5 * std::log2((double)g.n0);   // one real transform of every line
  if (P.mode == 0) {
    bytes = P.ncomp * 2.0 * fc + (P.wfield ? (P.wf_dd ? 2.0 * fr : fr) : 0.0);
    flops = P.ncomp * 2.0 * real_fft;
  } else {
    bytes = P.ncomp * (fc + fr);
    flops = P.ncomp * real_fft;
  }
  if (P.aux_out) {   // the inverse-only transform of in[0] and its real output
    bytes += fr;
    flops += real_fft;
  }
  bool sym = false;
  for (int c = 0; c < P.ncomp; ++c) sym = sym || ((P.pre[c] | P.post[c]) & MUL_SYM);
  if (sym) bytes += (double)g.ncplx * sizeof(T);
  ProfScope ps(std::is_same<T, dd>::value ? PC_XPASSDD : (sizeof(T) == 8 ? PC_XPASS64 : PC_XPASS32), st, bytes,
               flops);
  if constexpr (std::is_same<T, float>::value) {
    // register-resident kernel (float; the float-pair version needs too many registers),
    // unless the tuner chose the Stockham engine for this length
    const cpx<T>* twp = reinterpret_cast<const cpx<T>*>(tw);
    if (choice == kChoiceStaged) {
      bool ok = false;
      if (m == 128) ok = launch_xpass_tma<16, 8>(P, g, twp, st);
      else if (m == 64) ok = launch_xpass_tma<8, 8>(P, g, twp, st);
      else if (m == 256) ok = launch_xpass_tma<16, 16>(P, g, twp, st);
      if (ok) return;
      choice = 0;   // not a fused float program, or unaligned: the register kernel
    }
    if (choice <= 0 && m == 128) {
      launch_xpass_r<T, 16, 8>(P, g, twp, st);
      return;
    }
    if (choice <= 0 && m == 64) {
      launch_xpass_r<T, 8, 8>(P, g, twp, st);
      return;
    }
    if (choice <= 0 && m == 256) {
      launch_xpass_r<T, 16, 16>(P, g, twp, st);
      return;
    }
  }
  const cpx<T>* twp = reinterpret_cast<const cpx<T>*>(tw);
  if constexpr (std::is_same<T, dd>::value) {
    if (choice != kChoiceUnpacked && p_plan_ok(g.px, kThreads / L)) {
      // the packed twiddle tables: 3 m + 2 (m + 1) entries against 2 m + 2
      const size_t psmem = smem + sizeof(pdd) * (size_t)(3 * m);
      // four blocks per SM (64 registers) where their shared memory fits, else three
      const bool four = 4 * (psmem + 1024) <= 228 * 1024;
      if (cv && four) launch_k_xpass<T, true, true, 4>(P, g, twp, L, blocks, psmem, st);
      else if (cv) launch_k_xpass<T, true, true, 3>(P, g, twp, L, blocks, psmem, st);
      else if (four) launch_k_xpass<T, false, true, 4>(P, g, twp, L, blocks, psmem, st);
      else launch_k_xpass<T, false, true, 3>(P, g, twp, L, blocks, psmem, st);
      return;
    }
  }
  if (cv) launch_k_xpass<T, true, false>(P, g, twp, L, blocks, smem, st);
  else launch_k_xpass<T, false, false>(P, g, twp, L, blocks, smem, st);
}

template void launch_axis<dd>(const AxisProg&, int, const GridDesc&, const void*, cudaStream_t);
template void launch_xpass<dd>(const XProg&, const GridDesc&, const void*, cudaStream_t);
template void launch_axis<double>(const AxisProg&, int, const GridDesc&, const void*, cudaStream_t);
template void launch_axis<float>(const AxisProg&, int, const GridDesc&, const void*, cudaStream_t);
template void launch_xpass<double>(const XProg&, const GridDesc&, const void*, cudaStream_t);
template void launch_xpass<float>(const XProg&, const GridDesc&, const void*, cudaStream_t);
template size_t axis_smem_bytes<double>(const GridDesc&, int);
template size_t axis_smem_bytes<dd>(const GridDesc&, int);
template size_t xpass_smem_bytes<dd>(const GridDesc&);
template size_t axis_smem_bytes<float>(const GridDesc&, int);
template size_t xpass_smem_bytes<double>(const GridDesc&);
template size_t xpass_smem_bytes<float>(const GridDesc&);

}  // namespace vd
