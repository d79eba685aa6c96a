// Transform pass kernels: strided-axis passes (y, z) and the fused contiguous x pass.
#include "vd_passes.cuh"
#include "vd_fft.cuh"
#include "vd_prof.h"

#include <cmath>

#include <algorithm>

namespace vd {

constexpr int kThreads = 256;
template <typename T>
constexpr int kEPT = (sizeof(T) == 8) ? 8 : 16;   // tile elements per thread

static inline int tile_width(int n, int ept) {
  int w = 1;
  while (w < 64 && (2 * w) * n <= ept * kThreads) w *= 2;
  return w;
}
static inline int lines_per_cta(int m, int ept) {
  int l = 1;
  while (l < 64 && (2 * l) * m <= ept * kThreads / 2) l *= 2;
  return l;
}

// ---------------------------------------------------------------------------------------
// strided axis pass
// ---------------------------------------------------------------------------------------

template <typename T, int S>
__global__ void __launch_bounds__(kThreads) k_axis(const AxisProg P, const GridDesc g,
                                                   const cpx<T>* __restrict__ twg, int W) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int EPT = kEPT<T>;
  const int axis = P.axis;
  const FftPlan& pl = (axis == 2) ? g.pz : g.py;
  const int n = pl.n;
  cpx<T>* tw = reinterpret_cast<cpx<T>*>(smem_raw);
  cpx<T>* A = tw + n;
  cpx<T>* B = A + W * n;
  const int tid = threadIdx.x;
  for (int j = tid; j < n; j += kThreads) tw[j] = twg[pl.tw_off + j];

  long long line_stride, inner_n, outer_stride;
  if (axis == 2) {
    line_stride = (long long)g.n1 * g.h0;
    inner_n = line_stride;
    outer_stride = 0;
  } else {
    line_stride = g.h0;
    inner_n = g.h0;
    outer_stride = (long long)g.n1 * g.h0;
  }
  const long long tiles = (inner_n + W - 1) / W;
  const long long o = blockIdx.x / tiles;
  const long long col0 = (blockIdx.x % tiles) * W;
  const int tile_elems = W * n;
  const T* __restrict__ symarr = reinterpret_cast<const T*>(P.symarr);
  if (P.done && *P.done) return;

  // global offset of tile element e (or -1 outside the field)
  auto gofs = [&](int e) -> long long {
    const int i = e / W;
    const long long col = col0 + (e - i * W);
    return (e < tile_elems && col < inner_n) ? (o * outer_stride + i * line_stride + col) : -1;
  };
  // real factor of a multiplier at tile element e (global offset go >= 0)
  auto mult = [&](int flags, int e, long long go, T base) -> T {
    const int i = e / W;
    const long long col = col0 + (e - i * W);
    const T ka = (T)g.kfac[axis] * (T)freq_tilde(i, n);
    T c = base;
    if (flags & MUL_IK) c *= ka;
    if (flags & MUL_IK2) c *= -ka * ka;
    if (flags & MUL_SYM) c *= symarr[go];
    if (flags & MUL_NEGK2) {
      T kk = ka * ka;
      if (axis == 2) {
        const int kyi = (int)(col / g.h0);
        const int kxi = (int)(col - (long long)kyi * g.h0);
        const T kx = (T)g.kfac[0] * (T)freq_tilde(kxi, g.n0);
        const T ky = (T)g.kfac[1] * (T)freq_tilde(kyi, g.n1);
        kk += kx * kx + ky * ky;
      } else {
        const T kx = (T)g.kfac[0] * (T)freq_tilde((int)col, g.n0);
        kk += kx * kx;
        if (g.ndim == 3) {
          const T kz = (T)g.kfac[2] * (T)freq_tilde((int)o, g.n2);
          kk += kz * kz;
        }
      }
      c *= -kk;
    }
    return c;
  };

  cpx<T> acc[EPT];
#pragma unroll
  for (int q = 0; q < EPT; ++q) acc[q] = mk<T>(T(0), T(0));

  for (int t = 0; t < P.nxf; ++t) {
    const Xf xf = P.xf[t];
    const cpx<T>* __restrict__ src = reinterpret_cast<const cpx<T>*>(P.in[xf.src]);
    const T scale = (T)xf.scale;
    if (xf.nofft) {
#pragma unroll
      for (int q = 0; q < EPT; ++q) {
        const int e = tid + q * kThreads;
        const long long go = gofs(e);
        cpx<T> v = mk<T>(T(0), T(0));
        if (go >= 0) {
          v = scal(src[go], mult(xf.pre, e, go, scale));
          if (xf.pre & MUL_IK) v = mul_i(v);
        }
        acc[q] = xf.first ? v : (acc[q] + v);
      }
    } else {
      __syncthreads();
#pragma unroll
      for (int q = 0; q < EPT; ++q) {
        const int e = tid + q * kThreads;
        if (e < tile_elems) {
          const long long go = gofs(e);
          cpx<T> v = mk<T>(T(0), T(0));
          if (go >= 0) {
            v = src[go];
            if (xf.pre) {
              v = scal(v, mult(xf.pre, e, go, T(1)));
              if (xf.pre & MUL_IK) v = mul_i(v);
            }
          }
          A[e] = v;
        }
      }
      cpx<T>* res = fft_pingpong<T, S, true>(A, B, W, 1, W, pl, tw, tid, kThreads);
#pragma unroll
      for (int q = 0; q < EPT; ++q) {
        const int e = tid + q * kThreads;
        cpx<T> v = mk<T>(T(0), T(0));
        const long long go = gofs(e);
        if (go >= 0) {
          v = res[e];
          if (xf.post) {
            v = scal(v, mult(xf.post, e, go, scale));
            if (xf.post & MUL_IK) v = mul_i(v);
          } else {
            v = scal(v, scale);
          }
        }
        acc[q] = xf.first ? v : (acc[q] + v);
      }
    }
    if (xf.last) {
      cpx<T>* __restrict__ dst = reinterpret_cast<cpx<T>*>(P.out[xf.dst]);
#pragma unroll
      for (int q = 0; q < EPT; ++q) {
        const long long go = gofs(tid + q * kThreads);
        if (go >= 0) dst[go] = acc[q];
      }
    }
  }
}

// ---------------------------------------------------------------------------------------
// contiguous x pass (real <-> half spectrum through a complex FFT of length n0/2)
// ---------------------------------------------------------------------------------------

template <typename T>
__global__ void __launch_bounds__(kThreads) k_xpass(const XProg P, const GridDesc g,
                                                    const cpx<T>* __restrict__ twg, int LPC) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int m = g.n0 / 2;
  const int h0 = g.h0;
  const int ls = m + 1;
  cpx<T>* twm = reinterpret_cast<cpx<T>*>(smem_raw);
  cpx<T>* pk = twm + m;
  cpx<T>* A = pk + (m + 2);   // keep 16-byte alignment (m even)
  cpx<T>* B = A + LPC * ls;
  const int tid = threadIdx.x;
  for (int j = tid; j < m; j += kThreads) twm[j] = twg[g.px.tw_off + j];
  for (int j = tid; j <= m; j += kThreads) pk[j] = twg[g.pk_off + j];

  const long long nlines = (long long)g.n1 * g.n2;
  const long long line0 = (long long)blockIdx.x * LPC;
  const int nl = (int)min((long long)LPC, nlines - line0);
  const T kfx = (T)g.kfac[0];
  const T scale = (T)P.scale;
  const T* __restrict__ symarr = reinterpret_cast<const T*>(P.symarr) + line0 * h0;
  if (P.done && *P.done) return;

  for (int c = 0; c < P.ncomp; ++c) {
    cpx<T>* res;
    __syncthreads();
    if (P.mode == 1) {
      const cpx<T>* __restrict__ src = reinterpret_cast<const cpx<T>*>(P.in[c]) + line0 * m;
      for (int e = tid; e < nl * m; e += kThreads) {
        const int line = e / m, j = e - line * m;
        A[line * ls + j] = src[e];
      }
      res = fft_pingpong<T, -1, false>(A, B, 1, ls, nl, g.px, twm, tid, kThreads);
    } else {
      const cpx<T>* __restrict__ src = reinterpret_cast<const cpx<T>*>(P.in[c]) + line0 * h0;
      const int pre = P.pre[c];
      for (int e = tid; e < nl * h0; e += kThreads) {
        const int line = e / h0, k = e - line * h0;
        cpx<T> v = src[e];
        if (pre) {
          const T kx = kfx * (T)freq_tilde(k, g.n0);
          T cc = T(1);
          if (pre & MUL_IK) cc *= kx;
          if (pre & MUL_SYM) cc *= symarr[e];
          if (pre & (MUL_NEGK2 | MUL_IK2)) cc *= -kx * kx;
          v = scal(v, cc);
          if (pre & MUL_IK) v = mul_i(v);
        }
        B[line * ls + k] = v;
      }
      __syncthreads();
      // pack the half spectrum into a length-m complex spectrum (inverse real transform)
      for (int e = tid; e < nl * m; e += kThreads) {
        const int line = e / m, k = e - line * m;
        const cpx<T> X = B[line * ls + k];
        const cpx<T> Xc = conjg(B[line * ls + (m - k)]);
        A[line * ls + k] = (X + Xc) + mul_i(cmulc(X - Xc, pk[k]));
      }
      res = fft_pingpong<T, +1, false>(A, B, 1, ls, nl, g.px, twm, tid, kThreads);
      if (P.mode == 2) {
        cpx<T>* __restrict__ dst = reinterpret_cast<cpx<T>*>(P.out[c]) + line0 * m;
        for (int e = tid; e < nl * m; e += kThreads) {
          const int line = e / m, j = e - line * m;
          dst[e] = scal(res[line * ls + j], scale);
        }
        continue;
      }
      if (P.wfield) {
        const cpx<T>* __restrict__ wf = reinterpret_cast<const cpx<T>*>(P.wfield) + line0 * m;
        for (int e = tid; e < nl * m; e += kThreads) {
          const int line = e / m, j = e - line * m;
          const cpx<T> z = res[line * ls + j];
          const cpx<T> w = wf[e];
          res[line * ls + j] = mk<T>(z.x * w.x, z.y * w.y);
        }
      }
      cpx<T>* other = (res == A) ? B : A;
      res = fft_pingpong<T, -1, false>(res, other, 1, ls, nl, g.px, twm, tid, kThreads);
    }
    // unpack the length-m spectrum into the half spectrum of the real line
    cpx<T>* __restrict__ dst = reinterpret_cast<cpx<T>*>(P.out[c]) + line0 * h0;
    const int post = P.post[c];
    for (int e = tid; e < nl * h0; e += kThreads) {
      const int line = e / h0, k = e - line * h0;
      const cpx<T> Z = res[line * ls + (k == m ? 0 : k)];
      const cpx<T> Zc = conjg(res[line * ls + (k == 0 ? 0 : m - k)]);
      cpx<T> X = (Z + Zc) - mul_i(cmul(Z - Zc, pk[k]));
      T cc = scale;
      const T kx = kfx * (T)freq_tilde(k, g.n0);
      if (post & MUL_IK) cc *= kx;
      if (post & MUL_SYM) cc *= symarr[e];
      if (post & (MUL_NEGK2 | MUL_IK2)) cc *= -kx * kx;
      X = scal(X, cc);
      if (post & MUL_IK) X = mul_i(X);
      dst[e] = X;
    }
  }
}

// ---------------------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------------------

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

template <typename T, int S>
static void set_axis_attr(size_t smem) {
  static size_t done = 0;
  if (smem > 48 * 1024 && smem > done) {
    cudaFuncSetAttribute(k_axis<T, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    done = smem;
  }
}

template <typename T>
void launch_axis(const AxisProg& P, int dir, const GridDesc& g, const void* tw, cudaStream_t st) {
  const int n = (P.axis == 2) ? g.pz.n : g.py.n;
  const int W = tile_width(n, kEPT<T>);
  long long inner_n, outer_n;
  if (P.axis == 2) {
    inner_n = (long long)g.n1 * g.h0;
    outer_n = 1;
  } else {
    inner_n = g.h0;
    outer_n = g.n2;
  }
  const long long blocks = outer_n * ((inner_n + W - 1) / W);
  const size_t smem = axis_smem_bytes<T>(g, P.axis);
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
  ProfScope ps(sizeof(T) == 8 ? PC_AXIS64 : PC_AXIS32, st, bytes, flops);
  if (dir < 0) {
    set_axis_attr<T, -1>(smem);
    k_axis<T, -1><<<(unsigned)blocks, kThreads, smem, st>>>(P, g, twp, W);
  } else {
    set_axis_attr<T, +1>(smem);
    k_axis<T, +1><<<(unsigned)blocks, kThreads, smem, st>>>(P, g, twp, W);
  }
}

template <typename T>
void launch_xpass(const XProg& P, const GridDesc& g, const void* tw, cudaStream_t st) {
  const int m = g.n0 / 2;
  const int L = lines_per_cta(m, kEPT<T>);
  const long long nlines = (long long)g.n1 * g.n2;
  const long long blocks = (nlines + L - 1) / L;
  const size_t smem = xpass_smem_bytes<T>(g);
  static size_t done = 0;
  if (smem > 48 * 1024 && smem > done) {
    cudaFuncSetAttribute(k_xpass<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    done = smem;
  }
  const double fc = (double)g.ncplx * sizeof(cpx<T>), fr = (double)g.nreal * sizeof(T);
  double bytes = 0, flops = 0;
  const double real_fft = (double)g.nreal * 2.5 * std::log2((double)g.n0);   // one real transform of every line
  if (P.mode == 0) {
    bytes = P.ncomp * 2.0 * fc + (P.wfield ? fr : 0.0);
    flops = P.ncomp * 2.0 * real_fft;
  } else {
    bytes = P.ncomp * (fc + fr);
    flops = P.ncomp * real_fft;
  }
  bool sym = false;
  for (int c = 0; c < P.ncomp; ++c) sym = sym || ((P.pre[c] | P.post[c]) & MUL_SYM);
  if (sym) bytes += (double)g.ncplx * sizeof(T);
  ProfScope ps(sizeof(T) == 8 ? PC_XPASS64 : PC_XPASS32, st, bytes, flops);
  k_xpass<T><<<(unsigned)blocks, kThreads, smem, st>>>(P, g, reinterpret_cast<const cpx<T>*>(tw), L);
}

template void launch_axis<double>(const AxisProg&, int, const GridDesc&, const void*, cudaStream_t);
template void launch_axis<float>(const AxisProg&, int, const GridDesc&, const void*, cudaStream_t);
template void launch_xpass<double>(const XProg&, const GridDesc&, const void*, cudaStream_t);
template void launch_xpass<float>(const XProg&, const GridDesc&, const void*, cudaStream_t);
template size_t axis_smem_bytes<double>(const GridDesc&, int);
template size_t axis_smem_bytes<float>(const GridDesc&, int);
template size_t xpass_smem_bytes<double>(const GridDesc&);
template size_t xpass_smem_bytes<float>(const GridDesc&);

}  // namespace vd
