// Krylov solvers: CG, restarted GMRES (CGS2 Arnoldi) and Richardson Minimal Residual.
//
// Every reduction is a two-level deterministic sum in double precision: a fixed number of
// blocks writes per-block partials, and the last block to finish (atomic ticket) adds them
// in a fixed order and runs the scalar epilogue of the algorithm (step lengths, Givens
// rotations, convergence tests) in one thread.  The scalars never leave the device; the
// host only reads the `done` flag every `check_every` iterations, and (CG, RMR) one batch
// behind: it waits for the flag of batch k-1 with batch k already queued.  Kernels of an
// iteration return at once when the flag is set, so iterations enqueued ahead cost a launch
// each and change nothing.
#include "vd_krylov.cuh"
#include "vd_prof.h"

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstring>
#include <vector>
#include <mutex>

namespace vd {

// ---------------------------------------------------------------------------------------
// reduction machinery
// ---------------------------------------------------------------------------------------

__device__ __forceinline__ double wgt(long long e, int h0) {
  const int kx = (int)(e % h0);
  return (kx == 0 || kx == h0 - 1) ? 1.0 : 2.0;
}

template <typename T>
__device__ __forceinline__ cpx<double> ld(const cpx<T>* p, long long e) {
  const cpx<T> v = p[e];
  return mk<double>((double)v.x, (double)v.y);
}

// Block-sum v[0..NV) into per-block partials; the last block gets the totals in thread 0.
// Returns true (in every thread of the last block) when the caller must run the epilogue.
template <int NV>
__device__ bool reduce_last(double (&v)[NV], double* partials, unsigned* counter, double (&tot)[NV]) {
  __shared__ double sm[NV][kRedThreads / 32];
  __shared__ int am_last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    double s = v[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) sm[i][warp] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      double s = 0.0;
      for (int w = 0; w < kRedThreads / 32; ++w) s += sm[i][w];
      partials[blockIdx.x * NV + i] = s;
    }
    __threadfence();
    const unsigned t = atomicAdd(counter, 1u);
    am_last = (t == gridDim.x - 1) ? 1 : 0;
  }
  __syncthreads();
  if (!am_last) return false;
  __threadfence();
  double a[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) a[i] = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
#pragma unroll
    for (int i = 0; i < NV; ++i) a[i] += __ldcg(partials + b * NV + i);
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    double s = a[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) sm[i][warp] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      double s = 0.0;
      for (int w = 0; w < kRedThreads / 32; ++w) s += sm[i][w];
      tot[i] = s;
    }
    *counter = 0u;
  }
  return true;
}

static inline int red_blocks(long long len) {
  return (int)std::max<long long>(1, std::min<long long>(kRedBlocks, (len + kRedThreads - 1) / kRedThreads));
}

#define GRID_STRIDE(e, len) \
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < (len); e += (long long)gridDim.x * blockDim.x)

__device__ __forceinline__ bool bad(double v) { return !isfinite(v); }

__device__ void finish(KState* ks, int status) {
  ks->status = status;
  ks->done = 1;
  ks->cycle_done = 1;
}

__device__ void record(KState* ks, double* hist, double rel) {
  if (ks->iters < ks->hist_cap) hist[ks->iters] = rel;
}

// ---------------------------------------------------------------------------------------
// epilogues
// ---------------------------------------------------------------------------------------

enum Epi : int {
  EPI_INIT_CG = 0,    // tot = [bb, rr, rz]
  EPI_CG_ALPHA = 1,   // tot = [pq]
  EPI_CG_UPDATE = 2,  // tot = [rr, rz]
  EPI_INIT_RMR = 3,   // tot = [bb, rr]
  EPI_RMR_ALPHA = 4,  // tot = [rw, ww]
  EPI_RMR_UPDATE = 5, // tot = [rr]
  EPI_BB = 6,         // tot = [bb]
  EPI_GM_BETA = 7,    // tot = [rr]
  EPI_GM_H1 = 8,      // tot[i] -> h1[off + i]
  EPI_GM_H2 = 9,      // tot[i] -> h2[off + i]
  EPI_GM_NORM = 10,   // tot = [ww]
  EPI_NORM = 11,      // tot = [vv] -> ks->rr
};

template <int NV>
__device__ void epilogue(int epi, const double (&t)[NV], KState* ks, double* hist, double tol, int off, int j) {
  if (tol < 0.0) tol = ks->dtol;
  switch (epi) {
    case EPI_INIT_CG:
    case EPI_INIT_RMR: {
      ks->bb = t[0];
      ks->tol2bb = tol * tol * t[0];
      if (t[0] == 0.0) {
        ks->relres = 0.0;
        record(ks, hist, 0.0);
        finish(ks, 0);
        return;
      }
      const double rel = sqrt(t[1] / t[0]);
      ks->relres = rel;
      ks->best = rel;
      ks->ref = rel;
      ks->ref_it = 0;
      ks->rr = t[1];
      if (epi == EPI_INIT_CG) ks->rz = t[NV > 2 ? 2 : 0];
      record(ks, hist, rel);
      if (bad(rel)) finish(ks, VD_ERR_NONFINITE);
      else if (rel <= tol) finish(ks, 0);
      else if (ks->maxit <= 0) finish(ks, VD_ERR_NOT_CONVERGED);
      return;
    }
    case EPI_CG_ALPHA: {
      const double pq = t[0];
      ks->pq = pq;
      if (pq == 0.0 || ks->rz == 0.0) {
        ks->iters += 1;
        finish(ks, VD_ERR_BREAKDOWN);
        return;
      }
      ks->alpha = ks->rz / pq;
      if (bad(ks->alpha)) {
        ks->iters += 1;
        finish(ks, VD_ERR_NONFINITE);
      }
      return;
    }
    case EPI_CG_UPDATE:
    case EPI_RMR_UPDATE: {
      ks->iters += 1;
      const double rr = t[0];
      const double rel = sqrt(rr / ks->bb);
      ks->rr = rr;
      ks->relres = rel;
      record(ks, hist, rel);
      if (bad(rel)) {
        finish(ks, VD_ERR_NONFINITE);
        return;
      }
      if (rr <= ks->tol2bb) {
        finish(ks, 0);
        return;
      }
      // residual-growth divergence test: RMR only (CG's residual norm is not monotone), except
      // for guarded CG solves that have already converged well below their start
      if (epi == EPI_RMR_UPDATE && rel > 1e3 * ks->best) {
        finish(ks, VD_ERR_DIVERGED);
        return;
      }
      if (epi == EPI_CG_UPDATE && ks->guard > 0) {
        if (rel < 0.5 * ks->ref) {
          ks->ref = rel;
          ks->ref_it = ks->iters;
        } else if (ks->best < 1e-3 && ks->iters - ks->ref_it >= kStallWindow) {
          finish(ks, VD_ERR_DIVERGED);   // stalled at its attainable accuracy
          return;
        }
        if (ks->best < 1e-3 && rel > (double)ks->guard * ks->best) {
          finish(ks, VD_ERR_DIVERGED);
          return;
        }
      }
      ks->best = fmin(ks->best, rel);
      if (epi == EPI_CG_UPDATE) {
        const double rz = t[NV > 1 ? 1 : 0];
        ks->beta = rz / ks->rz;
        ks->rz = rz;
      }
      if (ks->iters >= ks->maxit) finish(ks, VD_ERR_NOT_CONVERGED);
      return;
    }
    case EPI_RMR_ALPHA: {
      const double ww = t[NV > 1 ? 1 : 0];
      ks->rw = t[0];
      ks->ww = ww;
      if (ww == 0.0) {
        ks->iters += 1;
        finish(ks, VD_ERR_BREAKDOWN);
        return;
      }
      ks->alpha = t[0] / ww;
      return;
    }
    case EPI_BB: {
      ks->bb = t[0];
      ks->tol2bb = tol * tol * t[0];
      return;
    }
    case EPI_GM_BETA: {
      const double beta = sqrt(t[0]);
      ks->beta0 = beta;
      if (ks->bb == 0.0) {
        ks->relres = 0.0;
        if (ks->iters == 0) record(ks, hist, 0.0);
        finish(ks, 0);
        return;
      }
      const double rel = beta / sqrt(ks->bb);
      if (ks->iters == 0) record(ks, hist, rel);
      ks->relres = rel;
      if (bad(rel)) finish(ks, VD_ERR_NONFINITE);
      else if (rel <= tol) finish(ks, 0);
      else if (ks->iters >= ks->maxit) finish(ks, VD_ERR_NOT_CONVERGED);
      else {
        ks->k = 0;
        ks->cycle_done = 0;
        ks->gv[0] = beta;
      }
      return;
    }
    case EPI_GM_H1:
    case EPI_GM_H2: {
      double* h = (epi == EPI_GM_H1) ? ks->h1 : ks->h2;
      for (int i = 0; i < NV; ++i)
        if (off + i <= j) h[off + i] = t[i];
      return;
    }
    case EPI_GM_NORM: {
      const int m = ks->m;
      const double hn = sqrt(t[0]);
      double* col = ks->H + (size_t)j * (m + 1);
      for (int i = 0; i <= j; ++i) col[i] = ks->h1[i] + ks->h2[i];
      col[j + 1] = hn;
      for (int i = 0; i < j; ++i) {
        const double a = ks->cs[i] * col[i] + ks->sn[i] * col[i + 1];
        col[i + 1] = -ks->sn[i] * col[i] + ks->cs[i] * col[i + 1];
        col[i] = a;
      }
      double c = 1.0, s = 0.0;
      if (col[j + 1] != 0.0) {
        const double h = hypot(col[j], col[j + 1]);
        c = col[j] / h;
        s = col[j + 1] / h;
      }
      ks->cs[j] = c;
      ks->sn[j] = s;
      col[j] = c * col[j] + s * col[j + 1];
      col[j + 1] = 0.0;
      ks->gv[j + 1] = -s * ks->gv[j];
      ks->gv[j] = c * ks->gv[j];
      ks->iters += 1;
      ks->k = j + 1;
      const double est = fabs(ks->gv[j + 1]) / sqrt(ks->bb);
      ks->relres = est;
      record(ks, hist, est);
      ks->ww = hn;
      if (bad(est)) {
        ks->status = VD_ERR_NONFINITE;
        ks->cycle_done = 1;
      } else if (est <= tol || hn == 0.0) {
        ks->status = 0;   // converged (or invariant Krylov space): finished after the update
        ks->cycle_done = 1;
      } else if (j + 1 >= m || ks->iters >= ks->maxit) {
        ks->cycle_done = 1;
      }
      return;
    }
    case EPI_NORM: {
      ks->rr = t[0];
      return;
    }
  }
}

// ---------------------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------------------

struct RedArgs {
  KState* ks;
  double* partials;
  unsigned* counter;
  double* hist;
  double tol;
};

// Grid-stride iteration over a spectral vector that tracks, without any division inside
// the loop, kx = e mod h0 (Parseval weight) and the symbol index e mod ncplx.
struct Ix {
  int len, h0, nc;   // vector length (complex elements), x half-spectrum length, field size
  int sh, sn;        // grid stride mod h0, grid stride mod nc
};

#define IX_LOOP(ix)                                                                          \
  const int ix_s_ = gridDim.x * blockDim.x;                                                 \
  int e = blockIdx.x * blockDim.x + threadIdx.x;                                            \
  int kx = e % (ix).h0, si = e % (ix).nc;                                                   \
  for (; e < (ix).len; e += ix_s_, kx += (ix).sh, kx -= (kx >= (ix).h0) ? (ix).h0 : 0,      \
                       si += (ix).sn, si -= (si >= (ix).nc) ? (ix).nc : 0)

template <typename T>
__device__ __forceinline__ T pweight(int kx, int h0) {
  return (kx == 0 || kx == h0 - 1) ? T(1) : T(2);
}

// Per-thread accumulator of a reduction.  Double vectors add in double.  Float vectors add
// with a compensated float sum (Knuth's two-sum carries the rounding error of every addition
// in a second float), about as accurate as a double accumulation of the float terms but
// without FP64 work per element: the FP64 pipe of GB300 is ~1/64 of the float rate and was
// the limiter of these memory-bound kernels.  The cross-thread sum of the per-thread totals
// is done in double (reduce_last).
template <typename T>
struct Acc {
  double a = 0.0;
  __device__ __forceinline__ void add(T v) { a += (double)v; }
  __device__ __forceinline__ double total() const { return a; }
};
template <>
struct Acc<float> {
  float s = 0.0f, c = 0.0f;   // value s + c
  __device__ __forceinline__ void add(float v) {
    const float t = s + v;
    const float bp = t - s;
    c += (s - (t - bp)) + (v - bp);
    s = t;
  }
  __device__ __forceinline__ double total() const { return (double)s + (double)c; }
};

// CG start: p = S r, reduce [bb, rr, rz]
template <typename T>
__global__ void __launch_bounds__(kRedThreads) k_cg_init(Ix ix, const cpx<T>* __restrict__ b,
                                                         const cpx<T>* __restrict__ r, cpx<T>* __restrict__ p,
                                                         const T* __restrict__ sym, RedArgs ra) {
  Acc<T> a0, a1, a2;
  IX_LOOP(ix) {
    const T w = pweight<T>(kx, ix.h0);
    const cpx<T> bv = b[e], rv = r[e];
    const T sv = sym[si];
    p[e] = scal(rv, sv);
    const T r2 = rv.x * rv.x + rv.y * rv.y;
    a0.add(w * (bv.x * bv.x + bv.y * bv.y));
    a1.add(w * r2);
    a2.add(w * sv * r2);
  }
  double v[3] = {a0.total(), a1.total(), a2.total()};
  double t[3];
  if (reduce_last<3>(v, ra.partials, ra.counter, t) && threadIdx.x == 0)
    epilogue<3>(EPI_INIT_CG, t, ra.ks, ra.hist, ra.tol, 0, 0);
}

// reduce [(u,v)_w] or [(u,v)_w, (v,v)_w]
template <typename T, int NV>
__global__ void __launch_bounds__(kRedThreads) k_dot(Ix ix, const cpx<T>* __restrict__ u,
                                                     const cpx<T>* __restrict__ v, int epi, RedArgs ra,
                                                     const int* done) {
  if (*done) return;
  Acc<T> a0, a1;
  IX_LOOP(ix) {
    const T w = pweight<T>(kx, ix.h0);
    const cpx<T> uu = u[e], vv = v[e];
    a0.add(w * (uu.x * vv.x + uu.y * vv.y));
    if (NV > 1) a1.add(w * (vv.x * vv.x + vv.y * vv.y));
  }
  double a[NV];
  a[0] = a0.total();
  if (NV > 1) a[NV - 1] = a1.total();
  double t[NV];
  if (reduce_last<NV>(a, ra.partials, ra.counter, t) && threadIdx.x == 0)
    epilogue<NV>(epi, t, ra.ks, ra.hist, ra.tol, 0, 0);
}

// CG: x += alpha p, r -= alpha q; reduce [rr, (r, S r)]
template <typename T>
__global__ void __launch_bounds__(kRedThreads) k_cg_update(Ix ix, cpx<T>* __restrict__ x,
                                                           const cpx<T>* __restrict__ p, cpx<T>* __restrict__ r,
                                                           const cpx<T>* __restrict__ q, const T* __restrict__ sym,
                                                           RedArgs ra) {
  if (ra.ks->done) return;
  const T al = (T)ra.ks->alpha;
  Acc<T> a0, a1;
  IX_LOOP(ix) {
    const T w = pweight<T>(kx, ix.h0);
    const cpx<T> pv = p[e], qv = q[e];
    cpx<T> xv = x[e], rv = r[e];
    xv = mk<T>(fma(al, pv.x, xv.x), fma(al, pv.y, xv.y));
    rv = mk<T>(fma(-al, qv.x, rv.x), fma(-al, qv.y, rv.y));
    x[e] = xv;
    r[e] = rv;
    const T r2 = rv.x * rv.x + rv.y * rv.y;
    a0.add(w * r2);
    a1.add(w * sym[si] * r2);
  }
  double v[2] = {a0.total(), a1.total()};
  double t[2];
  if (reduce_last<2>(v, ra.partials, ra.counter, t) && threadIdx.x == 0)
    epilogue<2>(EPI_CG_UPDATE, t, ra.ks, ra.hist, ra.tol, 0, 0);
}

// CG: p = S r + beta p
template <typename T>
__global__ void k_cg_p(Ix ix, cpx<T>* __restrict__ p, const cpx<T>* __restrict__ r, const T* __restrict__ sym,
                       const KState* ks) {
  if (ks->done) return;
  const T be = (T)ks->beta;
  IX_LOOP(ix) {
    const T sv = sym[si];
    const cpx<T> rv = r[e], pv = p[e];
    p[e] = mk<T>(fma(be, pv.x, sv * rv.x), fma(be, pv.y, sv * rv.y));
  }
}

// RMR / GMRES start: reduce [bb, rr] or [rr]
template <typename T, int NV>
__global__ void __launch_bounds__(kRedThreads) k_norms(Ix ix, const cpx<T>* __restrict__ b,
                                                       const cpx<T>* __restrict__ r, int epi, RedArgs ra,
                                                       const int* done) {
  if (done && *done) return;
  Acc<T> a0, a1;
  IX_LOOP(ix) {
    const T w = pweight<T>(kx, ix.h0);
    const cpx<T> rv = r[e];
    if (NV == 2) {
      const cpx<T> bv = b[e];
      a0.add(w * (bv.x * bv.x + bv.y * bv.y));
    }
    a1.add(w * (rv.x * rv.x + rv.y * rv.y));
  }
  double v[NV];
  if (NV == 2) v[0] = a0.total();
  v[NV - 1] = a1.total();
  double t[NV];
  if (reduce_last<NV>(v, ra.partials, ra.counter, t) && threadIdx.x == 0)
    epilogue<NV>(epi, t, ra.ks, ra.hist, ra.tol, 0, 0);
}

// weighted (Parseval) inner product of two spectral vectors -> ks->rr
template <typename T>
__global__ void __launch_bounds__(kRedThreads) k_pdot(Ix ix, const cpx<T>* __restrict__ a,
                                                      const cpx<T>* __restrict__ b, RedArgs ra) {
  Acc<T> a0;
  IX_LOOP(ix) {
    const cpx<T> u = a[e], v = b[e];
    a0.add(pweight<T>(kx, ix.h0) * (u.x * v.x + u.y * v.y));
  }
  double v[1] = {a0.total()};
  double t[1];
  if (reduce_last<1>(v, ra.partials, ra.counter, t) && threadIdx.x == 0) epilogue<1>(EPI_NORM, t, ra.ks, ra.hist, ra.tol, 0, 0);
}

// r = b - q and |r|^2 (weighted) -> ks->rr, accumulated like k_norms
template <typename T>
__global__ void __launch_bounds__(kRedThreads) k_sub_norm(Ix ix, const cpx<T>* __restrict__ b,
                                                          const cpx<T>* __restrict__ q, cpx<T>* __restrict__ r,
                                                          RedArgs ra) {
  Acc<T> a1;
  IX_LOOP(ix) {
    const cpx<T> rv = b[e] - q[e];
    r[e] = rv;
    a1.add(pweight<T>(kx, ix.h0) * (rv.x * rv.x + rv.y * rv.y));
  }
  double v[1] = {a1.total()};
  double t[1];
  if (reduce_last<1>(v, ra.partials, ra.counter, t) && threadIdx.x == 0) epilogue<1>(EPI_NORM, t, ra.ks, ra.hist, ra.tol, 0, 0);
}

// RMR: x += alpha S r, r -= alpha w; reduce [rr]
template <typename T>
__global__ void __launch_bounds__(kRedThreads) k_rmr_update(Ix ix, cpx<T>* __restrict__ x, cpx<T>* __restrict__ r,
                                                            const cpx<T>* __restrict__ wv, const T* __restrict__ sym,
                                                            RedArgs ra) {
  if (ra.ks->done) return;
  const T al = (T)ra.ks->alpha;
  Acc<T> a0;
  IX_LOOP(ix) {
    const T w = pweight<T>(kx, ix.h0);
    const T as = al * sym[si];
    const cpx<T> wq = wv[e];
    cpx<T> xv = x[e], rv = r[e];
    xv = mk<T>(fma(as, rv.x, xv.x), fma(as, rv.y, xv.y));
    rv = mk<T>(fma(-al, wq.x, rv.x), fma(-al, wq.y, rv.y));
    x[e] = xv;
    r[e] = rv;
    a0.add(w * (rv.x * rv.x + rv.y * rv.y));
  }
  double v[1] = {a0.total()};
  double t[1];
  if (reduce_last<1>(v, ra.partials, ra.counter, t) && threadIdx.x == 0)
    epilogue<1>(EPI_RMR_UPDATE, t, ra.ks, ra.hist, ra.tol, 0, 0);
}

// GMRES: dst = src / beta0 (first basis vector) or src / H[j+1,j] (next)
template <typename T>
__global__ void k_gm_scale(Ix ix, cpx<T>* __restrict__ dst, const cpx<T>* __restrict__ src, const KState* ks,
                           int first) {
  if (ks->cycle_done) return;
  const T s = (T)(1.0 / (first ? ks->beta0 : ks->ww));
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < ix.len; e += gridDim.x * blockDim.x)
    dst[e] = scal(src[e], s);
}

// GMRES: h[off + i] = (w, V_{off+i})_w for i < nv (<= 8)
template <typename T>
__global__ void __launch_bounds__(kRedThreads) k_gm_mdot(Ix ix, const cpx<T>* __restrict__ w,
                                                         const cpx<T>* __restrict__ V, int off, int nv, int epi, int j,
                                                         RedArgs ra) {
  if (ra.ks->cycle_done) return;
  Acc<T> a[8];
  IX_LOOP(ix) {
    const T wt = pweight<T>(kx, ix.h0);
    const cpx<T> wv = w[e];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      if (i < nv) {
        const cpx<T> vv = V[(size_t)(off + i) * ix.len + e];
        a[i].add(wt * (wv.x * vv.x + wv.y * vv.y));
      }
    }
  }
  double v[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = a[i].total();
  double t[8];
  if (reduce_last<8>(v, ra.partials, ra.counter, t) && threadIdx.x == 0)
    epilogue<8>(epi, t, ra.ks, ra.hist, ra.tol, off, j);
}

// GMRES: w -= sum_{i<=j} h_i V_i (h = h1 or h2); with_norm: reduce [(w,w)] -> EPI_GM_NORM
template <typename T>
__global__ void __launch_bounds__(kRedThreads) k_gm_maxpy(Ix ix, cpx<T>* __restrict__ w,
                                                          const cpx<T>* __restrict__ V, int j, int which, int with_norm,
                                                          RedArgs ra) {
  if (ra.ks->cycle_done) return;
  __shared__ T hs[kMaxRestart + 1];
  const double* h = which ? ra.ks->h2 : ra.ks->h1;
  for (int i = threadIdx.x; i <= j; i += blockDim.x) hs[i] = (T)h[i];
  __syncthreads();
  Acc<T> a0;
  IX_LOOP(ix) {
    cpx<T> wv = w[e];
    for (int i = 0; i <= j; ++i) {
      const T c = hs[i];
      const cpx<T> vv = V[(size_t)i * ix.len + e];
      wv = mk<T>(fma(-c, vv.x, wv.x), fma(-c, vv.y, wv.y));
    }
    w[e] = wv;
    a0.add(pweight<T>(kx, ix.h0) * (wv.x * wv.x + wv.y * wv.y));
  }
  if (!with_norm) return;
  double v[1] = {a0.total()};
  double t[1];
  if (reduce_last<1>(v, ra.partials, ra.counter, t) && threadIdx.x == 0)
    epilogue<1>(EPI_GM_NORM, t, ra.ks, ra.hist, ra.tol, 0, j);
}

// GMRES: back substitution H(0:k,0:k) y = g (one thread)
__global__ void k_gm_solve(KState* ks) {
  if (ks->done || threadIdx.x != 0 || blockIdx.x != 0) return;
  const int k = ks->k, m = ks->m;
  for (int i = k - 1; i >= 0; --i) {
    double s = ks->gv[i];
    for (int l = i + 1; l < k; ++l) s -= ks->H[i + (size_t)l * (m + 1)] * ks->y[l];
    ks->y[i] = s / ks->H[i + (size_t)i * (m + 1)];
  }
}

// GMRES: x += S sum_{i<k} y_i V_i
template <typename T>
__global__ void k_gm_update(Ix ix, cpx<T>* __restrict__ x, const cpx<T>* __restrict__ V, const T* __restrict__ sym,
                            const KState* ks) {
  if (ks->done) return;
  __shared__ T ys[kMaxRestart];
  const int k = ks->k;
  for (int i = threadIdx.x; i < k; i += blockDim.x) ys[i] = (T)ks->y[i];
  __syncthreads();
  IX_LOOP(ix) {
    T ax = T(0), ay = T(0);
    for (int i = 0; i < k; ++i) {
      const cpx<T> vv = V[(size_t)i * ix.len + e];
      ax = fma(ys[i], vv.x, ax);
      ay = fma(ys[i], vv.y, ay);
    }
    const T sv = sym[si];
    const cpx<T> xv = x[e];
    x[e] = mk<T>(fma(sv, ax, xv.x), fma(sv, ay, xv.y));
  }
}

// GMRES end of cycle: converged inside the cycle -> finished
__global__ void k_gm_close(KState* ks) {
  if (threadIdx.x != 0 || blockIdx.x != 0 || ks->done) return;
  if (ks->status == 0 || ks->status == VD_ERR_NONFINITE) ks->done = 1;
}

// ---------------------------------------------------------------------------------------
// small vector helpers
// ---------------------------------------------------------------------------------------

template <typename T>
__global__ void k_copy_scale(long long len, const cpx<T>* __restrict__ x, double s, cpx<T>* __restrict__ y) {
  GRID_STRIDE(e, len) {
    const cpx<double> v = ld(x, e);
    y[e] = mk<T>((T)(v.x * s), (T)(v.y * s));
  }
}
template <typename T>
__global__ void k_axpy(long long len, double a, const cpx<T>* __restrict__ x, cpx<T>* __restrict__ y) {
  GRID_STRIDE(e, len) {
    const cpx<double> v = ld(x, e), w = ld(y, e);
    y[e] = mk<T>((T)fma(a, v.x, w.x), (T)fma(a, v.y, w.y));
  }
}
template <typename T>
__global__ void k_sub(long long len, const cpx<T>* __restrict__ b, const cpx<T>* __restrict__ q,
                      cpx<T>* __restrict__ r, const int* done) {
  if (done && *done) return;
  GRID_STRIDE(e, len) { r[e] = b[e] - q[e]; }
}
// refinement steps fused over one pass of the double vectors (same arithmetic per element as
// the separate kernels): out = float(in * s) and y += a * double(xf); s and a come from the
// host, or from the refinement state (o->scale, o->rnorm) when o is set
__global__ void k_d2f_scaled(long long len, const cpx<double>* __restrict__ in, double s, const OState* o,
                             cpx<float>* __restrict__ out) {
  if (o) s = o->scale;
  GRID_STRIDE(e, len) {
    const cpx<double> v = in[e];
    out[e] = mk<float>((float)(v.x * s), (float)(v.y * s));
  }
}
__global__ void k_axpy_f2d(long long len, double a, const OState* o, const cpx<float>* __restrict__ xf,
                           cpx<double>* __restrict__ y) {
  if (o) a = o->rnorm;
  GRID_STRIDE(e, len) {
    const cpx<float> v = xf[e];
    const cpx<double> w = y[e];
    y[e] = mk<double>(fma(a, (double)v.x, w.x), fma(a, (double)v.y, w.y));
  }
}
template <typename T>
__global__ void k_project(GridDesc g, int ncomp, cpx<T>* v, double* removed) {
  const int t = threadIdx.x;   // one thread per corner mode and component
  const int d = g.ndim;
  const int ncorner = 1 << d;
  if (t >= ncorner * ncomp) return;
  const int c = t / ncorner, m = t % ncorner;
  const int kx = (m & 1) ? g.n0 / 2 : 0;
  const int ky = (d >= 2 && (m & 2)) ? g.n1 / 2 : 0;
  const int kz = (d >= 3 && (m & 4)) ? g.n2 / 2 : 0;
  const long long e = ((long long)kz * g.n1 + ky) * g.h0 + kx;
  cpx<T>* q = v + (long long)c * g.ncplx + e;
  // the removed coefficient's share of the squared norm (Parseval weight 1: kx is 0 or n0/2)
  if (removed) removed[t] = (double)q->x * (double)q->x + (double)q->y * (double)q->y;
  *q = mk<T>(T(0), T(0));
}

static inline Ix mkix(long long len, int h0, long long nc, int blocks, int threads) {
  const long long S = (long long)blocks * threads;
  Ix ix;
  ix.len = (int)len;
  ix.h0 = h0;
  ix.nc = (int)nc;
  ix.sh = (int)(S % h0);
  ix.sn = (int)(S % nc);
  return ix;
}

static inline int ew_blocks(long long len) {
  return (int)std::max<long long>(1, std::min<long long>((len + 255) / 256, 8 * 1024));
}

template <typename T>
void spec_copy_scale(long long len, const void* x, double s, void* y, cudaStream_t st) {
  { k_copy_scale<T><<<ew_blocks(len), 256, 0, st>>>(len, (const cpx<T>*)x, s, (cpx<T>*)y); count_launch(); }
}
template <typename T>
void spec_axpy(long long len, double a, const void* x, void* y, cudaStream_t st) {
  { k_axpy<T><<<ew_blocks(len), 256, 0, st>>>(len, a, (const cpx<T>*)x, (cpx<T>*)y); count_launch(); }
}
template <typename T>
void spec_sub(long long len, const void* b, const void* q, void* r, cudaStream_t st) {
  { ProfScope ps_(sizeof(T) == 4 ? PC_VEC32 : PC_VEC64, st, (double)3 * len * sizeof(cpx<T>), 0.0); k_sub<T><<<ew_blocks(len), 256, 0, st>>>(len, (const cpx<T>*)b, (const cpx<T>*)q, (cpx<T>*)r, nullptr); }
}
template <typename T>
void spec_project(const vd_grid* G, int ncomp, void* v, cudaStream_t st, double* removed) {
  { k_project<T><<<1, 32, 0, st>>>(G->g, ncomp, (cpx<T>*)v, removed); count_launch(); }
}

template <typename T>
double spec_norm2_host(const SpecSystem& sys, const void* v, const KWork& kw, cudaStream_t st) {
  RedArgs ra{kw.ks, kw.partials, kw.counter, kw.hist, 0.0};
  const int rb = red_blocks(sys.len);
  const Ix ix = mkix(sys.len, sys.h0, sys.G->g.ncplx, rb, kRedThreads);
  { ProfScope ps_(sizeof(T) == 4 ? PC_VEC32 : PC_VEC64, st, (double)1 * sys.len * sizeof(cpx<T>), 0.0); k_norms<T, 1><<<rb, kRedThreads, 0, st>>>(ix, nullptr, (const cpx<T>*)v, EPI_NORM, ra, nullptr); }
  double rr = 0.0;
  cudaMemcpyAsync(&rr, &kw.ks->rr, sizeof(double), cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  return rr;
}

template <typename T>
double spec_dot_host(const SpecSystem& sys, const void* a, const void* b, const KWork& kw, cudaStream_t st) {
  RedArgs ra{kw.ks, kw.partials, kw.counter, kw.hist, 0.0};
  const int rb = red_blocks(sys.len);
  const Ix ix = mkix(sys.len, sys.h0, sys.G->g.ncplx, rb, kRedThreads);
  { ProfScope ps_(sizeof(T) == 4 ? PC_VEC32 : PC_VEC64, st, (double)2 * sys.len * sizeof(cpx<T>), 0.0); k_pdot<T><<<rb, kRedThreads, 0, st>>>(ix, (const cpx<T>*)a, (const cpx<T>*)b, ra); }
  double rr = 0.0;
  cudaMemcpyAsync(&rr, &kw.ks->rr, sizeof(double), cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  return rr;
}

double spec_sub_norm2_host(const SpecSystem& sys, const void* b, const void* q, void* r, const KWork& kw,
                           cudaStream_t st) {
  RedArgs ra{kw.ks, kw.partials, kw.counter, kw.hist, 0.0};
  const int rb = red_blocks(sys.len);
  const Ix ix = mkix(sys.len, sys.h0, sys.G->g.ncplx, rb, kRedThreads);
  { ProfScope ps_(PC_VEC64, st, (double)3 * sys.len * sizeof(cpx<double>), 0.0); k_sub_norm<double><<<rb, kRedThreads, 0, st>>>(ix, (const cpx<double>*)b, (const cpx<double>*)q, (cpx<double>*)r, ra); }
  double rr = 0.0;
  cudaMemcpyAsync(&rr, &kw.ks->rr, sizeof(double), cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  return rr;
}

void spec_d2f_scaled(long long len, const void* in, double s, void* out, cudaStream_t st) {
  { ProfScope ps_(PC_VEC64, st, (double)len * (sizeof(cpx<double>) + sizeof(cpx<float>)), 0.0); k_d2f_scaled<<<ew_blocks(len), 256, 0, st>>>(len, (const cpx<double>*)in, s, nullptr, (cpx<float>*)out); }
}

void spec_axpy_f2d(long long len, double a, const void* xf, void* y, cudaStream_t st) {
  { ProfScope ps_(PC_VEC64, st, (double)len * (sizeof(cpx<float>) + 2 * sizeof(cpx<double>)), 0.0); k_axpy_f2d<<<ew_blocks(len), 256, 0, st>>>(len, a, nullptr, (const cpx<float>*)xf, (cpx<double>*)y); }
}

// ---------------------------------------------------------------------------------------
// host drivers
// ---------------------------------------------------------------------------------------

template <typename T>
size_t krylov_vec_bytes(const SpecSystem& sys, int solver, int restart) {
  const size_t v = sizeof(cpx<T>) * (size_t)sys.len;
  if (solver == VD_SOLVER_CG) return 3 * v;
  if (solver == VD_SOLVER_RMR) return 2 * v;
  const int m = restart > 0 ? restart : 30;
  return (size_t)(m + 2) * v;
}

struct KHead {   // host mirror of the first fields of KState
  double bb, tol2bb, rr, rz, pq, alpha, beta, rw, ww, best, relres;
  int iters, maxit, status, done, hist_cap, m, k, cycle_done, guard;
};
static_assert(offsetof(KState, bb) == 0, "layout");

static vd_status read_head(const KWork& kw, KHead* h, cudaStream_t st) {
  VD_CUDA(cudaMemcpyAsync(h, kw.ks, sizeof(KHead), cudaMemcpyDeviceToHost, st));
  VD_CUDA(cudaStreamSynchronize(st));
  return VD_OK;
}

// Convergence polling one batch behind: after enqueuing batch k the host waits for the head
// snapshot taken after batch k-1, so the device always has the next batch queued instead of
// idling while the host wakes up and launches.  Batches enqueued past convergence return at
// once (every kernel of an iteration checks the device `done` flag).  Two pinned snapshot
// slots and events per solve in flight, leased from a process-wide pool (server slots solve
// from several threads; the pool never shrinks, so it holds the peak number of concurrent
// solves).
struct HeadPipe {
  KHead* slot = nullptr;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  int taken = 0;
  bool ok = false;
  HeadPipe() {
    ok = cudaHostAlloc(reinterpret_cast<void**>(&slot), 2 * sizeof(KHead), cudaHostAllocDefault) == cudaSuccess &&
         cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming) == cudaSuccess;
  }
  // snapshot of the head after the work enqueued so far
  vd_status snapshot(const KWork& kw, cudaStream_t st) {
    const int k = taken & 1;
    VD_CUDA(cudaMemcpyAsync(slot + k, kw.ks, sizeof(KHead), cudaMemcpyDeviceToHost, st));
    VD_CUDA(cudaEventRecord(ev[k], st));
    ++taken;
    return VD_OK;
  }
  // wait for the latest snapshot (taken before the batch just enqueued) and copy it out
  vd_status latest(KHead* h) {
    const int k = (taken - 1) & 1;
    VD_CUDA(cudaEventSynchronize(ev[k]));
    *h = slot[k];
    return VD_OK;
  }
};

class HeadPipeLease {
 public:
  HeadPipeLease() {
    {
      std::lock_guard<std::mutex> lk(mu());
      if (!pool().empty()) {
        hp_ = pool().back();
        pool().pop_back();
      }
    }
    if (!hp_) hp_ = new HeadPipe();
    hp_->taken = 0;
  }
  ~HeadPipeLease() {
    // no snapshot copy may still be landing in the slots when the next solve takes them
    if (hp_->ok && hp_->taken > 0) {
      cudaEventSynchronize(hp_->ev[0]);
      if (hp_->taken > 1) cudaEventSynchronize(hp_->ev[1]);
    }
    std::lock_guard<std::mutex> lk(mu());
    pool().push_back(hp_);
  }
  HeadPipeLease(const HeadPipeLease&) = delete;
  HeadPipeLease& operator=(const HeadPipeLease&) = delete;
  // null when the pinned buffer or the events could not be created: poll synchronously
  HeadPipe* get() const { return hp_->ok ? hp_ : nullptr; }

 private:
  static std::mutex& mu() {
    static std::mutex m;
    return m;
  }
  static std::vector<HeadPipe*>& pool() {
    static std::vector<HeadPipe*> p;
    return p;
  }
  HeadPipe* hp_ = nullptr;
};

template <typename T>
vd_status krylov_solve(const SpecSystem& sys, const SolveOpts& o, const void* b, void* x, void* vecs,
                       const KWork& kw, double* host_hist, int host_hist_cap, SolveOut* out, cudaStream_t st) {
  const long long len = sys.len;
  const long long nc = sys.G->g.ncplx;
  const int h0 = sys.h0;
  const T* sym = (const T*)sys.sym;
  const int rb = red_blocks(len);
  const int eb = ew_blocks(len);
  const Ix ixr = mkix(len, h0, nc, rb, kRedThreads);
  const Ix ixe = mkix(len, h0, nc, eb, 256);
  RedArgs ra{kw.ks, kw.partials, kw.counter, kw.hist, o.tol};
  int* done = &kw.ks->done;
  int* cdone = &kw.ks->cycle_done;
  const int m = std::min(std::max(o.restart > 0 ? o.restart : 30, 1), kMaxRestart);
  const int check = std::max(1, o.check_every);

  // reset the scalar state
  KHead h0s;
  std::memset(&h0s, 0, sizeof(h0s));
  h0s.maxit = o.maxit;
  h0s.status = KS_RUNNING;
  h0s.hist_cap = host_hist_cap > 0 ? std::min(host_hist_cap, 1 << 20) : 0;
  h0s.m = m;
  h0s.guard = o.guard;
  VD_CUDA(cudaMemcpyAsync(kw.ks, &h0s, sizeof(KHead), cudaMemcpyHostToDevice, st));
  VD_CUDA(cudaMemsetAsync(kw.counter, 0, sizeof(unsigned), st));

  cpx<T>* X = (cpx<T>*)x;
  const cpx<T>* B = (const cpx<T>*)b;
  cpx<T>* vb = (cpx<T>*)vecs;
  KHead hd;

  if (o.solver == VD_SOLVER_CG) {
    cpx<T>* r = vb;
    cpx<T>* p = vb + len;
    cpx<T>* q = vb + 2 * len;
    if (o.x_zero) {
      VD_CUDA(cudaMemcpyAsync(r, B, sizeof(cpx<T>) * len, cudaMemcpyDeviceToDevice, st));
    } else {
      sys.apply(sys, X, q, false, nullptr, st);
      { ProfScope ps_(sizeof(T) == 4 ? PC_VEC32 : PC_VEC64, st, (double)3 * len * sizeof(cpx<T>), 0.0); k_sub<T><<<eb, 256, 0, st>>>(len, B, q, r, nullptr); }
    }
    { ProfScope ps_(sizeof(T) == 4 ? PC_VEC32 : PC_VEC64, st, (double)3 * len * sizeof(cpx<T>) + (double)nc * sizeof(T), 0.0); k_cg_init<T><<<rb, kRedThreads, 0, st>>>(ixr, B, r, p, sym, ra); }
    int it = 0;
    HeadPipeLease lease;
    HeadPipe* hp = lease.get();
    for (;;) {
      const long long mark = prof_mark();
      for (int c = 0; c < check && it < o.maxit; ++c, ++it) {
        sys.apply(sys, p, q, false, done, st);
        { ProfScope ps_(sizeof(T) == 4 ? PC_VEC32 : PC_VEC64, st, (double)2 * len * sizeof(cpx<T>), 0.0); k_dot<T, 1><<<rb, kRedThreads, 0, st>>>(ixr, p, q, EPI_CG_ALPHA, ra, done); }
        { ProfScope ps_(sizeof(T) == 4 ? PC_VEC32 : PC_VEC64, st, (double)6 * len * sizeof(cpx<T>) + (double)nc * sizeof(T), 0.0); k_cg_update<T><<<rb, kRedThreads, 0, st>>>(ixr, X, p, r, q, sym, ra); }
        { ProfScope ps_(sizeof(T) == 4 ? PC_VEC32 : PC_VEC64, st, (double)3 * len * sizeof(cpx<T>) + (double)nc * sizeof(T), 0.0); k_cg_p<T><<<eb, 256, 0, st>>>(ixe, p, r, sym, kw.ks); }
      }
      vd_status e = VD_OK;
      if (!hp) {
        e = read_head(kw, &hd, st);
        if (e != VD_OK) return e;
        if (hd.done || it >= o.maxit) break;
        continue;
      }
      if (hp->taken > 0) {
        e = hp->latest(&hd);   // the batch before the one just enqueued
        if (e != VD_OK) return e;
        if (hd.done) {
          prof_discard(mark, st);   // the batch just enqueued returns at once
          break;
        }
      }
      if (it >= o.maxit) break;
      e = hp->snapshot(kw, st);
      if (e != VD_OK) return e;
    }
  } else if (o.solver == VD_SOLVER_RMR) {
    cpx<T>* r = vb;
    cpx<T>* w = vb + len;
    if (o.x_zero) {
      VD_CUDA(cudaMemcpyAsync(r, B, sizeof(cpx<T>) * len, cudaMemcpyDeviceToDevice, st));
    } else {
      sys.apply(sys, X, w, false, nullptr, st);
      { ProfScope ps_(sizeof(T) == 4 ? PC_VEC32 : PC_VEC64, st, (double)3 * len * sizeof(cpx<T>), 0.0); k_sub<T><<<eb, 256, 0, st>>>(len, B, w, r, nullptr); }
    }
    { ProfScope ps_(sizeof(T) == 4 ? PC_VEC32 : PC_VEC64, st, (double)2 * len * sizeof(cpx<T>), 0.0); k_norms<T, 2><<<rb, kRedThreads, 0, st>>>(ixr, B, r, EPI_INIT_RMR, ra, nullptr); }
    int it = 0;
    HeadPipeLease lease;
    HeadPipe* hp = lease.get();
    for (;;) {
      const long long mark = prof_mark();
      for (int c = 0; c < check && it < o.maxit; ++c, ++it) {
        sys.apply(sys, r, w, true, done, st);
        { ProfScope ps_(sizeof(T) == 4 ? PC_VEC32 : PC_VEC64, st, (double)2 * len * sizeof(cpx<T>), 0.0); k_dot<T, 2><<<rb, kRedThreads, 0, st>>>(ixr, r, w, EPI_RMR_ALPHA, ra, done); }
        { ProfScope ps_(sizeof(T) == 4 ? PC_VEC32 : PC_VEC64, st, (double)5 * len * sizeof(cpx<T>) + (double)nc * sizeof(T), 0.0); k_rmr_update<T><<<rb, kRedThreads, 0, st>>>(ixr, X, r, w, sym, ra); }
      }
      vd_status e = VD_OK;
      if (!hp) {
        e = read_head(kw, &hd, st);
        if (e != VD_OK) return e;
        if (hd.done || it >= o.maxit) break;
        continue;
      }
      if (hp->taken > 0) {
        e = hp->latest(&hd);
        if (e != VD_OK) return e;
        if (hd.done) {
          prof_discard(mark, st);
          break;
        }
      }
      if (it >= o.maxit) break;
      e = hp->snapshot(kw, st);
      if (e != VD_OK) return e;
    }
  } else {
    cpx<T>* V = vb;
    cpx<T>* w = vb + (size_t)(m + 1) * len;
    { ProfScope ps_(sizeof(T) == 4 ? PC_VEC32 : PC_VEC64, st, (double)1 * len * sizeof(cpx<T>), 0.0); k_norms<T, 1><<<rb, kRedThreads, 0, st>>>(ixr, nullptr, B, EPI_BB, ra, nullptr); }
    for (int cycle = 0;; ++cycle) {
      // r = b - A x into V_0 (unnormalised), then V_0 /= beta
      if (cycle == 0 && o.x_zero) {
        VD_CUDA(cudaMemcpyAsync(V, B, sizeof(cpx<T>) * len, cudaMemcpyDeviceToDevice, st));
      } else {
        sys.apply(sys, X, w, false, done, st);
        { ProfScope ps_(sizeof(T) == 4 ? PC_VEC32 : PC_VEC64, st, (double)3 * len * sizeof(cpx<T>), 0.0); k_sub<T><<<eb, 256, 0, st>>>(len, B, w, V, done); }
      }
      { ProfScope ps_(sizeof(T) == 4 ? PC_VEC32 : PC_VEC64, st, (double)1 * len * sizeof(cpx<T>), 0.0); k_norms<T, 1><<<rb, kRedThreads, 0, st>>>(ixr, nullptr, V, EPI_GM_BETA, ra, done); }
      { ProfScope ps_(sizeof(T) == 4 ? PC_VEC32 : PC_VEC64, st, (double)2 * len * sizeof(cpx<T>), 0.0); k_gm_scale<T><<<eb, 256, 0, st>>>(ixe, V, V, kw.ks, 1); }
      for (int j = 0; j < m; ++j) {
        cpx<T>* Vj = V + (size_t)j * len;
        sys.apply(sys, Vj, w, true, cdone, st);
        for (int pass = 0; pass < 2; ++pass) {
          for (int off = 0; off <= j; off += 8) {
            const int nv = std::min(8, j + 1 - off);
            { ProfScope ps_(sizeof(T) == 4 ? PC_VEC32 : PC_VEC64, st, (double)(nv + 1) * len * sizeof(cpx<T>), 0.0); k_gm_mdot<T><<<rb, kRedThreads, 0, st>>>(ixr, w, V, off, nv, pass ? EPI_GM_H2 : EPI_GM_H1, j, ra); }
          }
          { ProfScope ps_(sizeof(T) == 4 ? PC_VEC32 : PC_VEC64, st, (double)(j + 3) * len * sizeof(cpx<T>), 0.0); k_gm_maxpy<T><<<rb, kRedThreads, 0, st>>>(ixr, w, V, j, pass, pass, ra); }
        }
        { ProfScope ps_(sizeof(T) == 4 ? PC_VEC32 : PC_VEC64, st, (double)2 * len * sizeof(cpx<T>), 0.0); k_gm_scale<T><<<eb, 256, 0, st>>>(ixe, V + (size_t)(j + 1) * len, w, kw.ks, 0); }
        if ((j + 1) % check == 0 || j + 1 == m) {
          vd_status e = read_head(kw, &hd, st);
          if (e != VD_OK) return e;
          if (hd.cycle_done || hd.done) break;
        }
      }
      { k_gm_solve<<<1, 1, 0, st>>>(kw.ks); count_launch(); }
      { ProfScope ps_(sizeof(T) == 4 ? PC_VEC32 : PC_VEC64, st, (double)(m + 2) * len * sizeof(cpx<T>) + (double)nc * sizeof(T), 0.0); k_gm_update<T><<<eb, 256, 0, st>>>(ixe, X, V, sym, kw.ks); }
      { k_gm_close<<<1, 1, 0, st>>>(kw.ks); count_launch(); }
      vd_status e = read_head(kw, &hd, st);
      if (e != VD_OK) return e;
      if (hd.done) break;
      if (hd.iters >= o.maxit) {
        // one more loop head forms the true residual and sets the final status
        sys.apply(sys, X, w, false, done, st);
        { ProfScope ps_(sizeof(T) == 4 ? PC_VEC32 : PC_VEC64, st, (double)3 * len * sizeof(cpx<T>), 0.0); k_sub<T><<<eb, 256, 0, st>>>(len, B, w, V, done); }
        { ProfScope ps_(sizeof(T) == 4 ? PC_VEC32 : PC_VEC64, st, (double)1 * len * sizeof(cpx<T>), 0.0); k_norms<T, 1><<<rb, kRedThreads, 0, st>>>(ixr, nullptr, V, EPI_GM_BETA, ra, done); }
        e = read_head(kw, &hd, st);
        if (e != VD_OK) return e;
        break;
      }
    }
  }
  VD_CUDA(cudaGetLastError());
  vd_status e = read_head(kw, &hd, st);
  if (e != VD_OK) return e;
  if (!hd.done) hd.status = VD_ERR_NOT_CONVERGED;
  out->iters = hd.iters;
  out->status = hd.status < 0 ? VD_ERR_NOT_CONVERGED : hd.status;
  out->relres = hd.relres;
  if (host_hist && h0s.hist_cap > 0) {
    const int nh = std::min(h0s.hist_cap, hd.iters + 1);
    VD_CUDA(cudaMemcpyAsync(host_hist, kw.hist, sizeof(double) * nh, cudaMemcpyDeviceToHost, st));
    VD_CUDA(cudaStreamSynchronize(st));
  }
  return VD_OK;
}

// ---------------------------------------------------------------------------------------
// graph form: the same kernels, with the iteration loop as a conditional WHILE node whose
// body ends in a kernel that sets the loop condition from the device `done` flag.  Nothing
// in it synchronises with the host, so it can be captured and replayed as a whole.
// ---------------------------------------------------------------------------------------

__global__ void k_ks_reset(KState* ks, int maxit, int m, cudaGraphConditionalHandle loop) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  // a loop nested in another conditional body keeps its last condition value: arm it here
  cudaGraphSetConditional(loop, 1u);
  KHead* h = reinterpret_cast<KHead*>(ks);
  unsigned* w = reinterpret_cast<unsigned*>(h);
  for (size_t i = 0; i < sizeof(KHead) / sizeof(unsigned); ++i) w[i] = 0u;
  h->maxit = maxit;
  h->status = KS_RUNNING;
  h->m = m;
}

// inner solve of a refinement sweep: budget and tolerance from the refinement state
__global__ void k_ks_reset_dev(KState* ks, const OState* o, int m, cudaGraphConditionalHandle loop) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  cudaGraphSetConditional(loop, 1u);
  KHead* h = reinterpret_cast<KHead*>(ks);
  unsigned* w = reinterpret_cast<unsigned*>(h);
  for (size_t i = 0; i < sizeof(KHead) / sizeof(unsigned); ++i) w[i] = 0u;
  h->maxit = o->maxit - o->total;
  h->status = KS_RUNNING;
  h->m = m;
  h->guard = kInnerGuard;
  ks->dtol = o->itol;
}

__global__ void k_graph_cond(cudaGraphConditionalHandle handle, const KState* ks) {
  if (threadIdx.x == 0 && blockIdx.x == 0) cudaGraphSetConditional(handle, ks->done ? 0u : 1u);
}

template <typename T>
vd_status krylov_enqueue_graph(const SpecSystem& sys, const SolveOpts& o, const void* b, void* x, void* vecs,
                               const KWork& kw, cudaStream_t st, cudaStream_t body_st) {
  const long long len = sys.len;
  const long long nc = sys.G->g.ncplx;
  const int h0 = sys.h0;
  const T* sym = (const T*)sys.sym;
  const int rb = red_blocks(len);
  const int eb = ew_blocks(len);
  const Ix ixr = mkix(len, h0, nc, rb, kRedThreads);
  const Ix ixe = mkix(len, h0, nc, eb, 256);
  RedArgs ra{kw.ks, kw.partials, kw.counter, kw.hist, o.dev_outer ? -1.0 : o.tol};
  int* done = &kw.ks->done;
  int* cdone = &kw.ks->cycle_done;
  const int m = std::min(std::max(o.restart > 0 ? o.restart : 30, 1), kMaxRestart);
  cpx<T>* X = (cpx<T>*)x;
  const cpx<T>* B = (const cpx<T>*)b;
  cpx<T>* vb = (cpx<T>*)vecs;

  // the loop's condition handle belongs to the graph being captured on st
  cudaGraphConditionalHandle hnd;
  {
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    VD_CUDA(cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, nullptr, nullptr, nullptr));
    if (cs != cudaStreamCaptureStatusActive) return fail(VD_ERR_INVALID_ARG, "graph solve needs a capturing stream");
    VD_CUDA(cudaGraphConditionalHandleCreate(&hnd, g, 1, cudaGraphCondAssignDefault));
  }
  if (o.dev_outer) k_ks_reset_dev<<<1, 1, 0, st>>>(kw.ks, o.dev_outer, m, hnd);
  else k_ks_reset<<<1, 1, 0, st>>>(kw.ks, o.maxit, m, hnd);
  count_launch();
  VD_CUDA(cudaMemsetAsync(kw.counter, 0, sizeof(unsigned), st));
  // the while node: splice it into the capture of st, then capture its body on body_st
  auto open_loop = [&](cudaGraphConditionalHandle* h) -> vd_status {
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    VD_CUDA(cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, &deps, nullptr, &nd));
    if (cs != cudaStreamCaptureStatusActive) return fail(VD_ERR_INVALID_ARG, "graph solve needs a capturing stream");
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = *h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    VD_CUDA(cudaGraphAddNode(&node, g, deps, nullptr, nd, &cp));
    VD_CUDA(cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    VD_CUDA(cudaStreamBeginCaptureToGraph(body_st, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                          cudaStreamCaptureModeRelaxed));
    return VD_OK;
  };
  auto close_loop = [&](cudaGraphConditionalHandle hnd) -> vd_status {
    k_graph_cond<<<1, 1, 0, body_st>>>(hnd, kw.ks);
    count_launch();
    cudaGraph_t body = nullptr;
    VD_CUDA(cudaStreamEndCapture(body_st, &body));
    return VD_OK;
  };
  vd_status e;
  if (o.solver == VD_SOLVER_CG) {
    cpx<T>* r = vb;
    cpx<T>* p = vb + len;
    cpx<T>* q = vb + 2 * len;
    if (o.x_zero) {
      VD_CUDA(cudaMemcpyAsync(r, B, sizeof(cpx<T>) * len, cudaMemcpyDeviceToDevice, st));
    } else {
      sys.apply(sys, X, q, false, nullptr, st);
      k_sub<T><<<eb, 256, 0, st>>>(len, B, q, r, nullptr);
      count_launch();
    }
    k_cg_init<T><<<rb, kRedThreads, 0, st>>>(ixr, B, r, p, sym, ra);
    count_launch();
    if ((e = open_loop(&hnd)) != VD_OK) return e;
    sys.apply(sys, p, q, false, done, body_st);
    k_dot<T, 1><<<rb, kRedThreads, 0, body_st>>>(ixr, p, q, EPI_CG_ALPHA, ra, done);
    k_cg_update<T><<<rb, kRedThreads, 0, body_st>>>(ixr, X, p, r, q, sym, ra);
    k_cg_p<T><<<eb, 256, 0, body_st>>>(ixe, p, r, sym, kw.ks);
    count_launch();
    count_launch();
    count_launch();
    if ((e = close_loop(hnd)) != VD_OK) return e;
  } else if (o.solver == VD_SOLVER_RMR) {
    cpx<T>* r = vb;
    cpx<T>* w = vb + len;
    if (o.x_zero) {
      VD_CUDA(cudaMemcpyAsync(r, B, sizeof(cpx<T>) * len, cudaMemcpyDeviceToDevice, st));
    } else {
      sys.apply(sys, X, w, false, nullptr, st);
      k_sub<T><<<eb, 256, 0, st>>>(len, B, w, r, nullptr);
      count_launch();
    }
    k_norms<T, 2><<<rb, kRedThreads, 0, st>>>(ixr, B, r, EPI_INIT_RMR, ra, nullptr);
    count_launch();
    if ((e = open_loop(&hnd)) != VD_OK) return e;
    sys.apply(sys, r, w, true, done, body_st);
    k_dot<T, 2><<<rb, kRedThreads, 0, body_st>>>(ixr, r, w, EPI_RMR_ALPHA, ra, done);
    k_rmr_update<T><<<rb, kRedThreads, 0, body_st>>>(ixr, X, r, w, sym, ra);
    count_launch();
    count_launch();
    if ((e = close_loop(hnd)) != VD_OK) return e;
  } else {
    cpx<T>* V = vb;
    cpx<T>* w = vb + (size_t)(m + 1) * len;
    k_norms<T, 1><<<rb, kRedThreads, 0, st>>>(ixr, nullptr, B, EPI_BB, ra, nullptr);
    count_launch();
    if ((e = open_loop(&hnd)) != VD_OK) return e;
    // one restart cycle: r = b - A x, V_0 = r / beta, m Arnoldi steps, update x
    sys.apply(sys, X, w, false, done, body_st);
    k_sub<T><<<eb, 256, 0, body_st>>>(len, B, w, V, done);
    k_norms<T, 1><<<rb, kRedThreads, 0, body_st>>>(ixr, nullptr, V, EPI_GM_BETA, ra, done);
    k_gm_scale<T><<<eb, 256, 0, body_st>>>(ixe, V, V, kw.ks, 1);
    count_launch();
    count_launch();
    count_launch();
    for (int j = 0; j < m; ++j) {
      cpx<T>* Vj = V + (size_t)j * len;
      sys.apply(sys, Vj, w, true, cdone, body_st);
      for (int pass = 0; pass < 2; ++pass) {
        for (int off = 0; off <= j; off += 8) {
          const int nv = std::min(8, j + 1 - off);
          k_gm_mdot<T><<<rb, kRedThreads, 0, body_st>>>(ixr, w, V, off, nv, pass ? EPI_GM_H2 : EPI_GM_H1, j, ra);
          count_launch();
        }
        k_gm_maxpy<T><<<rb, kRedThreads, 0, body_st>>>(ixr, w, V, j, pass, pass, ra);
        count_launch();
      }
      k_gm_scale<T><<<eb, 256, 0, body_st>>>(ixe, V + (size_t)(j + 1) * len, w, kw.ks, 0);
      count_launch();
    }
    k_gm_solve<<<1, 1, 0, body_st>>>(kw.ks);
    k_gm_update<T><<<eb, 256, 0, body_st>>>(ixe, X, V, sym, kw.ks);
    k_gm_close<<<1, 1, 0, body_st>>>(kw.ks);
    count_launch();
    count_launch();
    count_launch();
    if ((e = close_loop(hnd)) != VD_OK) return e;
  }
  VD_CUDA(cudaGetLastError());
  return VD_OK;
}

// result record of a graph solve: info[0] iterations, [1] status, [2] monitored relres,
// [3] |b|^2, [4] true relres
__global__ void k_graph_info(const KState* ks, double* info, int phase) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (phase == 0) {
    info[0] = (double)ks->iters;
    const int st = ks->done ? (ks->status < 0 ? VD_ERR_NOT_CONVERGED : ks->status) : VD_ERR_NOT_CONVERGED;
    info[1] = (double)st;
    info[2] = ks->relres;
  } else if (phase == 1) {
    info[3] = ks->rr;
  } else {
    info[4] = info[3] > 0.0 ? sqrt(ks->rr / info[3]) : 0.0;
  }
}

template <typename T>
vd_status krylov_graph_finish(const SpecSystem& sys, const void* b, const void* x, void* vecs, const KWork& kw,
                              double* info, cudaStream_t st) {
  const long long len = sys.len;
  const int rb = red_blocks(len);
  const int eb = ew_blocks(len);
  const Ix ixr = mkix(len, sys.h0, sys.G->g.ncplx, rb, kRedThreads);
  RedArgs ra{kw.ks, kw.partials, kw.counter, kw.hist, 0.0};
  const cpx<T>* B = (const cpx<T>*)b;
  cpx<T>* W = (cpx<T>*)vecs;
  k_graph_info<<<1, 1, 0, st>>>(kw.ks, info, 0);
  k_norms<T, 1><<<rb, kRedThreads, 0, st>>>(ixr, nullptr, B, EPI_NORM, ra, nullptr);
  k_graph_info<<<1, 1, 0, st>>>(kw.ks, info, 1);
  sys.apply(sys, x, W, false, nullptr, st);
  k_sub<T><<<eb, 256, 0, st>>>(len, B, W, W, nullptr);
  k_norms<T, 1><<<rb, kRedThreads, 0, st>>>(ixr, nullptr, W, EPI_NORM, ra, nullptr);
  k_graph_info<<<1, 1, 0, st>>>(kw.ks, info, 2);
  for (int i = 0; i < 6; ++i) count_launch();
  VD_CUDA(cudaGetLastError());
  return VD_OK;
}
template vd_status krylov_graph_finish<double>(const SpecSystem&, const void*, const void*, void*, const KWork&,
                                               double*, cudaStream_t);

// ---------------------------------------------------------------------------------------
// iterative refinement as a graph fragment
// ---------------------------------------------------------------------------------------

__global__ void k_out_init(OState* o, const KState* ks, double tol, double itol0, int maxit,
                           cudaGraphConditionalHandle loop) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  cudaGraphSetConditional(loop, 1u);
  o->bb = ks->rr;   // |b|^2, and the first residual is b
  o->rr = ks->rr;
  o->rnorm = o->rel = o->scale = 0.0;
  o->tol = tol;
  o->itol0 = itol0;
  o->itol = itol0;
  o->total = o->outer = 0;
  o->maxit = maxit;
  o->maxouter = 20;
  o->done = 0;
  o->status = VD_ERR_NOT_CONVERGED;
  o->force = 0;
}

// top of a refinement sweep: the same decisions as the host loop of vd_solve
__global__ void k_out_check(OState* o, cudaGraphConditionalHandle h_loop, cudaGraphConditionalHandle h_sweep) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double rnorm = sqrt(o->rr);
  const double bnorm = sqrt(o->bb);
  // a non-finite norm must not read as a zero right-hand side (NaN > 0 is false)
  const double rel = (!isfinite(bnorm) || !isfinite(rnorm)) ? (double)NAN : (bnorm > 0.0 ? rnorm / bnorm : 0.0);
  o->rnorm = rnorm;
  o->rel = rel;
  if (o->force) {
    o->done = 1;
    o->status = o->force;
  } else if (!isfinite(rel)) {
    o->done = 1;
    o->status = VD_ERR_NONFINITE;
  } else if (rel <= o->tol) {
    o->done = 1;
    o->status = VD_OK;
  } else if (o->total >= o->maxit || o->outer >= o->maxouter) {
    o->done = 1;
    o->status = VD_ERR_NOT_CONVERGED;
  } else {
    o->scale = 1.0 / rnorm;
    o->itol = fmax(o->itol0, 0.5 * o->tol / rel);
  }
  cudaGraphSetConditional(h_loop, o->done ? 0u : 1u);
  cudaGraphSetConditional(h_sweep, o->done ? 0u : 1u);
}

__global__ void k_out_after_inner(OState* o, const KState* ks) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  o->total += ks->iters;
  o->outer += 1;
  const int st = ks->done ? ks->status : VD_ERR_NOT_CONVERGED;
  if (st == VD_ERR_NONFINITE) o->force = VD_ERR_NONFINITE;
  else if (ks->iters == 0 && st != VD_OK) o->force = VD_ERR_NOT_CONVERGED;
}

__global__ void k_out_rr(OState* o, const KState* ks) {
  if (threadIdx.x == 0 && blockIdx.x == 0) o->rr = ks->rr;
}

__global__ void k_out_info(const OState* o, double* info) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  info[0] = (double)o->total;
  info[1] = (double)(o->done ? o->status : VD_ERR_NOT_CONVERGED);
  info[2] = o->rel;
  info[3] = o->bb;
  info[4] = o->rel;   // the refinement residual is the accurately computed true residual
  info[5] = (double)o->outer;
}

// v *= 1/|r| and x += |r| d with the scalars read from the refinement state

static vd_status open_cond(cudaStream_t st, cudaGraphConditionalNodeType type, cudaGraphConditionalHandle hnd,
                           cudaGraph_t* body) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  VD_CUDA(cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, &deps, nullptr, &nd));
  if (cs != cudaStreamCaptureStatusActive) return fail(VD_ERR_INVALID_ARG, "graph solve needs a capturing stream");
  cudaGraphNodeParams cp{};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = hnd;
  cp.conditional.type = type;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  VD_CUDA(cudaGraphAddNode(&node, g, deps, nullptr, nd, &cp));
  VD_CUDA(cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  *body = cp.conditional.phGraph_out[0];
  return VD_OK;
}

vd_status refine_enqueue_graph(const SpecSystem& sys64, const SpecSystem& sys32,
                               void (*resid)(const void* ctx, const void* x, void* y, cudaStream_t st),
                               const void* resid_ctx, const SolveOpts& inner, double tol, double itol0, int maxit,
                               void* bh, void* xh, void* rh, void* bh_f, void* xh_f, void* vecs, const KWork& kw,
                               OState* ost, double* info, cudaStream_t st, cudaStream_t s1, cudaStream_t s2,
                               cudaStream_t s3) {
  const long long len = sys64.len;
  const int rb = red_blocks(len);
  const int eb = ew_blocks(len);
  const Ix ixr = mkix(len, sys64.h0, sys64.G->g.ncplx, rb, kRedThreads);
  RedArgs ra{kw.ks, kw.partials, kw.counter, kw.hist, 0.0};
  cpx<double>* BH = (cpx<double>*)bh;
  cpx<double>* XH = (cpx<double>*)xh;
  cpx<double>* RH = (cpx<double>*)rh;
  // |b|^2, x = 0, r = b
  cudaGraphConditionalHandle h_loop, h_sweep;
  {
    cudaStreamCaptureStatus cs;
    cudaGraph_t g0 = nullptr;
    VD_CUDA(cudaStreamGetCaptureInfo(st, &cs, nullptr, &g0, nullptr, nullptr, nullptr));
    if (cs != cudaStreamCaptureStatusActive) return fail(VD_ERR_INVALID_ARG, "graph solve needs a capturing stream");
    VD_CUDA(cudaGraphConditionalHandleCreate(&h_loop, g0, 1, cudaGraphCondAssignDefault));
  }
  VD_CUDA(cudaMemsetAsync(kw.counter, 0, sizeof(unsigned), st));
  k_norms<double, 1><<<rb, kRedThreads, 0, st>>>(ixr, nullptr, BH, EPI_NORM, ra, nullptr);
  k_out_init<<<1, 1, 0, st>>>(ost, kw.ks, tol, itol0, maxit, h_loop);
  VD_CUDA(cudaMemsetAsync(XH, 0, sizeof(cpx<double>) * len, st));
  VD_CUDA(cudaMemcpyAsync(RH, BH, sizeof(cpx<double>) * len, cudaMemcpyDeviceToDevice, st));
  count_launch();
  count_launch();
  // while (not done) { check; if (sweep) { ... } }
  cudaGraph_t loop_body = nullptr, sweep_body = nullptr;
  vd_status e;
  if ((e = open_cond(st, cudaGraphCondTypeWhile, h_loop, &loop_body)) != VD_OK) return e;
  VD_CUDA(cudaStreamBeginCaptureToGraph(s1, loop_body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  {
    cudaStreamCaptureStatus cs;
    cudaGraph_t g1 = nullptr;
    VD_CUDA(cudaStreamGetCaptureInfo(s1, &cs, nullptr, &g1, nullptr, nullptr, nullptr));
    VD_CUDA(cudaGraphConditionalHandleCreate(&h_sweep, g1, 0, cudaGraphCondAssignDefault));
  }
  k_out_check<<<1, 1, 0, s1>>>(ost, h_loop, h_sweep);
  count_launch();
  {
    cudaStreamCaptureStatus cs;
    cudaGraph_t g1 = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    VD_CUDA(cudaStreamGetCaptureInfo(s1, &cs, nullptr, &g1, &deps, nullptr, &nd));
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h_sweep;
    cp.conditional.type = cudaGraphCondTypeIf;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    VD_CUDA(cudaGraphAddNode(&node, g1, deps, nullptr, nd, &cp));
    VD_CUDA(cudaStreamUpdateCaptureDependencies(s1, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    sweep_body = cp.conditional.phGraph_out[0];
  }
  VD_CUDA(cudaStreamBeginCaptureToGraph(s2, sweep_body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  // the sweep: d solves A32 d = r/|r| in float, x += |r| d, r = b - A x, |r|^2
  k_d2f_scaled<<<eb, 256, 0, s2>>>(len, RH, 0.0, ost, (cpx<float>*)bh_f);
  count_launch();
  VD_CUDA(cudaMemsetAsync(xh_f, 0, sizeof(cpx<float>) * len, s2));
  SolveOpts si = inner;
  si.x_zero = 1;
  si.dev_outer = ost;
  if ((e = krylov_enqueue_graph<float>(sys32, si, bh_f, xh_f, vecs, kw, s2, s3)) != VD_OK) return e;
  k_out_after_inner<<<1, 1, 0, s2>>>(ost, kw.ks);
  k_axpy_f2d<<<eb, 256, 0, s2>>>(len, 0.0, ost, (const cpx<float>*)xh_f, XH);
  resid(resid_ctx, XH, RH, s2);
  VD_CUDA(cudaMemsetAsync(kw.counter, 0, sizeof(unsigned), s2));
  k_sub_norm<double><<<rb, kRedThreads, 0, s2>>>(ixr, BH, RH, RH, ra);
  k_out_rr<<<1, 1, 0, s2>>>(ost, kw.ks);
  for (int i = 0; i < 4; ++i) count_launch();
  cudaGraph_t tmp = nullptr;
  VD_CUDA(cudaStreamEndCapture(s2, &tmp));
  VD_CUDA(cudaStreamEndCapture(s1, &tmp));
  k_out_info<<<1, 1, 0, st>>>(ost, info);
  count_launch();
  (void)sys64;
  VD_CUDA(cudaGetLastError());
  return VD_OK;
}

template vd_status krylov_enqueue_graph<double>(const SpecSystem&, const SolveOpts&, const void*, void*, void*,
                                                const KWork&, cudaStream_t, cudaStream_t);
template vd_status krylov_enqueue_graph<float>(const SpecSystem&, const SolveOpts&, const void*, void*, void*,
                                               const KWork&, cudaStream_t, cudaStream_t);

template vd_status krylov_solve<double>(const SpecSystem&, const SolveOpts&, const void*, void*, void*, const KWork&,
                                        double*, int, SolveOut*, cudaStream_t);
template vd_status krylov_solve<float>(const SpecSystem&, const SolveOpts&, const void*, void*, void*, const KWork&,
                                       double*, int, SolveOut*, cudaStream_t);
template size_t krylov_vec_bytes<double>(const SpecSystem&, int, int);
template size_t krylov_vec_bytes<float>(const SpecSystem&, int, int);
template void spec_copy_scale<double>(long long, const void*, double, void*, cudaStream_t);
template void spec_copy_scale<float>(long long, const void*, double, void*, cudaStream_t);
template void spec_axpy<double>(long long, double, const void*, void*, cudaStream_t);
template void spec_axpy<float>(long long, double, const void*, void*, cudaStream_t);
template void spec_sub<double>(long long, const void*, const void*, void*, cudaStream_t);
template void spec_sub<float>(long long, const void*, const void*, void*, cudaStream_t);
template void spec_project<double>(const vd_grid*, int, void*, cudaStream_t, double*);
template void spec_project<float>(const vd_grid*, int, void*, cudaStream_t, double*);
template double spec_dot_host<double>(const SpecSystem&, const void*, const void*, const KWork&, cudaStream_t);
template double spec_norm2_host<double>(const SpecSystem&, const void*, const KWork&, cudaStream_t);
template double spec_norm2_host<float>(const SpecSystem&, const void*, const KWork&, cudaStream_t);

}  // namespace vd
