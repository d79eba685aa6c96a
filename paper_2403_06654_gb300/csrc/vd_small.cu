// Whole preconditioned solves of 1D pressure problems in a single kernel launch.
//
// The 1D top-hat study of Sec. 3.2 (N = 256, density ratio 3, CG / GMRES / RMR to 1e-12) is a
// few tens of iterations on a half spectrum of n0/2 + 1 coefficients.  Launched pass by pass,
// an iteration is ~10 kernels and a host poll: latency, not arithmetic or memory, sets its
// time.  Here one thread block keeps the right-hand side, the Krylov vectors, 1/(N rho), the
// symbol of the preconditioner and the twiddle tables in shared memory and runs the whole
// solve: forward transform of b (and of x0), range projection, the Krylov loop with its
// operator applies, convergence tests and history, the inverse transform of x and the true
// residual.  Reductions are block-level with a fixed order (deterministic).
//
// The arithmetic is the library's own: the real-transform packing and the Stockham engine of
// the x pass, the same recurrences (PCG, right-preconditioned RMR, right-preconditioned
// GMRES(m) with classical Gram-Schmidt applied twice and Givens rotations), the same tests
// and statuses as the pass-by-pass solve (vd_krylov.cu).  Eligible: the pressure operator in
// FP64 on a 1D grid whose vectors fit in shared memory (GMRES: (m + 7) half spectra).
#include "vd_internal.h"
#include "vd_fft.cuh"
#include "vd_krylov.cuh"
#include "vd_prof.h"

#include <algorithm>
#include <cmath>
#include <cstdio>

namespace vd {

namespace {

struct SmallOut {   // result record (device, caller workspace)
  int iters, status, hist_len, pad;
  double relres, relres_true, removed2, bb;
};

struct SmallArgs {
  GridDesc g;
  const cpx<double>* tw;    // twiddle tables of the grid (x plan and packing)
  const double* rinv;       // 1/(N rho), n0 values
  const double* b;          // physical right-hand side
  double* x;                // physical solution (initial guess when use_x0)
  double* hist;             // monitored relres per iteration (device), hist_cap entries
  SmallOut* out;
  double tol;
  int solver, maxit, restart, use_x0, hist_cap;
};

// shared-memory carving (all cpx<double> arrays 16-byte aligned)
struct SmallSmem {
  cpx<double>*twm, *pk, *A, *B;
  double *rinv, *sym;
  cpx<double>*bh, *xh, *r, *p, *q, *V;
  double* H;      // (m+1) x m column-major, then cs, sn, g, y, h1, h2
  double* red;    // reduction scratch: 8 values x warps
};

__host__ __device__ inline size_t small_smem_bytes(int n0, int solver, int restart, int nthreads) {
  const size_t m = (size_t)n0 / 2, h0 = m + 1;
  size_t c = m + (m + 1) + 2 * (m + 1);   // twiddles, packing, FFT ping-pong
  c += 5 * h0;                            // b, x, r, p, q
  if (solver == VD_SOLVER_GMRES) c += (size_t)(restart + 2) * h0;   // basis + w
  size_t d = (size_t)n0 + h0;             // 1/(N rho), symbol
  if (solver == VD_SOLVER_GMRES) d += (size_t)(restart + 1) * restart + 6 * (restart + 1);
  d += 8 * (size_t)(nthreads / 32) + 8;
  return c * sizeof(cpx<double>) + d * sizeof(double);
}

template <int NT>
__device__ __forceinline__ double kt(const GridDesc& g, int k) {
  return g.kfac[0] * (double)freq_tilde(k, g.n0);
}

// sum over the block of NV values per thread, fixed order; every thread gets the totals
template <int NT, int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* red) {
  constexpr int NW = NT / 32;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_down_sync(0xffffffffu, v[i], o);
  __syncthreads();   // red may still be read by the previous reduction
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < NV; ++i) red[i * NW + wid] = v[i];
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < NW; ++w) s += red[i * NW + w];
    v[i] = s;
  }
}

__device__ __forceinline__ double pw(int k, int h0) { return (k == 0 || k == h0 - 1) ? 1.0 : 2.0; }


// o = A (S v) with S the symbol (with_sym) or 1: i k~ F[ (1/(N rho)) F^-1( i k~ S v ) ] through the
// x-pass arithmetic (pack, inverse complex FFT of length m, weight, forward FFT, unpack, 1/2)
template <int NT>
__device__ void apply1d(const SmallSmem& s, const GridDesc& g, const cpx<double>* v, cpx<double>* o, bool with_sym) {
  const int m = g.n0 / 2, tid = threadIdx.x;
  __syncthreads();   // v complete, A and B free
  for (int k = tid; k <= m; k += NT) {
    double cc = kt<NT>(g, k);
    if (with_sym) cc *= s.sym[k];
    s.B[k] = mul_i(scal(v[k], cc));
  }
  __syncthreads();
  for (int k = tid; k < m; k += NT) {
    const cpx<double> X = s.B[k];
    const cpx<double> Xc = conjg(s.B[m - k]);
    s.A[k] = (X + Xc) + mul_i(cmulc(X - Xc, s.pk[k]));
  }
  cpx<double>* res = fft_lines<double, +1>(s.A, s.B, 1, 0, tid, NT, g.px, s.twm);
  for (int j = tid; j < m; j += NT) {
    const cpx<double> z = res[j];
    res[j] = mk<double>(z.x * s.rinv[2 * j], z.y * s.rinv[2 * j + 1]);
  }
  cpx<double>* other = (res == s.A) ? s.B : s.A;
  res = fft_lines<double, -1>(res, other, 1, 0, tid, NT, g.px, s.twm);
  for (int k = tid; k <= m; k += NT) {
    const cpx<double> Z = res[k == m ? 0 : k];
    const cpx<double> Zc = conjg(res[k == 0 ? 0 : m - k]);
    const cpx<double> X = (Z + Zc) - mul_i(cmul(Z - Zc, s.pk[k]));
    o[k] = mul_i(scal(X, 0.5 * kt<NT>(g, k)));
  }
  __syncthreads();
}

// half spectrum of the physical field f (unnormalised DFT)
template <int NT>
__device__ void forward1d(const SmallSmem& s, const GridDesc& g, const double* f, cpx<double>* o) {
  const int m = g.n0 / 2, tid = threadIdx.x;
  __syncthreads();
  for (int j = tid; j < m; j += NT) s.A[j] = mk<double>(f[2 * j], f[2 * j + 1]);
  cpx<double>* res = fft_lines<double, -1>(s.A, s.B, 1, 0, tid, NT, g.px, s.twm);
  for (int k = tid; k <= m; k += NT) {
    const cpx<double> Z = res[k == m ? 0 : k];
    const cpx<double> Zc = conjg(res[k == 0 ? 0 : m - k]);
    o[k] = scal((Z + Zc) - mul_i(cmul(Z - Zc, s.pk[k])), 0.5);
  }
  __syncthreads();
}

// physical field of the half spectrum v (inverse DFT / N)
template <int NT>
__device__ void inverse1d(const SmallSmem& s, const GridDesc& g, const cpx<double>* v, double* f) {
  const int m = g.n0 / 2, tid = threadIdx.x;
  __syncthreads();
  for (int k = tid; k < m; k += NT) {
    const cpx<double> X = v[k];
    const cpx<double> Xc = conjg(v[m - k]);
    s.A[k] = (X + Xc) + mul_i(cmulc(X - Xc, s.pk[k]));
  }
  cpx<double>* res = fft_lines<double, +1>(s.A, s.B, 1, 0, tid, NT, g.px, s.twm);
  const double sc = 1.0 / (double)g.nreal;
  for (int j = tid; j < m; j += NT) {
    const cpx<double> z = scal(res[j], sc);
    f[2 * j] = z.x;
    f[2 * j + 1] = z.y;
  }
  __syncthreads();
}

template <int NT>
__global__ void __launch_bounds__(NT) k_small_solve_1d(const SmallArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const GridDesc& g = a.g;
  const int tid = threadIdx.x;
  const int m = g.n0 / 2, h0 = m + 1, n0 = g.n0;
  const int R = (a.solver == VD_SOLVER_GMRES) ? a.restart : 0;
  SmallSmem s;
  {
    cpx<double>* c = reinterpret_cast<cpx<double>*>(smem_raw);
    s.twm = c;
    s.pk = s.twm + m;
    s.A = s.pk + (m + 1);
    s.B = s.A + (m + 1);
    s.bh = s.B + (m + 1);
    s.xh = s.bh + h0;
    s.r = s.xh + h0;
    s.p = s.r + h0;
    s.q = s.p + h0;
    s.V = s.q + h0;                                   // GMRES: (R + 1) basis vectors, then w
    double* d = reinterpret_cast<double*>(s.V + (a.solver == VD_SOLVER_GMRES ? (size_t)(R + 2) * h0 : 0));
    s.rinv = d;
    s.sym = s.rinv + n0;
    s.H = s.sym + h0;
    s.red = s.H + (a.solver == VD_SOLVER_GMRES ? (size_t)(R + 1) * R + 6 * (R + 1) : 0);
  }
  for (int j = tid; j < m; j += NT) s.twm[j] = a.tw[g.px.tw_off + j];
  for (int j = tid; j <= m; j += NT) s.pk[j] = a.tw[g.pk_off + j];
  for (int j = tid; j < n0; j += NT) s.rinv[j] = a.rinv[j];
  for (int k = tid; k < h0; k += NT) {
    const double kk = kt<NT>(g, k);
    const double k2 = kk * kk;
    s.sym[k] = (k2 == 0.0) ? 0.0 : -recip(k2);   // pseudo-inverse of the Laplacian
  }
  // spectral right-hand side, projected onto the range (k = 0 and the Nyquist mode removed)
  forward1d<NT>(s, g, a.b, s.bh);
  double removed2 = 0.0;
  if (tid == 0) {
    removed2 = s.bh[0].x * s.bh[0].x + s.bh[0].y * s.bh[0].y + s.bh[m].x * s.bh[m].x + s.bh[m].y * s.bh[m].y;
    s.bh[0] = mk<double>(0.0, 0.0);
    s.bh[m] = mk<double>(0.0, 0.0);
  }
  // initial iterate
  if (a.use_x0) {
    forward1d<NT>(s, g, a.x, s.xh);
    if (tid == 0) {
      s.xh[0] = mk<double>(0.0, 0.0);
      s.xh[m] = mk<double>(0.0, 0.0);
    }
  } else {
    for (int k = tid; k < h0; k += NT) s.xh[k] = mk<double>(0.0, 0.0);
  }
  __syncthreads();
  // r = b - A x
  if (a.use_x0) {
    apply1d<NT>(s, g, s.xh, s.q, false);
    for (int k = tid; k < h0; k += NT) s.r[k] = s.bh[k] - s.q[k];
  } else {
    for (int k = tid; k < h0; k += NT) s.r[k] = s.bh[k];
  }
  __syncthreads();

  int iters = 0, status = -1;
  double rel = 0.0, bb = 0.0;
  auto record = [&](double v) {
    if (tid == 0 && iters < a.hist_cap) a.hist[iters] = v;
  };

  if (a.solver == VD_SOLVER_CG) {
    // p = S r; [bb, rr, rz]
    double v[3] = {0.0, 0.0, 0.0};
    for (int k = tid; k < h0; k += NT) {
      const double w = pw(k, h0), sv = s.sym[k];
      const cpx<double> bv = s.bh[k], rv = s.r[k];
      s.p[k] = scal(rv, sv);
      const double r2 = rv.x * rv.x + rv.y * rv.y;
      v[0] += w * (bv.x * bv.x + bv.y * bv.y);
      v[1] += w * r2;
      v[2] += w * sv * r2;
    }
    block_sum<NT, 3>(v, s.red);
    bb = v[0];
    double rz = v[2];
    rel = (bb == 0.0) ? 0.0 : sqrt(v[1] / bb);
    record(rel);
    if (bb == 0.0 || rel <= a.tol) status = 0;
    else if (!isfinite(rel)) status = VD_ERR_NONFINITE;
    else if (a.maxit <= 0) status = VD_ERR_NOT_CONVERGED;
    const double tol2bb = a.tol * a.tol * bb;
    while (status < 0) {
      apply1d<NT>(s, g, s.p, s.q, false);
      double d[1] = {0.0};
      for (int k = tid; k < h0; k += NT) {
        const cpx<double> pv = s.p[k], qv = s.q[k];
        d[0] += pw(k, h0) * (pv.x * qv.x + pv.y * qv.y);
      }
      block_sum<NT, 1>(d, s.red);
      const double pq = d[0];
      if (pq == 0.0 || rz == 0.0) {
        ++iters;
        status = VD_ERR_BREAKDOWN;
        break;
      }
      const double al = rz / pq;
      if (!isfinite(al)) {
        ++iters;
        status = VD_ERR_NONFINITE;
        break;
      }
      double u[2] = {0.0, 0.0};
      for (int k = tid; k < h0; k += NT) {
        const cpx<double> pv = s.p[k], qv = s.q[k];
        cpx<double> xv = s.xh[k], rv = s.r[k];
        xv = mk<double>(fma(al, pv.x, xv.x), fma(al, pv.y, xv.y));
        rv = mk<double>(fma(-al, qv.x, rv.x), fma(-al, qv.y, rv.y));
        s.xh[k] = xv;
        s.r[k] = rv;
        const double w = pw(k, h0), r2 = rv.x * rv.x + rv.y * rv.y;
        u[0] += w * r2;
        u[1] += w * s.sym[k] * r2;
      }
      block_sum<NT, 2>(u, s.red);
      ++iters;
      rel = sqrt(u[0] / bb);
      record(rel);
      if (!isfinite(rel)) {
        status = VD_ERR_NONFINITE;
        break;
      }
      if (u[0] <= tol2bb) {
        status = 0;
        break;
      }
      const double be = u[1] / rz;
      rz = u[1];
      if (iters >= a.maxit) {
        status = VD_ERR_NOT_CONVERGED;
        break;
      }
      for (int k = tid; k < h0; k += NT) {
        const double sv = s.sym[k];
        const cpx<double> rv = s.r[k], pv = s.p[k];
        s.p[k] = mk<double>(fma(be, pv.x, sv * rv.x), fma(be, pv.y, sv * rv.y));
      }
    }
  } else if (a.solver == VD_SOLVER_RMR) {
    double v[2] = {0.0, 0.0};
    for (int k = tid; k < h0; k += NT) {
      const double w = pw(k, h0);
      const cpx<double> bv = s.bh[k], rv = s.r[k];
      v[0] += w * (bv.x * bv.x + bv.y * bv.y);
      v[1] += w * (rv.x * rv.x + rv.y * rv.y);
    }
    block_sum<NT, 2>(v, s.red);
    bb = v[0];
    rel = (bb == 0.0) ? 0.0 : sqrt(v[1] / bb);
    double best = rel;
    record(rel);
    if (bb == 0.0 || rel <= a.tol) status = 0;
    else if (!isfinite(rel)) status = VD_ERR_NONFINITE;
    else if (a.maxit <= 0) status = VD_ERR_NOT_CONVERGED;
    const double tol2bb = a.tol * a.tol * bb;
    while (status < 0) {
      apply1d<NT>(s, g, s.r, s.q, true);   // w = A S r
      double d[2] = {0.0, 0.0};
      for (int k = tid; k < h0; k += NT) {
        const double w = pw(k, h0);
        const cpx<double> rv = s.r[k], wv = s.q[k];
        d[0] += w * (rv.x * wv.x + rv.y * wv.y);
        d[1] += w * (wv.x * wv.x + wv.y * wv.y);
      }
      block_sum<NT, 2>(d, s.red);
      if (d[1] == 0.0) {
        ++iters;
        status = VD_ERR_BREAKDOWN;
        break;
      }
      const double al = d[0] / d[1];
      double u[1] = {0.0};
      for (int k = tid; k < h0; k += NT) {
        const double as = al * s.sym[k];
        const cpx<double> wq = s.q[k];
        cpx<double> xv = s.xh[k], rv = s.r[k];
        xv = mk<double>(fma(as, rv.x, xv.x), fma(as, rv.y, xv.y));
        rv = mk<double>(fma(-al, wq.x, rv.x), fma(-al, wq.y, rv.y));
        s.xh[k] = xv;
        s.r[k] = rv;
        u[0] += pw(k, h0) * (rv.x * rv.x + rv.y * rv.y);
      }
      block_sum<NT, 1>(u, s.red);
      ++iters;
      rel = sqrt(u[0] / bb);
      record(rel);
      if (!isfinite(rel)) {
        status = VD_ERR_NONFINITE;
        break;
      }
      if (u[0] <= tol2bb) {
        status = 0;
        break;
      }
      if (rel > 1e3 * best) {
        status = VD_ERR_DIVERGED;
        break;
      }
      best = fmin(best, rel);
      if (iters >= a.maxit) {
        status = VD_ERR_NOT_CONVERGED;
        break;
      }
    }
  } else {
    // GMRES(R), right-preconditioned, x += S V y at the end of every cycle
    double* Hm = s.H;                              // (R+1) x R, column-major
    double* cs = Hm + (size_t)(R + 1) * R;
    double* sn = cs + (R + 1);
    double* gv = sn + (R + 1);
    double* yv = gv + (R + 1);
    double* h1 = yv + (R + 1);
    double* h2 = h1 + (R + 1);
    cpx<double>* w = s.V + (size_t)(R + 1) * h0;
    {
      double v[1] = {0.0};
      for (int k = tid; k < h0; k += NT) {
        const cpx<double> bv = s.bh[k];
        v[0] += pw(k, h0) * (bv.x * bv.x + bv.y * bv.y);
      }
      block_sum<NT, 1>(v, s.red);
      bb = v[0];
    }
    for (int cycle = 0; status < 0; ++cycle) {
      // V_0 = r = b - A x
      if (cycle > 0 || a.use_x0) {
        apply1d<NT>(s, g, s.xh, w, false);
        for (int k = tid; k < h0; k += NT) s.V[k] = s.bh[k] - w[k];
      } else {
        for (int k = tid; k < h0; k += NT) s.V[k] = s.r[k];
      }
      double v[1] = {0.0};
      for (int k = tid; k < h0; k += NT) {
        const cpx<double> rv = s.V[k];
        v[0] += pw(k, h0) * (rv.x * rv.x + rv.y * rv.y);
      }
      block_sum<NT, 1>(v, s.red);
      const double beta = sqrt(v[0]);
      if (bb == 0.0) {
        rel = 0.0;
        if (iters == 0) record(0.0);
        status = 0;
        break;
      }
      rel = beta / sqrt(bb);
      if (iters == 0) record(rel);
      if (!isfinite(rel)) {
        status = VD_ERR_NONFINITE;
        break;
      }
      if (rel <= a.tol) {
        status = 0;
        break;
      }
      if (iters >= a.maxit) {
        status = VD_ERR_NOT_CONVERGED;
        break;
      }
      const double ib = 1.0 / beta;
      for (int k = tid; k < h0; k += NT) s.V[k] = scal(s.V[k], ib);
      if (tid == 0) gv[0] = beta;
      int kdone = 0;
      bool cycle_done = false;
      for (int j = 0; j < R && !cycle_done; ++j) {
        cpx<double>* Vj = s.V + (size_t)j * h0;
        apply1d<NT>(s, g, Vj, w, true);   // w = A S V_j
        // classical Gram-Schmidt, twice
        for (int pass = 0; pass < 2; ++pass) {
          double* hh = pass ? h2 : h1;
          // the j + 1 dot products (w, V_i) in reductions of 8 at a time
          for (int i0 = 0; i0 <= j; i0 += 8) {
            double d[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
            for (int k = tid; k < h0; k += NT) {
              const cpx<double> wv = w[k];
              const double wk = pw(k, h0);
#pragma unroll
              for (int ii = 0; ii < 8; ++ii) {
                if (i0 + ii <= j) {
                  const cpx<double> vv = s.V[(size_t)(i0 + ii) * h0 + k];
                  d[ii] += wk * (wv.x * vv.x + wv.y * vv.y);
                }
              }
            }
            block_sum<NT, 8>(d, s.red);
            if (tid == 0)
              for (int ii = 0; ii < 8 && i0 + ii <= j; ++ii) hh[i0 + ii] = d[ii];
          }
          __syncthreads();
          for (int k = tid; k < h0; k += NT) {
            cpx<double> wv = w[k];
            for (int i = 0; i <= j; ++i) {
              const cpx<double> vv = s.V[(size_t)i * h0 + k];
              wv = mk<double>(fma(-hh[i], vv.x, wv.x), fma(-hh[i], vv.y, wv.y));
            }
            w[k] = wv;
          }
          __syncthreads();
        }
        double d[1] = {0.0};
        for (int k = tid; k < h0; k += NT) {
          const cpx<double> wv = w[k];
          d[0] += pw(k, h0) * (wv.x * wv.x + wv.y * wv.y);
        }
        block_sum<NT, 1>(d, s.red);
        const double hn = sqrt(d[0]);
        if (tid == 0) {
          double* col = Hm + (size_t)j * (R + 1);
          for (int i = 0; i <= j; ++i) col[i] = h1[i] + h2[i];
          col[j + 1] = hn;
          for (int i = 0; i < j; ++i) {
            const double t0 = cs[i] * col[i] + sn[i] * col[i + 1];
            col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
            col[i] = t0;
          }
          double c = 1.0, sgn = 0.0;
          if (col[j + 1] != 0.0) {
            const double h = hypot(col[j], col[j + 1]);
            c = col[j] / h;
            sgn = col[j + 1] / h;
          }
          cs[j] = c;
          sn[j] = sgn;
          col[j] = c * col[j] + sgn * col[j + 1];
          col[j + 1] = 0.0;
          gv[j + 1] = -sgn * gv[j];
          gv[j] = c * gv[j];
        }
        __syncthreads();
        ++iters;
        kdone = j + 1;
        const double est = fabs(gv[j + 1]) / sqrt(bb);
        rel = est;
        record(est);
        if (!isfinite(est)) {
          status = VD_ERR_NONFINITE;
          cycle_done = true;
        } else if (est <= a.tol || hn == 0.0) {
          status = 0;
          cycle_done = true;
        } else if (j + 1 >= R || iters >= a.maxit) {
          cycle_done = true;
        } else {
          const double ihn = 1.0 / hn;
          cpx<double>* Vn = s.V + (size_t)(j + 1) * h0;
          for (int k = tid; k < h0; k += NT) Vn[k] = scal(w[k], ihn);
        }
      }
      // y = H^-1 g (back substitution), x += S V y
      if (tid == 0) {
        for (int i = kdone - 1; i >= 0; --i) {
          double t0 = gv[i];
          for (int l = i + 1; l < kdone; ++l) t0 -= Hm[i + (size_t)l * (R + 1)] * yv[l];
          yv[i] = t0 / Hm[i + (size_t)i * (R + 1)];
        }
      }
      __syncthreads();
      if (status != VD_ERR_NONFINITE) {
        for (int k = tid; k < h0; k += NT) {
          double ax = 0.0, ay = 0.0;
          for (int i = 0; i < kdone; ++i) {
            const cpx<double> vv = s.V[(size_t)i * h0 + k];
            ax = fma(yv[i], vv.x, ax);
            ay = fma(yv[i], vv.y, ay);
          }
          const double sv = s.sym[k];
          const cpx<double> xv = s.xh[k];
          s.xh[k] = mk<double>(fma(sv, ax, xv.x), fma(sv, ay, xv.y));
        }
      }
      __syncthreads();
      // the loop head of the next cycle forms the true residual (and the final status when
      // the budget is spent)
    }
  }
  __syncthreads();
  // back to physical space, and the true residual of the returned iterate
  inverse1d<NT>(s, g, s.xh, a.x);
  apply1d<NT>(s, g, s.xh, s.q, false);
  double t[1] = {0.0};
  for (int k = tid; k < h0; k += NT) {
    const cpx<double> rv = s.bh[k] - s.q[k];
    t[0] += pw(k, h0) * (rv.x * rv.x + rv.y * rv.y);
  }
  block_sum<NT, 1>(t, s.red);
  if (tid == 0) {
    a.out->iters = iters;
    a.out->status = status < 0 ? VD_ERR_NOT_CONVERGED : status;
    a.out->hist_len = min(a.hist_cap, iters + 1);
    a.out->relres = rel;
    a.out->relres_true = (bb > 0.0) ? sqrt(t[0] / bb) : 0.0;
    a.out->removed2 = removed2;
    a.out->bb = bb;
  }
}

}  // namespace

bool small_solve_eligible(const vd_grid* G, vd_op op, int solver, int precision, int restart) {
  if (op != VD_OP_PRESSURE || precision != VD_PREC_FP64 || G->g.ndim != 1) return false;
  const int nt = 128;   // four warps: every SM partition issues FP64 work
  return small_smem_bytes(G->g.n0, solver, restart, nt) <= 200 * 1024;
}

// the whole solve in one launch; results into info (and hist) after a stream synchronisation
vd_status small_solve_1d(const vd_grid* G, int solver, const vd_solve_params* prm, int restart, const double* b,
                         double* x, vd_solve_info* info, void* out_dev, double* hist_dev, int hist_cap,
                         cudaStream_t st) {
  SmallArgs a;
  a.g = G->g;
  a.tw = reinterpret_cast<const cpx<double>*>(G->tw_d);
  a.rinv = G->rinv_s;
  a.b = b;
  a.x = x;
  a.hist = hist_dev;
  a.hist_cap = hist_cap;
  a.out = reinterpret_cast<SmallOut*>(out_dev);
  a.tol = prm->tol;
  a.solver = solver;
  a.maxit = prm->max_it;
  a.restart = restart;
  a.use_x0 = prm->use_x0 ? 1 : 0;
  const int nt = 128;   // four warps: every SM partition issues FP64 work
  const size_t smem = small_smem_bytes(G->g.n0, solver, restart, nt);
  VD_CUDA(cudaFuncSetAttribute(k_small_solve_1d<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_small_solve_1d<128><<<1, 128, smem, st>>>(a);
  count_launch();
  VD_CUDA(cudaGetLastError());
  SmallOut o;
  VD_CUDA(cudaMemcpyAsync(&o, out_dev, sizeof o, cudaMemcpyDeviceToHost, st));
  if (info && info->hist && info->hist_cap > 0) {
    const int n = std::min(info->hist_cap, hist_cap);
    if (n > 0) VD_CUDA(cudaMemcpyAsync(info->hist, hist_dev, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
  }
  VD_CUDA(cudaStreamSynchronize(st));
  if (info) {
    info->iters = o.iters;
    info->outer_iters = 0;
    info->status = o.status;
    info->relres = o.relres;
    info->relres_true = o.relres_true;
    info->hist_len = (info->hist && info->hist_cap > 0) ? std::min(info->hist_cap, o.hist_len) : 0;
    info->rhs_removed = (o.removed2 > 0.0) ? std::sqrt(o.removed2 / (o.bb + o.removed2)) : 0.0;
    info->coef_pair = 0;
  }
  if (o.status != VD_OK) {
    char buf[160];
    std::snprintf(buf, sizeof buf, "solve ended with status %d after %d iterations (relres %.3e)", o.status, o.iters,
                  o.relres);
    fail((vd_status)o.status, buf);
  }
  return (vd_status)o.status;
}

}  // namespace vd
