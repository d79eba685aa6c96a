// Operator pipelines built from the transform passes.
//
// Pressure operator (Eq. VDINSE.Lrho.num), spectral in -> spectral out:
//   L~ psi = sum_j i k~_j F[ rho^-1 F^-1( i k~_j psi ) ]
// Velocity operator (Eq. VDINSE.zeta with the Crank--Nicolson factor a = dt/(2 Re)):
//   V~ u = u - a F[ rho^-1 ( Lap u + Sc^-1 ( (u.grad) grad rho + (grad rho.grad) u ) ) ]
#include "vd_internal.h"
#include "vd_prof.h"
#include "vd_fft.cuh"
#include "vd_dd.cuh"

#include <algorithm>
#include <type_traits>

namespace vd {

static inline Xf mkxf(int src, int dst, int pre, int post, bool first, bool last, double scale = 1.0,
                      bool nofft = false) {
  Xf x;
  x.src = (int8_t)src;
  x.dst = (int8_t)dst;
  x.pre = (int8_t)pre;
  x.post = (int8_t)post;
  x.first = first ? 1 : 0;
  x.last = last ? 1 : 0;
  x.nofft = nofft ? 1 : 0;
  x.pad = 0;
  x.scale = scale;
  return x;
}

template <typename T>
static const void* twtab(const vd_grid* G) {
  if (std::is_same<T, dd>::value) return G->tw_dd;
  return (sizeof(T) == 8) ? G->tw_d : G->tw_f;
}

int pressure_tmp_fields(int ndim) { return ndim == 3 ? 3 : (ndim == 2 ? 2 : 0); }
// spectral temporaries of the velocity apply: the shared inverse passes of a component (3D:
// four fields, 2D: three) and the forward transforms of the d brackets
int velocity_spec_tmps(int ndim) { return ndim == 3 ? 4 : (ndim == 2 ? 3 : 1); }
int velocity_tmp_fields(int ndim) { return velocity_spec_tmps(ndim) + ndim * ndim + 2 * ndim; }

// ---------------------------------------------------------------------------------------
// plain transforms
// ---------------------------------------------------------------------------------------

template <typename T>
void fwd_transform(const vd_grid* G, const T* in, cpx<T>* out, cudaStream_t st) {
  const GridDesc& g = G->g;
  XProg X{};
  X.ncomp = 1;
  X.mode = 1;
  X.in[0] = in;
  X.out[0] = out;
  X.scale = 0.5;
  launch_xpass<T>(X, g, twtab<T>(G), st);
  if (g.ndim >= 2) {
    AxisProg P{};
    P.nxf = 1;
    P.xf[0] = mkxf(0, 0, 0, 0, true, true);
    P.in[0] = out;
    P.out[0] = out;
    P.axis = 1;
    launch_axis<T>(P, -1, g, twtab<T>(G), st);
    if (g.ndim == 3) {
      P.axis = 2;
      launch_axis<T>(P, -1, g, twtab<T>(G), st);
    }
  }
}

template <typename T>
void inv_transform(const vd_grid* G, const cpx<T>* in, const Mult& mu, T* out, cpx<T>* tmp, cudaStream_t st) {
  const GridDesc& g = G->g;
  auto dflag = [](int d) { return d == 1 ? MUL_IK : (d == 2 ? MUL_IK2 : 0); };
  const int allk = (mu.sym ? MUL_SYM : 0) | (mu.negk2 ? MUL_NEGK2 : 0);
  const cpx<T>* cur = in;
  int pending = allk;   // multipliers that need every axis spectral: applied in the first pass
  double scale = mu.scale;
  if (g.ndim == 3) {
    AxisProg P{};
    P.nxf = 1;
    P.xf[0] = mkxf(0, 0, dflag(mu.deriv[2]) | pending, 0, true, true, scale);
    P.in[0] = cur;
    P.out[0] = tmp;
    P.symarr = mu.symarr;
    P.axis = 2;
    launch_axis<T>(P, +1, g, twtab<T>(G), st);
    cur = tmp;
    pending = 0;
    scale = 1.0;
  }
  if (g.ndim >= 2) {
    AxisProg P{};
    P.nxf = 1;
    P.xf[0] = mkxf(0, 0, dflag(mu.deriv[1]) | pending, 0, true, true, scale);
    P.in[0] = cur;
    P.out[0] = tmp;
    P.symarr = mu.symarr;
    P.axis = 1;
    launch_axis<T>(P, +1, g, twtab<T>(G), st);
    cur = tmp;
    pending = 0;
    scale = 1.0;
  }
  XProg X{};
  X.ncomp = 1;
  X.mode = 2;
  X.in[0] = cur;
  X.out[0] = out;
  X.pre[0] = dflag(mu.deriv[0]) | pending;
  X.symarr = mu.symarr;
  X.scale = scale / (double)g.nreal;
  launch_xpass<T>(X, g, twtab<T>(G), st);
}

template <typename T>
void fwd_transform_n(const vd_grid* G, int ncomp, const T* in, cpx<T>* out, cudaStream_t st) {
  const GridDesc& g = G->g;
  const size_t nc = (size_t)g.ncplx, nr = (size_t)g.nreal;
  XProg X{};
  X.ncomp = ncomp;
  X.mode = 1;
  for (int c = 0; c < ncomp; ++c) {
    X.in[c] = in + c * nr;
    X.out[c] = out + c * nc;
  }
  X.scale = 0.5;
  launch_xpass<T>(X, g, twtab<T>(G), st);
  for (int axis = 1; axis < g.ndim; ++axis) {
    AxisProg P{};
    P.nxf = ncomp;
    for (int c = 0; c < ncomp; ++c) {
      P.xf[c] = mkxf(c, c, 0, 0, true, true);
      P.in[c] = out + c * nc;
      P.out[c] = out + c * nc;
    }
    P.axis = axis;
    launch_axis<T>(P, -1, g, twtab<T>(G), st);
  }
}

template <typename T>
void inv_transform_n(const vd_grid* G, int ncomp, const cpx<T>* in, T* out, cpx<T>* tmp, cudaStream_t st) {
  const GridDesc& g = G->g;
  const size_t nc = (size_t)g.ncplx, nr = (size_t)g.nreal;
  const cpx<T>* cur = in;
  for (int axis = g.ndim - 1; axis >= 1; --axis) {
    AxisProg P{};
    P.nxf = ncomp;
    for (int c = 0; c < ncomp; ++c) {
      P.xf[c] = mkxf(c, c, 0, 0, true, true);
      P.in[c] = cur + c * nc;
      P.out[c] = tmp + c * nc;
    }
    P.axis = axis;
    launch_axis<T>(P, +1, g, twtab<T>(G), st);
    cur = tmp;
  }
  XProg X{};
  X.ncomp = ncomp;
  X.mode = 2;
  for (int c = 0; c < ncomp; ++c) {
    X.in[c] = cur + c * nc;
    X.out[c] = out + c * nr;
  }
  X.scale = 1.0 / (double)g.nreal;
  launch_xpass<T>(X, g, twtab<T>(G), st);
}

// First and second derivatives of a field from its spectrum rh (double): grad[j] = F^-1(i k_j rh),
// hess[hidx(a, b)] = F^-1((i k_a)(i k_b) rh).  The inverse transforms sharing a z multiplier
// share their z and y passes (each output gets its own transform's multipliers in the same
// passes: the fields are those of separate inverse transforms bit for bit).  tmp: three
// spectral fields.
void derivative_fields(const vd_grid* G, const cpx<double>* rh, double* const grad[3], double* const hess[6],
                       cpx<double>* tmp, cudaStream_t st) {
  const GridDesc& g = G->g;
  const int d = g.ndim;
  const size_t nc = (size_t)g.ncplx;
  const void* tw = G->tw_d;
  auto fl = [](int k) { return k == 1 ? MUL_IK : (k == 2 ? MUL_IK2 : 0); };
  // x pass over a list of (spectral input, x derivative order, output)
  auto xpass = [&](int n, const cpx<double>* const* in, const int* kx, double* const* out) {
    XProg X{};
    X.ncomp = n;
    X.mode = 2;
    for (int c = 0; c < n; ++c) {
      X.in[c] = in[c];
      X.pre[c] = fl(kx[c]);
      X.out[c] = out[c];
    }
    X.scale = 1.0 / (double)g.nreal;
    launch_xpass<double>(X, g, tw, st);
  };
  if (d == 1) {
    const cpx<double>* in[2] = {rh, rh};
    const int kx[2] = {1, 2};
    double* out[2] = {grad[0], hess[hidx(0, 0)]};
    xpass(2, in, kx, out);
    return;
  }
  // outputs by (z order, y order): x orders and destinations
  struct Out {
    int kz, ky, kx;
    double* dst;
  };
  Out outs[9];
  int no = 0;
  for (int j = 0; j < d; ++j) {
    int k[3] = {0, 0, 0};
    k[j] = 1;
    outs[no++] = {k[2], k[1], k[0], grad[j]};
  }
  for (int a = 0; a < d; ++a)
    for (int b = a; b < d; ++b) {
      int k[3] = {0, 0, 0};
      k[a] += 1;
      k[b] += 1;
      outs[no++] = {k[2], k[1], k[0], hess[hidx(a, b)]};
    }
  for (int kz = 0; kz <= (d == 3 ? 2 : 0); ++kz) {
    const cpx<double>* zin = rh;
    if (d == 3) {
      // z inverse with this z multiplier into tmp[0]
      AxisProg P{};
      P.nxf = 1;
      P.xf[0] = mkxf(0, 0, fl(kz), 0, true, true);
      P.in[0] = rh;
      P.out[0] = tmp;
      P.axis = 2;
      launch_axis<double>(P, +1, g, tw, st);
      zin = tmp;
    }
    // y inverse: one output per y order used by this group; the y order 0 in place last
    int ys[3] = {-1, -1, -1};   // y order -> tmp slot
    for (int o = 0; o < no; ++o)
      if (outs[o].kz == kz) ys[outs[o].ky] = 0;
    AxisProg Q{};
    int slot = (d == 3) ? 1 : 0;
    for (int ky = 2; ky >= 0; --ky) {
      if (ys[ky] < 0) continue;
      const bool inplace = (d == 3 && ky == 0);
      ys[ky] = inplace ? 0 : slot++;
      Q.xf[Q.nxf] = mkxf(0, Q.nxf, fl(ky), 0, true, true);
      Q.out[Q.nxf] = tmp + (size_t)ys[ky] * nc;
      ++Q.nxf;
    }
    Q.in[0] = zin;
    Q.axis = 1;
    launch_axis<double>(Q, +1, g, tw, st);
    const cpx<double>* in[kMaxXComp];
    int kx[kMaxXComp];
    double* out[kMaxXComp];
    int n = 0;
    for (int o = 0; o < no; ++o) {
      if (outs[o].kz != kz) continue;
      in[n] = tmp + (size_t)ys[outs[o].ky] * nc;
      kx[n] = outs[o].kx;
      out[n] = outs[o].dst;
      ++n;
    }
    xpass(n, in, kx, out);
  }
}

// Plain transforms with float-pair arithmetic; double fields in and out, float-pair
// intermediates in tmp (one spectral field of 16-byte elements).
void fwd_transform_dd(const vd_grid* G, const double* in, cpx<double>* out, void* tmp, cudaStream_t st) {
  const GridDesc& g = G->g;
  cpx<dd>* t = reinterpret_cast<cpx<dd>*>(tmp);
  XProg X{};
  X.ncomp = 1;
  X.mode = 1;
  X.in[0] = in;
  X.conv_in = 1;
  X.scale = 0.5;
  if (g.ndim == 1) {
    X.out[0] = out;
    X.conv_out = 1;
    launch_xpass<dd>(X, g, G->tw_dd, st);
    return;
  }
  X.out[0] = t;
  launch_xpass<dd>(X, g, G->tw_dd, st);
  AxisProg P{};
  P.nxf = 1;
  P.xf[0] = mkxf(0, 0, 0, 0, true, true);
  P.in[0] = t;
  P.axis = 1;
  if (g.ndim == 2) {
    P.out[0] = out;
    P.conv_out = 1;
    launch_axis<dd>(P, -1, g, G->tw_dd, st);
    return;
  }
  P.out[0] = t;
  launch_axis<dd>(P, -1, g, G->tw_dd, st);
  P.axis = 2;
  P.out[0] = out;
  P.conv_out = 1;
  launch_axis<dd>(P, -1, g, G->tw_dd, st);
}

void inv_transform_dd(const vd_grid* G, const cpx<double>* in, double* out, void* tmp, cudaStream_t st) {
  const GridDesc& g = G->g;
  cpx<dd>* t = reinterpret_cast<cpx<dd>*>(tmp);
  const void* cur = in;
  int conv = 1;
  if (g.ndim == 3) {
    AxisProg P{};
    P.nxf = 1;
    P.xf[0] = mkxf(0, 0, 0, 0, true, true);
    P.in[0] = cur;
    P.out[0] = t;
    P.conv_in = conv;
    P.axis = 2;
    launch_axis<dd>(P, +1, g, G->tw_dd, st);
    cur = t;
    conv = 0;
  }
  if (g.ndim >= 2) {
    AxisProg P{};
    P.nxf = 1;
    P.xf[0] = mkxf(0, 0, 0, 0, true, true);
    P.in[0] = cur;
    P.out[0] = t;
    P.conv_in = conv;
    P.axis = 1;
    launch_axis<dd>(P, +1, g, G->tw_dd, st);
    cur = t;
    conv = 0;
  }
  XProg X{};
  X.ncomp = 1;
  X.mode = 2;
  X.in[0] = cur;
  X.conv_in = conv;
  X.out[0] = out;
  X.conv_out = 1;
  X.scale = 1.0 / (double)g.nreal;
  launch_xpass<dd>(X, g, G->tw_dd, st);
}

// ---------------------------------------------------------------------------------------
// pressure operator
// ---------------------------------------------------------------------------------------

// conv: the float-pair instantiation reads `in` and writes `out` as double fields
// phys_out (may be null): the fused x pass also writes the inverse transform of `in` there,
// equal bit for bit to the separate inverse transform when the apply is unpreconditioned
// wf_pair (float programs, may be null): 1/(N rho) as float pairs, used instead of rinv_s so
// that the multiply runs in float-pair arithmetic (high density ratios)
template <typename T>
static void pressure_impl(const vd_grid* G, const void* in, void* out, const T* symarr, const void* rinv_s,
                          cpx<T>* tmp, const int* done, cudaStream_t st, int conv, void* phys_out = nullptr,
                          const void* wf_pair = nullptr) {
  const int wf_dd = (std::is_same<T, float>::value && wf_pair) ? 1 : 0;
  if (wf_dd) rinv_s = wf_pair;
  const GridDesc& g = G->g;
  const int S = symarr ? MUL_SYM : 0;
  if (symarr) phys_out = nullptr;   // the by-product is the inverse of `in` itself: unpreconditioned applies only
  const size_t nc = (size_t)g.ncplx;
  const void* tw = twtab<T>(G);
  if (g.ndim == 1) {
    XProg X{};
    X.ncomp = 1;
    X.mode = 0;
    X.in[0] = in;
    X.out[0] = out;
    X.pre[0] = S | MUL_IK;
    X.post[0] = MUL_IK;
    X.wfield = rinv_s;
    X.wf_dd = wf_dd;
    X.aux_out = phys_out;
    X.aux_scale = 1.0 / (double)g.nreal;
    X.aux_conv = conv;
    X.scale = 0.5;
    X.symarr = symarr;
    X.done = done;
    X.conv_in = conv;
    X.conv_out = conv;
    launch_xpass<T>(X, g, tw, st);
    return;
  }
  cpx<T>* T0 = tmp;
  cpx<T>* T1 = tmp + nc;
  if (g.ndim == 2) {
    // y inverse: T1 = F_y^-1(i ky S v), T0 = F_y^-1(S v)
    AxisProg P{};
    P.nxf = 2;
    P.xf[0] = mkxf(0, 1, S | MUL_IK, 0, true, true);
    P.xf[1] = mkxf(0, 0, S, 0, true, true);
    P.in[0] = in;
    P.out[0] = T0;
    P.out[1] = T1;
    P.symarr = symarr;
    P.done = done;
    P.axis = 1;
    P.conv_in = conv;
    launch_axis<T>(P, +1, g, tw, st);
    // x fused: T0 <- i kx R2C(w C2R(i kx T0)), T1 <- R2C(w C2R(T1))
    XProg X{};
    X.ncomp = 2;
    X.mode = 0;
    X.in[0] = T0;
    X.out[0] = T0;
    X.pre[0] = MUL_IK;
    X.post[0] = MUL_IK;
    X.in[1] = T1;
    X.out[1] = T1;
    X.wfield = rinv_s;
    X.wf_dd = wf_dd;
    X.aux_out = phys_out;
    X.aux_scale = 1.0 / (double)g.nreal;
    X.aux_conv = conv;
    X.scale = 0.5;
    X.done = done;
    launch_xpass<T>(X, g, tw, st);
    // y forward + divergence: out = F_y(T0) + i ky F_y(T1)
    AxisProg Q{};
    Q.nxf = 2;
    Q.xf[0] = mkxf(0, 0, 0, 0, true, false);
    Q.xf[1] = mkxf(1, 0, 0, MUL_IK, false, true);
    Q.in[0] = T0;
    Q.in[1] = T1;
    Q.out[0] = out;
    Q.done = done;
    Q.axis = 1;
    Q.conv_out = conv;
    launch_axis<T>(Q, -1, g, tw, st);
    return;
  }
  cpx<T>* T2 = tmp + 2 * nc;
  // P1, z inverse: T0 = F_z^-1(S v), T1 = F_z^-1(i kz S v)
  {
    AxisProg P{};
    P.nxf = 2;
    P.xf[0] = mkxf(0, 1, S | MUL_IK, 0, true, true);
    P.xf[1] = mkxf(0, 0, S, 0, true, true);
    P.in[0] = in;
    P.out[0] = T0;
    P.out[1] = T1;
    P.symarr = symarr;
    P.done = done;
    P.axis = 2;
    P.conv_in = conv;
    launch_axis<T>(P, +1, g, tw, st);
  }
  // P2, y inverse: T2 = F_y^-1(i ky T0), T0 <- F_y^-1(T0), T1 <- F_y^-1(T1)
  {
    AxisProg P{};
    P.nxf = 3;
    P.xf[0] = mkxf(0, 2, MUL_IK, 0, true, true);
    P.xf[1] = mkxf(0, 0, 0, 0, true, true);
    P.xf[2] = mkxf(1, 1, 0, 0, true, true);
    P.in[0] = T0;
    P.in[1] = T1;
    P.out[0] = T0;
    P.out[1] = T1;
    P.out[2] = T2;
    P.done = done;
    P.axis = 1;
    launch_axis<T>(P, +1, g, tw, st);
  }
  // P3, x fused (in place): T0 <- i kx R2C(w C2R(i kx T0)), T2 <- R2C(w C2R(T2)), T1 likewise
  {
    XProg X{};
    X.ncomp = 3;
    X.mode = 0;
    X.in[0] = T0;
    X.out[0] = T0;
    X.pre[0] = MUL_IK;
    X.post[0] = MUL_IK;
    X.in[1] = T2;
    X.out[1] = T2;
    X.in[2] = T1;
    X.out[2] = T1;
    X.wfield = rinv_s;
    X.wf_dd = wf_dd;
    X.aux_out = phys_out;
    X.aux_scale = 1.0 / (double)g.nreal;
    X.aux_conv = conv;
    X.scale = 0.5;
    X.done = done;
    launch_xpass<T>(X, g, tw, st);
  }
  // P4, y forward: T0 <- F_y(T0) + i ky F_y(T2), T1 <- F_y(T1)
  {
    AxisProg P{};
    P.nxf = 3;
    P.xf[0] = mkxf(0, 0, 0, 0, true, false);
    P.xf[1] = mkxf(1, 0, 0, MUL_IK, false, true);
    P.xf[2] = mkxf(2, 1, 0, 0, true, true);
    P.in[0] = T0;
    P.in[1] = T2;
    P.in[2] = T1;
    P.out[0] = T0;
    P.out[1] = T1;
    P.done = done;
    P.axis = 1;
    launch_axis<T>(P, -1, g, tw, st);
  }
  // P5, z forward + divergence: out = F_z(T0) + i kz F_z(T1)
  {
    AxisProg P{};
    P.nxf = 2;
    P.xf[0] = mkxf(0, 0, 0, 0, true, false);
    P.xf[1] = mkxf(1, 0, 0, MUL_IK, false, true);
    P.in[0] = T0;
    P.in[1] = T1;
    P.out[0] = out;
    P.done = done;
    P.axis = 2;
    P.conv_out = conv;
    launch_axis<T>(P, -1, g, tw, st);
  }
}

template <typename T>
void apply_pressure_spec(const vd_grid* G, const cpx<T>* in, cpx<T>* out, const T* symarr, const T* rinv_s,
                         cpx<T>* tmp, const int* done, cudaStream_t st, const void* wf_pair) {
  pressure_impl<T>(G, in, out, symarr, rinv_s, tmp, done, st, 0, nullptr, wf_pair);
}

void apply_pressure_spec_dd(const vd_grid* G, const cpx<double>* in, cpx<double>* out, void* tmp, const int* done,
                            cudaStream_t st, double* phys_out) {
  pressure_impl<dd>(G, in, out, nullptr, G->rinv_s_dd, reinterpret_cast<cpx<dd>*>(tmp), done, st, 1, phys_out);
}

// ---------------------------------------------------------------------------------------
// K_rho operator (Eq. VDINSE.Krho): two scalar transforms with the coefficient multiply
// fused into the x pass, plus the pointwise local term
// ---------------------------------------------------------------------------------------

int krho_tmp_fields(int ndim) { return ndim >= 2 ? 1 : 0; }

// out += Lap S in: with_inv (S = pseudo-inverse of Lap): the mean-free part of in; otherwise
// -|k|^2 in.  Double I/O for the float-pair path (conv), else type T.
template <typename T>
__global__ void k_krho_local(GridDesc g, const cpx<T>* __restrict__ in, cpx<T>* __restrict__ out, int with_inv,
                             const int* done) {
  if (done && *done) return;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < g.ncplx;
       e += (long long)gridDim.x * blockDim.x) {
    const cpx<T> v = in[e];
    cpx<T> o = out[e];
    if (with_inv) {
      if (e != 0) o = o + v;
    } else {
      const long long line = e / g.h0;
      const int kxi = (int)(e - line * g.h0);
      const int kyi = (int)(line % g.n1);
      const int kzi = (int)(line / g.n1);
      const T kx = (T)g.kfac[0] * (T)freq_full(kxi, g.n0);
      T k2 = kx * kx;
      if (g.ndim >= 2) {
        const T ky = (T)g.kfac[1] * (T)freq_full(kyi, g.n1);
        k2 += ky * ky;
      }
      if (g.ndim == 3) {
        const T kz = (T)g.kfac[2] * (T)freq_full(kzi, g.n2);
        k2 += kz * kz;
      }
      o = o - scal(v, k2);
    }
    out[e] = o;
  }
}

template <typename U>
static void krho_local(const vd_grid* G, const void* in, void* out, bool with_inv, const int* done, cudaStream_t st) {
  const long long n = G->g.ncplx;
  const int blocks = (int)std::min<long long>((n + 255) / 256, 4096);
  k_krho_local<U><<<blocks, 256, 0, st>>>(G->g, (const cpx<U>*)in, (cpx<U>*)out, with_inv ? 1 : 0, done);
  count_launch();
}

// out = F(c F^-1(S in)) through the pass chain; conv: float-pair arithmetic on double fields
template <typename T>
static void krho_transforms(const vd_grid* G, const void* in, void* out, const T* symarr, const void* coef_s,
                            cpx<T>* tmp, const int* done, cudaStream_t st, int conv, const void* wf_pair = nullptr) {
  const GridDesc& g = G->g;
  const int wf_dd = (std::is_same<T, float>::value && wf_pair) ? 1 : 0;
  if (wf_dd) coef_s = wf_pair;
  const int S = symarr ? MUL_SYM : 0;
  const void* tw = twtab<T>(G);
  if (g.ndim == 1) {
    XProg X{};
    X.ncomp = 1;
    X.mode = 0;
    X.in[0] = in;
    X.out[0] = out;
    X.pre[0] = S;
    X.wfield = coef_s;
    X.wf_dd = wf_dd;
    X.scale = 0.5;
    X.symarr = symarr;
    X.done = done;
    X.conv_in = conv;
    X.conv_out = conv;
    launch_xpass<T>(X, g, tw, st);
    return;
  }
  // inverse along z (3D) and y, in the order z, y: T0 = F_y^-1 F_z^-1 (S in)
  const void* cur = in;
  int cin = conv;
  int pre = S;
  if (g.ndim == 3) {
    AxisProg P{};
    P.nxf = 1;
    P.xf[0] = mkxf(0, 0, pre, 0, true, true);
    P.in[0] = cur;
    P.out[0] = tmp;
    P.symarr = symarr;
    P.done = done;
    P.axis = 2;
    P.conv_in = cin;
    launch_axis<T>(P, +1, g, tw, st);
    cur = tmp;
    cin = 0;
    pre = 0;
  }
  {
    AxisProg P{};
    P.nxf = 1;
    P.xf[0] = mkxf(0, 0, pre, 0, true, true);
    P.in[0] = cur;
    P.out[0] = tmp;
    P.symarr = symarr;
    P.done = done;
    P.axis = 1;
    P.conv_in = cin;
    launch_axis<T>(P, +1, g, tw, st);
  }
  // x fused (in place): T0 <- R2C(c C2R(T0))
  {
    XProg X{};
    X.ncomp = 1;
    X.mode = 0;
    X.in[0] = tmp;
    X.out[0] = tmp;
    X.wfield = coef_s;
    X.wf_dd = wf_dd;
    X.scale = 0.5;
    X.done = done;
    launch_xpass<T>(X, g, tw, st);
  }
  // forward along y, then z
  {
    AxisProg P{};
    P.nxf = 1;
    P.xf[0] = mkxf(0, 0, 0, 0, true, true);
    P.in[0] = tmp;
    P.out[0] = (g.ndim == 3) ? (void*)tmp : out;
    P.done = done;
    P.axis = 1;
    P.conv_out = (g.ndim == 3) ? 0 : conv;
    launch_axis<T>(P, -1, g, tw, st);
  }
  if (g.ndim == 3) {
    AxisProg P{};
    P.nxf = 1;
    P.xf[0] = mkxf(0, 0, 0, 0, true, true);
    P.in[0] = tmp;
    P.out[0] = out;
    P.done = done;
    P.axis = 2;
    P.conv_out = conv;
    launch_axis<T>(P, -1, g, tw, st);
  }
}

template <typename T>
void apply_krho_spec(const vd_grid* G, const cpx<T>* in, cpx<T>* out, const T* symarr, const T* coef_s,
                     cpx<T>* tmp, const int* done, cudaStream_t st, const void* wf_pair) {
  krho_transforms<T>(G, in, out, symarr, coef_s, tmp, done, st, 0, wf_pair);
  krho_local<T>(G, in, out, symarr != nullptr, done, st);
}

void apply_krho_spec_dd(const vd_grid* G, const cpx<double>* in, cpx<double>* out, void* tmp, const int* done,
                        cudaStream_t st) {
  krho_transforms<dd>(G, in, out, nullptr, G->kc_dd, reinterpret_cast<cpx<dd>*>(tmp), done, st, 1);
  krho_local<double>(G, in, out, false, done, st);
}

// ---------------------------------------------------------------------------------------
// velocity operator
// ---------------------------------------------------------------------------------------

void spec_axpby_sym_launch(const vd_grid* G, int sz, int ncomp, const void* x, const void* symarr, double alpha,
                           const void* y, double beta, void* out, const int* done, cudaStream_t st);
void velocity_combine_launch(const vd_grid* G, int sz, const void* u, const void* du, void* lap, double inv_sc,
                             const int* done, cudaStream_t st);

template <typename T>
void apply_velocity_spec(const vd_grid* G, const cpx<T>* in, cpx<T>* out, const T* symarr, double a,
                         double inv_sc, cpx<T>* tmp, const int* done, cudaStream_t st) {
  const GridDesc& g = G->g;
  const int d = g.ndim;
  const size_t nc = (size_t)g.ncplx;
  const size_t nr = (size_t)g.nreal;
  // physical scratch carved from spectral-sized temporaries (a spectral field holds >= nreal reals)
  cpx<T>* ttmp = tmp;                                      // spectral temporaries: ttmp[0..ns)
  const int ns = velocity_spec_tmps(d);
  T* u = reinterpret_cast<T*>(tmp + nc * ns);              // d fields
  T* du = reinterpret_cast<T*>(tmp + nc * (ns + d));       // d*d fields
  T* lap = reinterpret_cast<T*>(tmp + nc * (ns + d + d * d));  // d fields
  static_assert(sizeof(cpx<T>) == 2 * sizeof(T), "layout");
  const void* tw = twtab<T>(G);
  const int S = symarr ? MUL_SYM : 0;
  // u_i = F^-1(S in_i), du_ij = F^-1(i k_j S in_i), lap_i = F^-1(-|k|^2 S in_i): the d + 2
  // inverse transforms of a component share their passes.  Each output gets the multipliers
  // of its own inverse transform, in the same passes, so the fields equal those of d + 2
  // separate inverse transforms bit for bit.
  for (int i = 0; i < d; ++i) {
    const cpx<T>* vi = in + i * nc;
    XProg X{};
    X.mode = 2;
    X.symarr = symarr;
    X.done = done;
    X.scale = 1.0 / (double)g.nreal;
    if (d == 1) {
      // u (S), du (i k S), lap (-k^2 S) straight from the spectrum
      X.ncomp = 3;
      X.in[0] = X.in[1] = X.in[2] = vi;
      X.pre[0] = S;
      X.pre[1] = S | MUL_IK;
      X.pre[2] = S | MUL_NEGK2;
      X.out[0] = u + i * nr;
      X.out[1] = du + i * nr;
      X.out[2] = lap + i * nr;
      launch_xpass<T>(X, g, tw, st);
      continue;
    }
    cpx<T>* A = ttmp;            // S v, then its y inverse
    cpx<T>* B = ttmp + nc;       // i k_y S v after the y inverse (3D: from A)
    cpx<T>* Cf = ttmp + 2 * nc;  // -|k|^2 S v
    cpx<T>* Z = ttmp + 3 * nc;   // 3D: i k_z S v
    if (d == 3) {
      // z inverse: A = F_z^-1(S v), Z = F_z^-1(i k_z S v), Cf = F_z^-1(-|k|^2 S v)
      AxisProg P{};
      P.nxf = 3;
      P.xf[0] = mkxf(0, 0, S, 0, true, true);
      P.xf[1] = mkxf(0, 1, S | MUL_IK, 0, true, true);
      P.xf[2] = mkxf(0, 2, S | MUL_NEGK2, 0, true, true);
      P.in[0] = vi;
      P.out[0] = A;
      P.out[1] = Z;
      P.out[2] = Cf;
      P.symarr = symarr;
      P.done = done;
      P.axis = 2;
      launch_axis<T>(P, +1, g, tw, st);
      // y inverse: B = F_y^-1(i k_y A) before A is transformed in place; Z, Cf in place
      AxisProg Q{};
      Q.nxf = 4;
      Q.xf[0] = mkxf(0, 1, MUL_IK, 0, true, true);
      Q.xf[1] = mkxf(0, 0, 0, 0, true, true);
      Q.xf[2] = mkxf(1, 2, 0, 0, true, true);
      Q.xf[3] = mkxf(2, 3, 0, 0, true, true);
      Q.in[0] = A;
      Q.in[1] = Z;
      Q.in[2] = Cf;
      Q.out[0] = A;
      Q.out[1] = B;
      Q.out[2] = Z;
      Q.out[3] = Cf;
      Q.done = done;
      Q.axis = 1;
      launch_axis<T>(Q, +1, g, tw, st);
    } else {
      // y inverse of the spectrum: A = F_y^-1(S v), B = F_y^-1(i k_y S v), Cf = F_y^-1(-|k|^2 S v)
      AxisProg Q{};
      Q.nxf = 3;
      Q.xf[0] = mkxf(0, 0, S, 0, true, true);
      Q.xf[1] = mkxf(0, 1, S | MUL_IK, 0, true, true);
      Q.xf[2] = mkxf(0, 2, S | MUL_NEGK2, 0, true, true);
      Q.in[0] = vi;
      Q.out[0] = A;
      Q.out[1] = B;
      Q.out[2] = Cf;
      Q.symarr = symarr;
      Q.done = done;
      Q.axis = 1;
      launch_axis<T>(Q, +1, g, tw, st);
    }
    // x inverse: u (A), du_x (i k_x A), du_y (B), [du_z (Z),] lap (Cf)
    const cpx<T>* xin[5] = {A, A, B, Z, Cf};
    T* xout[5] = {u + i * nr, du + (i * d + 0) * nr, du + (i * d + 1) * nr, du + (i * d + 2) * nr, lap + i * nr};
    const int xpre[5] = {0, MUL_IK, 0, 0, 0};
    X.ncomp = 0;
    for (int c = 0; c < 5; ++c) {
      if (d == 2 && c == 3) continue;   // no z derivative
      X.in[X.ncomp] = xin[c];
      X.out[X.ncomp] = xout[c];
      X.pre[X.ncomp] = xpre[c];
      ++X.ncomp;
    }
    launch_xpass<T>(X, g, tw, st);
  }
  // pointwise bracket g_i = rho^-1 (lap_i + Sc^-1 sum_j (u_j D_j D_i rho + D_j rho D_j u_i)),
  // written over lap_i
  velocity_combine_launch(G, (int)sizeof(T), u, du, lap, inv_sc, done, st);
  // F(g_i) for all components at once (each as its own forward transform), then
  // out_i = S in_i - a F(g_i)
  fwd_transform_n<T>(G, d, lap, ttmp, st);
  spec_axpby_sym_launch(G, (int)sizeof(T), d, in, symarr, 1.0, ttmp, -a, out, done, st);
}

// The velocity operator without preconditioner in float-pair arithmetic (the refinement
// residual of mixed_dd): double spectral fields in and out, the transforms of
// apply_velocity_spec in float pairs (split from double on the first pass's loads, summed to
// double on the last pass's stores), the physical fields u, du, lap in double so that the
// pointwise bracket is the double one.  tmp: velocity_tmp_fields(d) fields of 16-byte complex
// elements (the float-pair spectral scratch takes the same room as double).
void apply_velocity_spec_dd(const vd_grid* G, const cpx<double>* in, cpx<double>* out, double a, double inv_sc,
                            void* tmp_, const int* done, cudaStream_t st) {
  const GridDesc& g = G->g;
  const int d = g.ndim;
  const size_t nc = (size_t)g.ncplx;
  const size_t nr = (size_t)g.nreal;
  cpx<dd>* ttmp = reinterpret_cast<cpx<dd>*>(tmp_);
  cpx<double>* dtmp = reinterpret_cast<cpx<double>*>(tmp_);
  const int ns = velocity_spec_tmps(d);
  double* u = reinterpret_cast<double*>(dtmp + nc * ns);
  double* du = reinterpret_cast<double*>(dtmp + nc * (ns + d));
  double* lap = reinterpret_cast<double*>(dtmp + nc * (ns + d + d * d));
  const void* tw = G->tw_dd;
  for (int i = 0; i < d; ++i) {
    const cpx<double>* vi = in + i * nc;
    XProg X{};
    X.mode = 2;
    X.done = done;
    X.scale = 1.0 / (double)g.nreal;
    if (d == 1) {
      X.ncomp = 3;
      X.in[0] = X.in[1] = X.in[2] = vi;
      X.pre[0] = 0;
      X.pre[1] = MUL_IK;
      X.pre[2] = MUL_NEGK2;
      X.out[0] = u + i * nr;
      X.out[1] = du + i * nr;
      X.out[2] = lap + i * nr;
      X.conv_in = 7;
      X.conv_out = 7;
      launch_xpass<dd>(X, g, tw, st);
      continue;
    }
    cpx<dd>* A = ttmp;
    cpx<dd>* B = ttmp + nc;
    cpx<dd>* Cf = ttmp + 2 * nc;
    cpx<dd>* Z = ttmp + 3 * nc;
    if (d == 3) {
      AxisProg P{};
      P.nxf = 3;
      P.xf[0] = mkxf(0, 0, 0, 0, true, true);
      P.xf[1] = mkxf(0, 1, MUL_IK, 0, true, true);
      P.xf[2] = mkxf(0, 2, MUL_NEGK2, 0, true, true);
      P.in[0] = vi;
      P.conv_in = 1;
      P.out[0] = A;
      P.out[1] = Z;
      P.out[2] = Cf;
      P.done = done;
      P.axis = 2;
      launch_axis<dd>(P, +1, g, tw, st);
      AxisProg Q{};
      Q.nxf = 4;
      Q.xf[0] = mkxf(0, 1, MUL_IK, 0, true, true);
      Q.xf[1] = mkxf(0, 0, 0, 0, true, true);
      Q.xf[2] = mkxf(1, 2, 0, 0, true, true);
      Q.xf[3] = mkxf(2, 3, 0, 0, true, true);
      Q.in[0] = A;
      Q.in[1] = Z;
      Q.in[2] = Cf;
      Q.out[0] = A;
      Q.out[1] = B;
      Q.out[2] = Z;
      Q.out[3] = Cf;
      Q.done = done;
      Q.axis = 1;
      launch_axis<dd>(Q, +1, g, tw, st);
    } else {
      AxisProg Q{};
      Q.nxf = 3;
      Q.xf[0] = mkxf(0, 0, 0, 0, true, true);
      Q.xf[1] = mkxf(0, 1, MUL_IK, 0, true, true);
      Q.xf[2] = mkxf(0, 2, MUL_NEGK2, 0, true, true);
      Q.in[0] = vi;
      Q.conv_in = 1;
      Q.out[0] = A;
      Q.out[1] = B;
      Q.out[2] = Cf;
      Q.done = done;
      Q.axis = 1;
      launch_axis<dd>(Q, +1, g, tw, st);
    }
    const cpx<dd>* xin[5] = {A, A, B, Z, Cf};
    double* xout[5] = {u + i * nr, du + (i * d + 0) * nr, du + (i * d + 1) * nr, du + (i * d + 2) * nr, lap + i * nr};
    const int xpre[5] = {0, MUL_IK, 0, 0, 0};
    X.ncomp = 0;
    for (int c = 0; c < 5; ++c) {
      if (d == 2 && c == 3) continue;
      X.in[X.ncomp] = xin[c];
      X.out[X.ncomp] = xout[c];
      X.pre[X.ncomp] = xpre[c];
      ++X.ncomp;
    }
    X.conv_out = (1 << X.ncomp) - 1;
    launch_xpass<dd>(X, g, tw, st);
  }
  velocity_combine_launch(G, 8, u, du, lap, inv_sc, done, st);
  // F(g_i): x pass from the double brackets, y (and z) passes, the last one summing to double
  cpx<double>* F = dtmp;   // over the float-pair scratch, element by element on the last pass
  {
    XProg X{};
    X.ncomp = d;
    X.mode = 1;
    for (int i = 0; i < d; ++i) {
      X.in[i] = lap + i * nr;
      X.out[i] = ttmp + i * nc;
    }
    X.conv_in = (1 << d) - 1;
    if (d == 1) X.conv_out = 1;
    X.scale = 0.5;
    X.done = done;
    launch_xpass<dd>(X, g, tw, st);
    for (int axis = 1; axis < d; ++axis) {
      AxisProg P{};
      P.nxf = d;
      for (int i = 0; i < d; ++i) {
        P.xf[i] = mkxf(i, i, 0, 0, true, true);
        P.in[i] = ttmp + i * nc;
        P.out[i] = ttmp + i * nc;
      }
      if (axis == d - 1) P.conv_out = (1 << d) - 1;
      P.done = done;
      P.axis = axis;
      launch_axis<dd>(P, -1, g, tw, st);
    }
  }
  spec_axpby_sym_launch(G, 8, d, in, nullptr, 1.0, F, -a, out, done, st);
}

// ---------------------------------------------------------------------------------------
// small pointwise kernels used above
// ---------------------------------------------------------------------------------------

// over ncomp fields of nc elements stored back to back, the symbol indexed per field
template <typename T>
__global__ void k_spec_axpby_sym(long long n, long long nc, const cpx<T>* __restrict__ x, const T* __restrict__ sym,
                                 T alpha, const cpx<T>* __restrict__ y, T beta, cpx<T>* __restrict__ out,
                                 const int* done) {
  if (done && *done) return;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const T s = sym ? sym[e % nc] * alpha : alpha;
    out[e] = scal(x[e], s) + scal(y[e], beta);
  }
}

void spec_axpby_sym_launch(const vd_grid* G, int sz, int ncomp, const void* x, const void* symarr, double alpha,
                           const void* y, double beta, void* out, const int* done, cudaStream_t st) {
  const long long nc = G->g.ncplx;
  const long long n = nc * ncomp;
  const int blocks = (int)std::min<long long>((n + 255) / 256, 4096);
  if (sz == 8)
    { k_spec_axpby_sym<double><<<blocks, 256, 0, st>>>(n, nc, (const cpx<double>*)x, (const double*)symarr, alpha,
                                                     (const cpx<double>*)y, beta, (cpx<double>*)out, done); count_launch(); }
  else
    { k_spec_axpby_sym<float><<<blocks, 256, 0, st>>>(n, nc, (const cpx<float>*)x, (const float*)symarr, (float)alpha,
                                                    (const cpx<float>*)y, (float)beta, (cpx<float>*)out, done); count_launch(); }
}

struct DensPtrs {
  const double* g[3];
  const double* h[6];
};

template <typename T>
__global__ void k_vel_combine(int d, long long nreal, const T* __restrict__ u, const T* __restrict__ du,
                              T* __restrict__ lap, const double* __restrict__ rho, DensPtrs dp, double inv_sc,
                              const int* done) {
  if (done && *done) return;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nreal;
       e += (long long)gridDim.x * blockDim.x) {
    const double rinv = 1.0 / rho[e];
    T out[3];
    for (int i = 0; i < d; ++i) {
      double t = 0.0;
      for (int j = 0; j < d; ++j) {
        const int a = i < j ? i : j, b = i < j ? j : i;
        const int hi = (a == 0) ? b : (a == 1 ? 2 + b : 5);
        t += (double)u[j * nreal + e] * dp.h[hi][e] + dp.g[j][e] * (double)du[(i * d + j) * nreal + e];
      }
      out[i] = (T)(rinv * ((double)lap[i * nreal + e] + inv_sc * t));
    }
    for (int i = 0; i < d; ++i) lap[i * nreal + e] = out[i];
  }
}

void velocity_combine_launch(const vd_grid* G, int sz, const void* u, const void* du, void* lap, double inv_sc,
                             const int* done, cudaStream_t st) {
  const long long n = G->g.nreal;
  DensPtrs dp;
  for (int j = 0; j < 3; ++j) dp.g[j] = G->grho[j];
  for (int j = 0; j < 6; ++j) dp.h[j] = G->hrho[j];
  const int blocks = (int)std::min<long long>((n + 255) / 256, 4096);
  if (sz == 8)
    { k_vel_combine<double><<<blocks, 256, 0, st>>>(G->g.ndim, n, (const double*)u, (const double*)du, (double*)lap,
                                                  G->rho, dp, inv_sc, done); count_launch(); }
  else
    { k_vel_combine<float><<<blocks, 256, 0, st>>>(G->g.ndim, n, (const float*)u, (const float*)du, (float*)lap,
                                                 G->rho, dp, inv_sc, done); count_launch(); }
}

// ---------------------------------------------------------------------------------------
// symbol arrays
// ---------------------------------------------------------------------------------------

template <typename T>
__global__ void k_fill_symbol(GridDesc g, int kind, double a, T* __restrict__ out) {
  // field offsets fit in 32 bits (ncplx < 2^31 is checked when the grid is created)
  const int nc = (int)g.ncplx;
  // K_rho symbols use the full wavenumbers (Nyquist kept); the others k~
  const bool full = (kind == SYM_KLAP_INV || kind == SYM_KLAP);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nc; e += gridDim.x * blockDim.x) {
    const int line = e / g.h0;
    const int kxi = e - line * g.h0;
    const int kyi = line % g.n1;
    const int kzi = line / g.n1;
    auto fq = [&](int m, int n) { return full ? freq_full(m, n) : freq_tilde(m, n); };
    const T kx = (T)g.kfac[0] * (T)fq(kxi, g.n0);
    T k2 = kx * kx;
    if (g.ndim >= 2) {
      const T ky = (T)g.kfac[1] * (T)fq(kyi, g.n1);
      k2 += ky * ky;
    }
    if (g.ndim == 3) {
      const T kz = (T)g.kfac[2] * (T)fq(kzi, g.n2);
      k2 += kz * kz;
    }
    T v = T(1);
    if (kind == SYM_PRESSURE || kind == SYM_KLAP_INV) v = (k2 == T(0)) ? T(0) : -recip(k2);
    else if (kind == SYM_VELOCITY) v = recip(T(1) + (T)a * k2);
    else if (kind == SYM_PROJECT) v = (k2 == T(0)) ? T(0) : T(1);
    else if (kind == SYM_KLAP) v = -k2;
    out[e] = v;
  }
}

template <typename T>
void fill_symbol(const vd_grid* G, int kind, double a, T* out, cudaStream_t st) {
  const long long n = G->g.ncplx;
  const int blocks = (int)std::min<long long>((n + 255) / 256, 4096);
  { k_fill_symbol<T><<<blocks, 256, 0, st>>>(G->g, kind, a, out); count_launch(); }
}

template void fwd_transform<double>(const vd_grid*, const double*, cpx<double>*, cudaStream_t);
template void fwd_transform_n<double>(const vd_grid*, int, const double*, cpx<double>*, cudaStream_t);
template void fwd_transform_n<float>(const vd_grid*, int, const float*, cpx<float>*, cudaStream_t);
template void inv_transform_n<double>(const vd_grid*, int, const cpx<double>*, double*, cpx<double>*, cudaStream_t);
template void inv_transform_n<float>(const vd_grid*, int, const cpx<float>*, float*, cpx<float>*, cudaStream_t);
template void fwd_transform<float>(const vd_grid*, const float*, cpx<float>*, cudaStream_t);
template void inv_transform<double>(const vd_grid*, const cpx<double>*, const Mult&, double*, cpx<double>*,
                                    cudaStream_t);
template void inv_transform<float>(const vd_grid*, const cpx<float>*, const Mult&, float*, cpx<float>*, cudaStream_t);
template void apply_krho_spec<double>(const vd_grid*, const cpx<double>*, cpx<double>*, const double*,
                                      const double*, cpx<double>*, const int*, cudaStream_t, const void*);
template void apply_krho_spec<float>(const vd_grid*, const cpx<float>*, cpx<float>*, const float*, const float*,
                                     cpx<float>*, const int*, cudaStream_t, const void*);
template void apply_pressure_spec<double>(const vd_grid*, const cpx<double>*, cpx<double>*, const double*,
                                          const double*, cpx<double>*, const int*, cudaStream_t, const void*);
template void apply_pressure_spec<float>(const vd_grid*, const cpx<float>*, cpx<float>*, const float*, const float*,
                                         cpx<float>*, const int*, cudaStream_t, const void*);
template void apply_velocity_spec<double>(const vd_grid*, const cpx<double>*, cpx<double>*, const double*, double,
                                          double, cpx<double>*, const int*, cudaStream_t);
template void apply_velocity_spec<float>(const vd_grid*, const cpx<float>*, cpx<float>*, const float*, double,
                                         double, cpx<float>*, const int*, cudaStream_t);
template void fill_symbol<double>(const vd_grid*, int, double, double*, cudaStream_t);
template void fill_symbol<float>(const vd_grid*, int, double, float*, cudaStream_t);

}  // namespace vd
