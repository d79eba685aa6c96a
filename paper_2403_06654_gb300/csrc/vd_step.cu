// One semi-implicit, second-order fractional step on the GPU (Sec. 2 of the paper):
//
//  1. mass, Crank--Nicolson diffusion + Adams--Bashforth advection (Eq. VDINSE.num.mass.proj),
//     diagonal in Fourier: (1 + c|k~|^2) rho^ = (1 - c|k~|^2) rho^n^ - dt [u.grad rho]^, c = dt/(2 Re Sc);
//  2. rho_h = (rho^{n+1} + rho^n)/2;
//  3. predictor (Eq. VDINSE.num.momentum.proj): V~_{rho_h} u* = u + dt(-[u.grad u] - grad p/rho_h + f)
//     + (dt/2) zeta(rho_h, u), with (dt/2) zeta(rho, w) = w - V~_rho w and a = dt/(2 Re);
//  4. pressure (Eq. VDINSE.Lrho.num): L~_{rho_h} phi = div u* / dt;
//  5. projection (Eq. VDINSE.num.proj): u^{n+1} = u* - dt grad phi / rho_h;
//  6. pressure update in the scalar form (Eq. VDINSE.num.p.update), stored as its gradient:
//     grad p += grad phi - grad Lap^+ div(c),  c = rho_h (dt/2) zeta(rho_h, grad phi / rho_h).
//     The gradient form (Eq. VDINSE.num.gradp.update, grad p += grad phi - c) would keep the
//     solenoidal part of c, which with variable density accumulates into grad p and costs the
//     scheme its second order in time at strong viscosity (Sec. 4.1: Re = 1, s = 10).
// Optional sources (vd_flow_set_sources; Sec. 4.1 adds them so that a manufactured field is an
// exact solution): a mass source S and a body force F, both at t^{n+1/2}, enter as
// -dt [u.grad rho - S] in step 1 and +dt F in step 3.
// Readings: Adams--Bashforth 2 (1.5 N^n - 0.5 N^{n-1}), Euler on the first step; periodic
// gravity f = -Fr^-1 (1 - <rho_h>/rho_h) e_g.  Both solves are warm-started from the
// previous solution (u^n for u*, the previous phi for phi).
#include "vd_internal.h"
#include "vd_prof.h"

#include <algorithm>
#include <cstring>
#include <vector>

struct vd_flow {
  vd_grid* G;
  vd_flow_params p;
  int d;
  size_t nr;
  // state
  double *rho, *u, *gradp, *phi, *nrho_prev, *nu_prev;
  int have_prev;
  // optional sources at t^{n+1/2}
  double *msrc, *force;
  int has_msrc, has_force;
  // temporaries
  double *rho_new, *rho_h, *grad, *nrho, *nu, *rhs, *hz, *ustar, *fphi, *w, *sum;
  void* spec;          // 3 spectral fields
  size_t spec_bytes;
  void* dens;          // density workspace (velocity data)
  size_t dens_bytes;
  void* ws;            // solve / apply workspace
  size_t ws_bytes;
};

namespace vd {

#define EW_LOOP(e, n) \
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < (n); e += (long long)gridDim.x * blockDim.x)

// out = sum_j a_j b_j   (a, b: d fields of n points)
__global__ void k_dotvec(long long n, int d, const double* __restrict__ a, const double* __restrict__ b,
                         double* __restrict__ out) {
  EW_LOOP(e, n) {
    double s = 0.0;
    for (int j = 0; j < d; ++j) s += a[j * n + e] * b[j * n + e];
    out[e] = s;
  }
}
// out = alpha x + beta y
__global__ void k_lin(long long n, double alpha, const double* __restrict__ x, double beta, const double* __restrict__ y,
                      double* __restrict__ out) {
  EW_LOOP(e, n) { out[e] = alpha * x[e] + (y ? beta * y[e] : 0.0); }
}
// spectral Crank--Nicolson mass update
__global__ void k_mass(GridDesc g, double c, double dt, const cpx<double>* __restrict__ rh,
                       const cpx<double>* __restrict__ ab, cpx<double>* __restrict__ out) {
  EW_LOOP(e, g.ncplx) {
    const long long line = e / g.h0;
    const int kxi = (int)(e - line * g.h0);
    const int kyi = (int)(line % g.n1);
    const int kzi = (int)(line / g.n1);
    const double kx = g.kfac[0] * freq_tilde(kxi, g.n0);
    double k2 = kx * kx;
    if (g.ndim >= 2) {
      const double ky = g.kfac[1] * freq_tilde(kyi, g.n1);
      k2 += ky * ky;
    }
    if (g.ndim == 3) {
      const double kz = g.kfac[2] * freq_tilde(kzi, g.n2);
      k2 += kz * kz;
    }
    const double a = 1.0 - c * k2, b = 1.0 / (1.0 + c * k2);
    out[e] = mk<double>((a * rh[e].x - dt * ab[e].x) * b, (a * rh[e].y - dt * ab[e].y) * b);
  }
}
// predictor right-hand side (fext: optional body force, d fields)
__global__ void k_rhs(long long n, int d, const double* __restrict__ u, const double* __restrict__ ab,
                      const double* __restrict__ gradp, const double* __restrict__ rho_h, const double* __restrict__ hz,
                      double dt, int gaxis, double inv_fr, double mean_rho, const double* __restrict__ fext,
                      double* __restrict__ out) {
  EW_LOOP(e, n) {
    const double r = rho_h[e];
    for (int i = 0; i < d; ++i) {
      const long long k = i * n + e;
      double f = (i == gaxis) ? -inv_fr * (1.0 - mean_rho / r) : 0.0;
      if (fext) f += fext[k];
      out[k] = u[k] + dt * (-ab[k] - gradp[k] / r + f) + hz[k];
    }
  }
}
// out_i = rho a_i
__global__ void k_mul_by(long long n, int d, const double* __restrict__ a, const double* __restrict__ rho,
                         double* __restrict__ out) {
  EW_LOOP(e, n) {
    const double r = rho[e];
    for (int i = 0; i < d; ++i) out[i * n + e] = r * a[i * n + e];
  }
}
// out_i = a_i / rho
__global__ void k_div_by(long long n, int d, const double* __restrict__ a, const double* __restrict__ rho,
                         double* __restrict__ out) {
  EW_LOOP(e, n) {
    const double r = rho[e];
    for (int i = 0; i < d; ++i) out[i * n + e] = a[i * n + e] / r;
  }
}
// u = u* - dt gphi / rho_h
__global__ void k_project(long long n, int d, const double* __restrict__ us, const double* __restrict__ gphi,
                          const double* __restrict__ rho_h, double dt, double* __restrict__ out) {
  EW_LOOP(e, n) {
    const double r = rho_h[e];
    for (int i = 0; i < d; ++i) out[i * n + e] = us[i * n + e] - dt * gphi[i * n + e] / r;
  }
}
// gradient part of d vector fields, in Fourier: c_j <- k~_j (k~ . c) / |k~|^2 (0 where |k~| = 0),
// i.e. grad Lap^+ div c with the discrete D_j = F^-1 diag(i k~_j) F
__global__ void k_grad_part(GridDesc g, int d, cpx<double>* __restrict__ c) {
  EW_LOOP(e, g.ncplx) {
    const long long line = e / g.h0;
    const int kxi = (int)(e - line * g.h0);
    const int kyi = (int)(line % g.n1);
    const int kzi = (int)(line / g.n1);
    double k[3] = {g.kfac[0] * freq_tilde(kxi, g.n0), 0.0, 0.0};
    if (g.ndim >= 2) k[1] = g.kfac[1] * freq_tilde(kyi, g.n1);
    if (g.ndim == 3) k[2] = g.kfac[2] * freq_tilde(kzi, g.n2);
    double k2 = 0.0, dx = 0.0, dy = 0.0;
    for (int j = 0; j < d; ++j) {
      const cpx<double> v = c[(long long)j * g.ncplx + e];
      k2 += k[j] * k[j];
      dx += k[j] * v.x;
      dy += k[j] * v.y;
    }
    const double s = (k2 == 0.0) ? 0.0 : 1.0 / k2;
    for (int j = 0; j < d; ++j) c[(long long)j * g.ncplx + e] = mk<double>(k[j] * s * dx, k[j] * s * dy);
  }
}
// gradp += gphi - gq  (gq: gradient of the scalar-form correction)
__global__ void k_gradp(long long n, int d, const double* __restrict__ gphi, const double* __restrict__ gq,
                        double* __restrict__ gradp) {
  EW_LOOP(e, n) {
    for (int i = 0; i < d; ++i) gradp[i * n + e] += gphi[i * n + e] - gq[i * n + e];
  }
}
// per-block sums (fixed grid: deterministic order)
__global__ void k_blocksum(long long n, const double* __restrict__ a, double* __restrict__ part) {
  __shared__ double sm[256];
  double s = 0.0;
  EW_LOOP(e, n) { s += a[e]; }
  sm[threadIdx.x] = s;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if (threadIdx.x < k) sm[threadIdx.x] += sm[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sm[0];
}

static int ewb(long long n) { return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 4096)); }

static size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

// physical gradient of a scalar field into d fields (spectral scratch: 2 fields)
static void grad_phys(const vd_grid* G, const double* f, double* out, cpx<double>* s0, cpx<double>* s1,
                      cudaStream_t st) {
  fwd_transform<double>(G, f, s0, st);
  for (int j = 0; j < G->g.ndim; ++j) {
    Mult m;
    m.deriv[j] = 1;
    inv_transform<double>(G, s0, m, out + (size_t)j * G->g.nreal, s1, st);
  }
}

}  // namespace vd

using namespace vd;

static size_t flow_layout(vd_grid* G, const vd_flow_params* p, vd_flow* F, char* base) {
  const int d = G->g.ndim;
  const size_t nr = (size_t)G->g.nreal, fb = nr * sizeof(double);
  size_t off = 0;
  auto take = [&](size_t bytes) -> char* {
    char* q = base ? base + off : nullptr;
    off = a256(off + bytes);
    return q;
  };
  F->rho = (double*)take(fb);
  F->u = (double*)take(d * fb);
  F->gradp = (double*)take(d * fb);
  F->phi = (double*)take(fb);
  F->nrho_prev = (double*)take(fb);
  F->nu_prev = (double*)take(d * fb);
  F->msrc = (double*)take(fb);
  F->force = (double*)take(d * fb);
  F->rho_new = (double*)take(fb);
  F->rho_h = (double*)take(fb);
  F->grad = (double*)take(d * fb);
  F->nrho = (double*)take(fb);
  F->nu = (double*)take(d * fb);
  F->rhs = (double*)take(d * fb);
  F->hz = (double*)take(d * fb);
  F->ustar = (double*)take(d * fb);
  F->fphi = (double*)take(fb);
  F->w = (double*)take(d * fb);
  F->sum = (double*)take(4096 * sizeof(double));
  F->spec_bytes = a256((size_t)G->g.ncplx * 16 * 3);
  F->spec = take(F->spec_bytes);
  F->dens_bytes = vd_density_bytes(G, VD_OP_VELOCITY);
  F->dens = take(F->dens_bytes);
  vd_solve_params sp{};
  sp.tol = p->tol;
  sp.max_it = p->max_it;
  sp.restart = p->restart;
  sp.precision = p->precision;
  const size_t wv = vd_workspace_bytes(G, VD_OP_VELOCITY, (vd_solver)p->vel_solver, &sp);
  const size_t wp = vd_workspace_bytes(G, VD_OP_PRESSURE, (vd_solver)p->pres_solver, &sp);
  F->ws_bytes = std::max(wv, wp);
  F->ws = take(F->ws_bytes);
  return off;
}

static vd_status check_params(const vd_grid* G, const vd_flow_params* p) {
  if (!G || !p) return fail(VD_ERR_INVALID_ARG, "null argument");
  if (!(p->Re > 0) || !(p->Sc > 0) || !(p->Fr > 0)) return fail(VD_ERR_INVALID_ARG, "Re, Sc, Fr must be positive");
  if (p->gravity_axis < -1 || p->gravity_axis >= G->g.ndim) return fail(VD_ERR_INVALID_ARG, "bad gravity axis");
  if (p->vel_solver == VD_SOLVER_CG) return fail(VD_ERR_INVALID_ARG, "the velocity system is not symmetric: no CG");
  if (p->vel_solver < 0 || p->vel_solver > 2 || p->pres_solver < 0 || p->pres_solver > 2)
    return fail(VD_ERR_INVALID_ARG, "unknown solver");
  if (!(p->tol > 0) || p->max_it <= 0) return fail(VD_ERR_INVALID_ARG, "tol > 0 and max_it > 0 required");
  return VD_OK;
}

extern "C" {

size_t vd_flow_bytes(vd_grid* G, const vd_flow_params* p) {
  if (check_params(G, p) != VD_OK) return 0;
  vd_flow F;
  return flow_layout(G, p, &F, nullptr);
}

vd_status vd_flow_create(vd_grid* G, const vd_flow_params* p, void* mem, size_t bytes, vd_flow** out) {
  vd_status e = check_params(G, p);
  if (e != VD_OK) return e;
  if (!mem || !out) return fail(VD_ERR_INVALID_ARG, "null argument");
  vd_flow* F = new vd_flow();
  F->G = G;
  F->p = *p;
  F->d = G->g.ndim;
  F->nr = (size_t)G->g.nreal;
  const size_t need = flow_layout(G, p, F, (char*)mem);
  if (bytes < need) {
    delete F;
    return fail(VD_ERR_OOM, "flow memory smaller than vd_flow_bytes()");
  }
  F->have_prev = 0;
  F->has_msrc = 0;
  F->has_force = 0;
  *out = F;
  return VD_OK;
}

vd_status vd_flow_destroy(vd_flow* F) {
  delete F;
  return VD_OK;
}

vd_status vd_flow_set_state(vd_flow* F, const double* rho, const double* u, vd_stream stream) {
  if (!F || !rho || !u) return fail(VD_ERR_INVALID_ARG, "null argument");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t fb = F->nr * sizeof(double);
  VD_CUDA(cudaMemcpyAsync(F->rho, rho, fb, cudaMemcpyDeviceToDevice, st));
  VD_CUDA(cudaMemcpyAsync(F->u, u, F->d * fb, cudaMemcpyDeviceToDevice, st));
  VD_CUDA(cudaMemsetAsync(F->gradp, 0, F->d * fb, st));
  VD_CUDA(cudaMemsetAsync(F->phi, 0, fb, st));
  F->have_prev = 0;
  return VD_OK;
}

vd_status vd_flow_set_sources(vd_flow* F, const double* mass_source, const double* force, vd_stream stream) {
  if (!F) return fail(VD_ERR_INVALID_ARG, "null flow");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t fb = F->nr * sizeof(double);
  if (mass_source) VD_CUDA(cudaMemcpyAsync(F->msrc, mass_source, fb, cudaMemcpyDeviceToDevice, st));
  if (force) VD_CUDA(cudaMemcpyAsync(F->force, force, F->d * fb, cudaMemcpyDeviceToDevice, st));
  F->has_msrc = mass_source ? 1 : 0;
  F->has_force = force ? 1 : 0;
  return VD_OK;
}

vd_status vd_flow_get_state(const vd_flow* F, double* rho, double* u, double* gradp, double* phi, vd_stream stream) {
  if (!F) return fail(VD_ERR_INVALID_ARG, "null flow");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t fb = F->nr * sizeof(double);
  if (rho) VD_CUDA(cudaMemcpyAsync(rho, F->rho, fb, cudaMemcpyDeviceToDevice, st));
  if (u) VD_CUDA(cudaMemcpyAsync(u, F->u, F->d * fb, cudaMemcpyDeviceToDevice, st));
  if (gradp) VD_CUDA(cudaMemcpyAsync(gradp, F->gradp, F->d * fb, cudaMemcpyDeviceToDevice, st));
  if (phi) VD_CUDA(cudaMemcpyAsync(phi, F->phi, fb, cudaMemcpyDeviceToDevice, st));
  return VD_OK;
}

// snapshot layout: header, then rho (1), u (d), grad p (d), phi (1), nrho_prev (1), nu_prev (d)
struct SnapHeader {
  char magic[8];
  int version, ndim, n[3], have_prev;
  long long nreal;
};
static const char kSnapMagic[8] = {'v', 'd', 'f', 'l', 'o', 'w', 's', '1'};

static size_t snap_fields(const vd_flow* F) { return (size_t)(3 * F->d + 3); }

size_t vd_flow_snapshot_bytes(const vd_flow* F) {
  if (!F) return 0;
  return sizeof(SnapHeader) + snap_fields(F) * F->nr * sizeof(double);
}

vd_status vd_flow_save(const vd_flow* F, void* host, size_t bytes, vd_stream stream) {
  if (!F || !host) return fail(VD_ERR_INVALID_ARG, "null argument");
  if (bytes < vd_flow_snapshot_bytes(F)) return fail(VD_ERR_OOM, "buffer smaller than vd_flow_snapshot_bytes()");
  cudaStream_t st = (cudaStream_t)stream;
  SnapHeader h{};
  std::memcpy(h.magic, kSnapMagic, 8);
  h.version = 1;
  h.ndim = F->d;
  h.n[0] = F->G->g.n0;
  h.n[1] = F->G->g.n1;
  h.n[2] = F->G->g.n2;
  h.have_prev = F->have_prev;
  h.nreal = (long long)F->nr;
  char* o = static_cast<char*>(host);
  std::memcpy(o, &h, sizeof h);
  o += sizeof h;
  const size_t fb = F->nr * sizeof(double);
  const double* src[6] = {F->rho, F->u, F->gradp, F->phi, F->nrho_prev, F->nu_prev};
  const size_t cnt[6] = {1, (size_t)F->d, (size_t)F->d, 1, 1, (size_t)F->d};
  for (int k = 0; k < 6; ++k) {
    VD_CUDA(cudaMemcpyAsync(o, src[k], cnt[k] * fb, cudaMemcpyDeviceToHost, st));
    o += cnt[k] * fb;
  }
  VD_CUDA(cudaStreamSynchronize(st));
  return VD_OK;
}

vd_status vd_flow_load(vd_flow* F, const void* host, size_t bytes, vd_stream stream) {
  if (!F || !host) return fail(VD_ERR_INVALID_ARG, "null argument");
  if (bytes < sizeof(SnapHeader)) return fail(VD_ERR_INVALID_ARG, "snapshot too short");
  SnapHeader h;
  std::memcpy(&h, host, sizeof h);
  if (std::memcmp(h.magic, kSnapMagic, 8) != 0 || h.version != 1) return fail(VD_ERR_INVALID_ARG, "not a snapshot");
  if (h.ndim != F->d || h.n[0] != F->G->g.n0 || h.n[1] != F->G->g.n1 || h.n[2] != F->G->g.n2 ||
      h.nreal != (long long)F->nr)
    return fail(VD_ERR_INVALID_ARG, "snapshot of another grid");
  if (bytes < vd_flow_snapshot_bytes(F)) return fail(VD_ERR_INVALID_ARG, "snapshot too short");
  cudaStream_t st = (cudaStream_t)stream;
  const char* o = static_cast<const char*>(host) + sizeof h;
  const size_t fb = F->nr * sizeof(double);
  double* dst[6] = {F->rho, F->u, F->gradp, F->phi, F->nrho_prev, F->nu_prev};
  const size_t cnt[6] = {1, (size_t)F->d, (size_t)F->d, 1, 1, (size_t)F->d};
  for (int k = 0; k < 6; ++k) {
    VD_CUDA(cudaMemcpyAsync(dst[k], o, cnt[k] * fb, cudaMemcpyHostToDevice, st));
    o += cnt[k] * fb;
  }
  VD_CUDA(cudaStreamSynchronize(st));
  F->have_prev = h.have_prev;
  return VD_OK;
}

vd_status vd_flow_step(vd_flow* F, double dt, vd_step_info* info, vd_stream stream) {
  if (!F || !(dt > 0)) return fail(VD_ERR_INVALID_ARG, "null flow or dt <= 0");
  vd_grid* G = F->G;
  const GridDesc& g = G->g;
  cudaStream_t st = (cudaStream_t)stream;
  const int d = F->d;
  const long long n = (long long)F->nr;
  const vd_flow_params& p = F->p;
  cpx<double>* s0 = (cpx<double>*)F->spec;
  cpx<double>* s1 = s0 + g.ncplx;
  cpx<double>* s2 = s1 + g.ncplx;
  const int b = ewb(n);
  vd_status e;

  // 1. mass equation
  grad_phys(G, F->rho, F->grad, s0, s1, st);
  { k_dotvec<<<b, 256, 0, st>>>(n, d, F->u, F->grad, F->nrho); count_launch(); }
  const double* ab = F->nrho;
  if (F->have_prev) {
    { k_lin<<<b, 256, 0, st>>>(n, 1.5, F->nrho, -0.5, F->nrho_prev, F->rhs); count_launch(); }
    ab = F->rhs;
  }
  if (F->has_msrc) {   // [u.grad rho]^{n+1/2} - S^{n+1/2}
    { k_lin<<<b, 256, 0, st>>>(n, 1.0, ab, -1.0, F->msrc, F->fphi); count_launch(); }
    ab = F->fphi;
  }
  fwd_transform<double>(G, F->rho, s0, st);
  fwd_transform<double>(G, ab, s1, st);
  const double c = dt / (2.0 * p.Re * p.Sc);
  { k_mass<<<ewb(g.ncplx), 256, 0, st>>>(g, c, dt, s0, s1, s2); count_launch(); }
  {
    Mult m;
    inv_transform<double>(G, s2, m, F->rho_new, s0, st);
  }
  // 2. mid-step density, attached to the grid with the viscous-operator data
  { k_lin<<<b, 256, 0, st>>>(n, 0.5, F->rho_new, 0.5, F->rho, F->rho_h); count_launch(); }
  e = vd_density_set(G, VD_OP_VELOCITY, F->rho_h, F->dens, F->dens_bytes, stream);
  if (e != VD_OK) return e;
  // 3. predictor
  const double a = dt / (2.0 * p.Re);
  const vd_op_params opp{a, 1.0 / p.Sc};
  for (int i = 0; i < d; ++i) {
    grad_phys(G, F->u + i * n, F->grad, s0, s1, st);
    { k_dotvec<<<b, 256, 0, st>>>(n, d, F->u, F->grad, F->nu + i * n); count_launch(); }
  }
  const double* abu = F->nu;
  if (F->have_prev) {
    { k_lin<<<b, 256, 0, st>>>(n * d, 1.5, F->nu, -0.5, F->nu_prev, F->w); count_launch(); }
    abu = F->w;
  }
  // hz = u - V u  ( = (dt/2) zeta(rho_h, u) )
  e = vd_apply_op(G, VD_OP_VELOCITY, &opp, F->u, F->hz, F->ws, F->ws_bytes, stream);
  if (e != VD_OK) return e;
  { k_lin<<<ewb(n * d), 256, 0, st>>>(n * d, 1.0, F->u, -1.0, F->hz, F->hz); count_launch(); }
  double mean_rho = 0.0;
  if (p.gravity_axis >= 0) {
    const int nb = std::min(b, 4096);
    { k_blocksum<<<nb, 256, 0, st>>>(n, F->rho_h, F->sum); count_launch(); }
    std::vector<double> part(nb);
    VD_CUDA(cudaMemcpyAsync(part.data(), F->sum, nb * sizeof(double), cudaMemcpyDeviceToHost, st));
    VD_CUDA(cudaStreamSynchronize(st));
    double s = 0.0;
    for (double v : part) s += v;
    mean_rho = s / (double)n;
  }
  { k_rhs<<<b, 256, 0, st>>>(n, d, F->u, abu, F->gradp, F->rho_h, F->hz, dt, p.gravity_axis, 1.0 / p.Fr, mean_rho,
                             F->has_force ? F->force : nullptr, F->rhs); count_launch(); }
  VD_CUDA(cudaMemcpyAsync(F->ustar, F->u, d * n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  vd_solve_params sp{};
  sp.tol = p.tol;
  sp.max_it = p.max_it;
  sp.restart = p.restart;
  sp.use_x0 = 1;
  sp.precision = p.precision;
  sp.inner_tol = 0.0;   // automatic
  sp.check_every = 1;
  vd_solve_info iv{};
  vd_status sv = vd_solve(G, VD_OP_VELOCITY, (vd_solver)p.vel_solver, &opp, &sp, F->rhs, F->ustar, &iv, F->ws,
                          F->ws_bytes, stream);
  if (sv == VD_ERR_INVALID_ARG || sv == VD_ERR_OOM || sv == VD_ERR_CUDA || sv == VD_ERR_NO_DENSITY) return sv;
  // 4. pressure increment
  e = vd_divergence(G, F->ustar, F->fphi, F->spec, F->spec_bytes, stream);
  if (e != VD_OK) return e;
  { k_lin<<<b, 256, 0, st>>>(n, 1.0 / dt, F->fphi, 0.0, nullptr, F->fphi); count_launch(); }
  vd_solve_info ip{};
  vd_status spr = vd_solve(G, VD_OP_PRESSURE, (vd_solver)p.pres_solver, nullptr, &sp, F->fphi, F->phi, &ip, F->ws,
                           F->ws_bytes, stream);
  if (spr == VD_ERR_INVALID_ARG || spr == VD_ERR_OOM || spr == VD_ERR_CUDA || spr == VD_ERR_NO_DENSITY) return spr;
  // 5. projection
  e = vd_gradient(G, F->phi, F->grad, F->spec, F->spec_bytes, stream);
  if (e != VD_OK) return e;
  // 6. pressure update, scalar form: w = gphi/rho_h, hz = w - V w, c = rho_h hz, and
  //    grad p += gphi - grad Lap^+ div c, the gradient part of c taken in Fourier
  //    (d forward and d inverse transforms; the solve workspace is free here: scratch)
  { k_div_by<<<b, 256, 0, st>>>(n, d, F->grad, F->rho_h, F->w); count_launch(); }
  e = vd_apply_op(G, VD_OP_VELOCITY, &opp, F->w, F->hz, F->ws, F->ws_bytes, stream);
  if (e != VD_OK) return e;
  { k_lin<<<ewb(n * d), 256, 0, st>>>(n * d, 1.0, F->w, -1.0, F->hz, F->hz); count_launch(); }
  { k_mul_by<<<b, 256, 0, st>>>(n, d, F->hz, F->rho_h, F->hz); count_launch(); }
  for (int j = 0; j < d; ++j) fwd_transform<double>(G, F->hz + (size_t)j * n, s0 + (size_t)j * g.ncplx, st);
  { k_grad_part<<<ewb(g.ncplx), 256, 0, st>>>(g, d, s0); count_launch(); }
  for (int j = 0; j < d; ++j) {
    Mult m;
    inv_transform<double>(G, s0 + (size_t)j * g.ncplx, m, F->w + (size_t)j * n, reinterpret_cast<cpx<double>*>(F->ws),
                          st);
  }
  { k_gradp<<<b, 256, 0, st>>>(n, d, F->grad, F->w, F->gradp); count_launch(); }
  { k_project<<<b, 256, 0, st>>>(n, d, F->ustar, F->grad, F->rho_h, dt, F->u); count_launch(); }
  // history and new density
  VD_CUDA(cudaMemcpyAsync(F->nrho_prev, F->nrho, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  VD_CUDA(cudaMemcpyAsync(F->nu_prev, F->nu, d * n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  VD_CUDA(cudaMemcpyAsync(F->rho, F->rho_new, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  F->have_prev = 1;
  VD_CUDA(cudaGetLastError());
  if (info) {
    info->vel_iters = iv.iters;
    info->vel_status = iv.status;
    info->vel_relres = iv.relres_true;
    info->pres_iters = ip.iters;
    info->pres_status = ip.status;
    info->pres_relres = ip.relres_true;
  }
  return (sv != VD_OK) ? sv : spr;
}

}  // extern "C"
