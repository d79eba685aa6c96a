// C ABI of the library: grids, density data, operator/preconditioner application and
// the preconditioned solves (double and mixed precision).
#include "vd_krylov.cuh"
#include "vd_dd.cuh"
#include "vd_internal.h"
#include "vd_prof.h"

#include <algorithm>
#include <cmath>
#include <limits>
#include <cstdio>
#include <cstring>
#include <string>

namespace vd {

static thread_local std::string g_err = "no error";

vd_status fail(vd_status st, const std::string& msg) {
  g_err = msg;
  return st;
}
vd_status cuda_fail(cudaError_t e, const char* what) {
  g_err = std::string("CUDA error in ") + what + ": " + cudaGetErrorString(e);
  return (e == cudaErrorMemoryAllocation) ? VD_ERR_OOM : VD_ERR_CUDA;
}

// ---------------------------------------------------------------------------------------
// plans and twiddles
// ---------------------------------------------------------------------------------------

static bool make_plan(int n, FftPlan* p) {
  if (n < 2 || n > 4096) return false;
  int a = 0, b = 0, c = 0, r = n;
  while (r % 2 == 0) { r /= 2; ++a; }
  while (r % 3 == 0) { r /= 3; ++b; }
  while (r % 5 == 0) { r /= 5; ++c; }
  if (r != 1) return false;
  p->n = n;
  p->nst = 0;
  auto push = [&](int R) { p->rad[p->nst++] = R; };
  while (a >= 3) { push(8); a -= 3; }
  if (a == 2) push(4);
  if (a == 1) push(2);
  while (b-- > 0) push(3);
  while (c-- > 0) push(5);
  return p->nst <= kMaxStages;
}

// exp(-2 pi i j / n) evaluated in extended precision
static void twiddle_ld(long long j, long long n, long double* re, long double* im) {
  j %= n;
  const long double th = 2.0L * 3.14159265358979323846264338327950288L * (long double)j / (long double)n;
  *re = cosl(th);
  *im = -sinl(th);
}
static void twiddle(long long j, long long n, double* re, double* im) {
  long double r, i;
  twiddle_ld(j, n, &r, &i);
  *re = (double)r;
  *im = (double)i;
}
// float-pair split of an extended-precision value
static void split_ld(long double v, float* hi, float* lo) {
  *hi = (float)v;
  *lo = (float)(v - (long double)*hi);
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Carver {
  char* base;
  size_t off = 0;
  size_t cap;
  template <typename P>
  P* take(size_t bytes) {
    P* p = reinterpret_cast<P*>(base ? base + off : nullptr);
    off = align256(off + bytes);
    return p;
  }
  bool ok() const { return off <= cap; }
};

}  // namespace vd

using namespace vd;

extern "C" {
const char* vd_last_error(void) { return g_err.c_str(); }
const char* vd_version(void) { return "vdspectral 0.1 (sm_103a)"; }
}  // extern "C"

namespace vd {
// Fill the grid description (plans, sizes) without touching the device; false on bad sizes.
bool grid_desc_only(int ndim, const int n[3], const double L[3], vd_grid* G) {
  if (ndim < 1 || ndim > 3) return false;
  int nn[3] = {1, 1, 1};
  for (int j = 0; j < ndim; ++j) {
    if (n[j] < 4 || n[j] > 1024 || (n[j] % 2) != 0 || !(L[j] > 0.0)) return false;
    nn[j] = n[j];
  }
  GridDesc& g = G->g;
  g.ndim = ndim;
  g.n0 = nn[0];
  g.n1 = nn[1];
  g.n2 = nn[2];
  g.h0 = nn[0] / 2 + 1;
  g.nreal = (long long)nn[0] * nn[1] * nn[2];
  g.ncplx = (long long)g.h0 * nn[1] * nn[2];
  for (int j = 0; j < 3; ++j) G->L[j] = (j < ndim) ? L[j] : 1.0;
  bool ok = make_plan(nn[0] / 2, &g.px);
  if (ndim >= 2) ok = ok && make_plan(nn[1], &g.py);
  if (ndim == 3) ok = ok && make_plan(nn[2], &g.pz);
  return ok && g.ncplx * 3 < (1ll << 31);
}
}  // namespace vd

extern "C" {

vd_status vd_grid_create(int ndim, const int n[3], const double L[3], vd_grid** out) {
  if (!out || !n || !L) return fail(VD_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  if (ndim < 1 || ndim > 3) return fail(VD_ERR_INVALID_ARG, "ndim must be 1, 2 or 3");
  int nn[3] = {1, 1, 1};
  for (int j = 0; j < ndim; ++j) {
    nn[j] = n[j];
    if (n[j] < 4 || n[j] > 1024 || (n[j] % 2) != 0)
      return fail(VD_ERR_INVALID_ARG, "axis lengths must be even and in [4, 1024]");
    if (!(L[j] > 0.0) || !std::isfinite(L[j])) return fail(VD_ERR_INVALID_ARG, "box lengths must be positive");
  }
  vd_grid* G = new vd_grid();
  GridDesc& g = G->g;
  g.ndim = ndim;
  g.n0 = nn[0];
  g.n1 = nn[1];
  g.n2 = nn[2];
  g.h0 = nn[0] / 2 + 1;
  g.nreal = (long long)nn[0] * nn[1] * nn[2];
  g.ncplx = (long long)g.h0 * nn[1] * nn[2];
  if (g.ncplx * 3 >= (1ll << 31)) {
    delete G;
    return fail(VD_ERR_INVALID_ARG, "grid too large: field offsets must fit in 32 bits");
  }
  for (int j = 0; j < 3; ++j) {
    G->L[j] = (j < ndim) ? L[j] : 1.0;
    g.kfac[j] = 2.0 * 3.14159265358979323846 / G->L[j];
    const long double kl = 2.0L * 3.14159265358979323846264338327950288L / (long double)G->L[j];
    split_ld(kl, &g.kfac_dd[j][0], &g.kfac_dd[j][1]);
    g.kfac_f[j] = (float)g.kfac[j];
  }
  bool ok = make_plan(nn[0] / 2, &g.px);
  if (ndim >= 2) ok = ok && make_plan(nn[1], &g.py);
  else g.py = g.px;
  if (ndim == 3) ok = ok && make_plan(nn[2], &g.pz);
  else g.pz = g.py;
  if (!ok) {
    delete G;
    return fail(VD_ERR_INVALID_ARG, "axis lengths must factor into 2, 3 and 5");
  }
  // twiddle tables: px (m), py (n1), pz (n2), packing (m + 1)
  std::vector<double> tw;
  auto add = [&](FftPlan& p) {
    p.tw_off = (int)(tw.size() / 2);
    for (int j = 0; j < p.n; ++j) {
      double re, im;
      twiddle(j, p.n, &re, &im);
      tw.push_back(re);
      tw.push_back(im);
    }
  };
  add(g.px);
  if (ndim >= 2) add(g.py);
  else g.py.tw_off = g.px.tw_off;
  if (ndim == 3) add(g.pz);
  else g.pz.tw_off = g.py.tw_off;
  g.pk_off = (int)(tw.size() / 2);
  for (int k = 0; k <= nn[0] / 2; ++k) {
    double re, im;
    twiddle(k, nn[0], &re, &im);
    tw.push_back(re);
    tw.push_back(im);
  }
  std::vector<float> twf(tw.size());
  for (size_t i = 0; i < tw.size(); ++i) twf[i] = (float)tw[i];
  // float-pair table, split from the extended-precision values (same index layout)
  std::vector<float> twdd(2 * tw.size());
  {
    auto put = [&](size_t at, int j, int len) {
      long double re, im;
      twiddle_ld(j, len, &re, &im);
      split_ld(re, &twdd[4 * at + 0], &twdd[4 * at + 1]);
      split_ld(im, &twdd[4 * at + 2], &twdd[4 * at + 3]);
    };
    for (int j = 0; j < g.px.n; ++j) put(g.px.tw_off + j, j, g.px.n);
    if (ndim >= 2)
      for (int j = 0; j < g.py.n; ++j) put(g.py.tw_off + j, j, g.py.n);
    if (ndim == 3)
      for (int j = 0; j < g.pz.n; ++j) put(g.pz.tw_off + j, j, g.pz.n);
    for (int k = 0; k <= nn[0] / 2; ++k) put(g.pk_off + k, k, nn[0]);
  }
  // The tables are uploaded on a private stream that is synchronised before returning.  A plain
  // cudaMemcpy from pageable memory may return while its DMA is still in flight, and kernels
  // that a caller then launches on a non-blocking stream (server slots, torch side streams) are
  // not ordered behind the legacy stream: they could read a partly written table.
  cudaStream_t up = nullptr;
  cudaError_t e = cudaMalloc(&G->tw_d, tw.size() * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&G->tw_f, twf.size() * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&G->tw_dd, twdd.size() * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&G->g.dev_err, 256);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&up, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMemsetAsync(G->g.dev_err, 0, 256, up);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(G->tw_d, tw.data(), tw.size() * sizeof(double), cudaMemcpyHostToDevice, up);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(G->tw_f, twf.data(), twf.size() * sizeof(float), cudaMemcpyHostToDevice, up);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(G->tw_dd, twdd.data(), twdd.size() * sizeof(float), cudaMemcpyHostToDevice, up);
  if (up) {
    const cudaError_t es = cudaStreamSynchronize(up);
    if (e == cudaSuccess) e = es;
    cudaStreamDestroy(up);
  }
  if (e != cudaSuccess) {
    if (G->tw_d) cudaFree(G->tw_d);
    if (G->tw_f) cudaFree(G->tw_f);
    if (G->tw_dd) cudaFree(G->tw_dd);
    if (G->g.dev_err) cudaFree(G->g.dev_err);
    delete G;
    return cuda_fail(e, "vd_grid_create");
  }
  *out = G;
  return VD_OK;
}

vd_status vd_grid_destroy(vd_grid* G) {
  if (!G) return VD_OK;
  if (G->tw_d) cudaFree(G->tw_d);
  if (G->tw_f) cudaFree(G->tw_f);
  if (G->tw_dd) cudaFree(G->tw_dd);
  if (G->g.dev_err) cudaFree(G->g.dev_err);
  delete G;
  return VD_OK;
}

size_t vd_grid_points(const vd_grid* G) { return G ? (size_t)G->g.nreal : 0; }
size_t vd_grid_modes(const vd_grid* G) { return G ? (size_t)G->g.ncplx : 0; }

}  // extern "C"

// ---------------------------------------------------------------------------------------
// density
// ---------------------------------------------------------------------------------------

namespace vd {

__global__ void k_density_prep(long long n, const double* __restrict__ rho, double* __restrict__ rcopy,
                               double* __restrict__ rinv_s, float* __restrict__ rinv_f, dd* __restrict__ rinv_dd,
                               double invN,
                               double* __restrict__ stats /* [min, max, bad] via block partials */) {
  __shared__ double smin[256], smax[256], sbad[256];
  double mn = 1e308, mx = -1e308, bd = 0.0;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const double r = rho[e];
    rcopy[e] = r;
    const double ri = invN / r;
    rinv_s[e] = ri;
    rinv_f[e] = (float)ri;
    rinv_dd[e] = dd_from_double(ri);
    if (!(r > 0.0) || !isfinite(r)) bd = 1.0;
    mn = fmin(mn, r);
    mx = fmax(mx, r);
  }
  smin[threadIdx.x] = mn;
  smax[threadIdx.x] = mx;
  sbad[threadIdx.x] = bd;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      smin[threadIdx.x] = fmin(smin[threadIdx.x], smin[threadIdx.x + s]);
      smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + s]);
      sbad[threadIdx.x] = fmax(sbad[threadIdx.x], sbad[threadIdx.x + s]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    stats[3 * blockIdx.x + 0] = smin[0];
    stats[3 * blockIdx.x + 1] = smax[0];
    stats[3 * blockIdx.x + 2] = sbad[0];
  }
}

struct DensLayout {
  double* rho;
  double* rinv_s;
  float* rinv_f;
  dd* rinv_dd;
  double* stats;
  double* grho;     // d fields
  double* hrho;     // 6 fields, slot hidx(i, j)
  cpx<double>* s0;  // scratch spectral fields (2)
  // K_rho data
  double* kw;       // w = rho^-1/2
  double* kc_s;     // c/N
  float* kc_f;
  dd* kc_dd;
  cpx<double>* kw_hat;   // spectrum of w, unit Parseval norm
};

static DensLayout dens_layout(const vd_grid* G, vd_op op, void* base, size_t* bytes) {
  const GridDesc& g = G->g;
  Carver c{(char*)base, 0, (size_t)-1};
  DensLayout L;
  const size_t nr = (size_t)g.nreal, nc = (size_t)g.ncplx;
  L.rho = c.take<double>(nr * 8);
  L.rinv_s = c.take<double>(nr * 8);
  L.rinv_f = c.take<float>(nr * 4);
  L.rinv_dd = c.take<dd>(nr * sizeof(dd));
  L.stats = c.take<double>(3 * 1024 * 8);
  L.grho = L.hrho = nullptr;
  L.s0 = nullptr;
  L.kw = L.kc_s = nullptr;
  L.kc_f = nullptr;
  L.kc_dd = nullptr;
  L.kw_hat = nullptr;
  if (op == VD_OP_VELOCITY) {
    L.grho = c.take<double>(nr * 8 * g.ndim);
    L.hrho = c.take<double>(nr * 8 * 6);   // indexed by hidx(i, j) in [0, 6)
    L.s0 = c.take<cpx<double>>(nc * 16 * 4);   // spectrum of rho + 3 derivative scratch fields
  }
  if (op == VD_OP_KRHO) {
    L.kw = c.take<double>(nr * 8);
    L.kc_s = c.take<double>(nr * 8);
    L.kc_f = c.take<float>(nr * 4);
    L.kc_dd = c.take<dd>(nr * sizeof(dd));
    L.kw_hat = c.take<cpx<double>>(nc * 16);
    L.s0 = c.take<cpx<double>>(nc * 16 * 2);   // symbol + transform scratch of the preparation
  }
  *bytes = c.off;
  return L;
}

// w = rho^-1/2 and per-block partial sums of w^2 (fixed grid: deterministic)
__global__ void k_krho_w(long long n, const double* __restrict__ rho, double* __restrict__ w,
                         double* __restrict__ part) {
  __shared__ double sm[256];
  double s = 0.0;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const double v = 1.0 / sqrt(rho[e]);
    w[e] = v;
    s += v * v;
  }
  sm[threadIdx.x] = s;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if (threadIdx.x < k) sm[threadIdx.x] += sm[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sm[0];
}

// c = -Lap(w)/w; stored as c/N in double, float and float-pair (lapw may alias cs)
__global__ void k_krho_coef(long long n, const double* __restrict__ w, const double* lapw, double invN, double* cs,
                            float* __restrict__ cf, dd* __restrict__ cdd) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const double c = -lapw[e] / w[e] * invN;
    cs[e] = c;
    cf[e] = (float)c;
    cdd[e] = dd_from_double(c);
  }
}

}  // namespace vd

extern "C" {

size_t vd_density_bytes(const vd_grid* G, vd_op op) {
  if (!G) return 0;
  size_t b = 0;
  dens_layout(G, op, nullptr, &b);
  return b;
}

vd_status vd_density_set(vd_grid* G, vd_op op, const double* rho, void* ws, size_t ws_bytes, vd_stream stream) {
  if (!G || !rho || !ws) return fail(VD_ERR_INVALID_ARG, "null argument");
  if (op != VD_OP_PRESSURE && op != VD_OP_VELOCITY && op != VD_OP_KRHO)
    return fail(VD_ERR_INVALID_ARG, "unknown operator");
  cudaStream_t st = (cudaStream_t)stream;
  size_t need = 0;
  DensLayout L = dens_layout(G, op, ws, &need);
  if (ws_bytes < need) return fail(VD_ERR_OOM, "density workspace too small");
  const GridDesc& g = G->g;
  const int blocks = (int)std::min<long long>(1024, (g.nreal + 255) / 256);
  { k_density_prep<<<blocks, 256, 0, st>>>(g.nreal, rho, L.rho, L.rinv_s, L.rinv_f, L.rinv_dd, 1.0 / (double)g.nreal,
                                        L.stats); count_launch(); }
  VD_CUDA(cudaGetLastError());
  std::vector<double> stats(3 * blocks);
  VD_CUDA(cudaMemcpyAsync(stats.data(), L.stats, stats.size() * 8, cudaMemcpyDeviceToHost, st));
  VD_CUDA(cudaStreamSynchronize(st));
  double mn = 1e308, mx = -1e308, bd = 0;
  for (int b = 0; b < blocks; ++b) {
    mn = std::min(mn, stats[3 * b]);
    mx = std::max(mx, stats[3 * b + 1]);
    bd = std::max(bd, stats[3 * b + 2]);
  }
  if (bd != 0.0) {
    G->has_density = 0;
    return fail(VD_ERR_INVALID_ARG, "density must be positive and finite");
  }
  G->rho = L.rho;
  G->rinv_s = L.rinv_s;
  G->rinv_s_f = L.rinv_f;
  G->rinv_s_dd = L.rinv_dd;
  G->rho_min = mn;
  G->rho_max = mx;
  G->has_density = 1;
  G->has_velocity_data = 0;
  for (int j = 0; j < 3; ++j) G->grho[j] = nullptr;
  for (int j = 0; j < 6; ++j) G->hrho[j] = nullptr;
  if (op == VD_OP_VELOCITY) {
    const int d = g.ndim;
    const size_t nr = (size_t)g.nreal, nc = (size_t)g.ncplx;
    cpx<double>* rh = L.s0;
    cpx<double>* tmp = L.s0 + nc;
    fwd_transform<double>(G, L.rho, rh, st);
    double* grad[3] = {nullptr, nullptr, nullptr};
    double* hess[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    for (int j = 0; j < d; ++j) {
      grad[j] = L.grho + j * nr;
      G->grho[j] = grad[j];
    }
    for (int i = 0; i < d; ++i)
      for (int j = i; j < d; ++j) {
        hess[hidx(i, j)] = L.hrho + hidx(i, j) * nr;
        G->hrho[hidx(i, j)] = hess[hidx(i, j)];
      }
    derivative_fields(G, rh, grad, hess, tmp, st);
    VD_CUDA(cudaGetLastError());
    G->has_velocity_data = 1;
  }
  G->has_krho_data = 0;
  G->kc_s = nullptr;
  G->kc_f = nullptr;
  G->kc_dd = nullptr;
  G->kw_hat = nullptr;
  if (op == VD_OP_KRHO) {
    const size_t nc = (size_t)g.ncplx;
    { k_krho_w<<<blocks, 256, 0, st>>>(g.nreal, rho, L.kw, L.stats); count_launch(); }
    std::vector<double> part(blocks);
    VD_CUDA(cudaMemcpyAsync(part.data(), L.stats, part.size() * 8, cudaMemcpyDeviceToHost, st));
    VD_CUDA(cudaStreamSynchronize(st));
    double ww = 0.0;
    for (int b = 0; b < blocks; ++b) ww += part[b];
    // Lap w with the full-wavenumber symbol, then c = -Lap(w)/w
    cpx<double>* sym = L.s0;
    cpx<double>* tmp = L.s0 + nc;
    fwd_transform<double>(G, L.kw, L.kw_hat, st);
    fill_symbol<double>(G, SYM_KLAP, 0.0, reinterpret_cast<double*>(sym), st);
    Mult m;
    m.sym = 1;
    m.symarr = sym;
    inv_transform<double>(G, L.kw_hat, m, L.kc_s, tmp, st);
    { k_krho_coef<<<blocks, 256, 0, st>>>(g.nreal, L.kw, L.kc_s, 1.0 / (double)g.nreal, L.kc_s, L.kc_f, L.kc_dd);
      count_launch(); }
    // unit Parseval norm: sum over the half spectrum with weights = N sum_x w^2
    spec_copy_scale<double>((long long)nc, L.kw_hat, 1.0 / std::sqrt((double)g.nreal * ww), L.kw_hat, st);
    VD_CUDA(cudaGetLastError());
    G->kc_s = L.kc_s;
    G->kc_f = L.kc_f;
    G->kc_dd = L.kc_dd;
    G->kw_hat = L.kw_hat;
    G->has_krho_data = 1;
  }
  return VD_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------
// workspace layout of apply / solve
// ---------------------------------------------------------------------------------------

namespace vd {

struct SolveLayout {
  KState* ks;
  OState* ost;           // refinement state of graph solves
  double* removed;       // null-space shares removed from b by the range projection (2^d)
  double* partials;
  unsigned* counter;
  double* hist;
  double* sym;           // ncplx
  float* sym_f;          // ncplx (mixed)
  cpx<double>* bh;       // len
  cpx<double>* xh;       // len
  cpx<double>* rh;       // len (true residual / refinement)
  void* vecs;            // Krylov vectors (double, or float for mixed)
  cpx<double>* tmp;      // operator temporaries (double)
  cpx<float>* tmp_f;     // operator temporaries (float, mixed)
  cpx<float>* bh_f;      // inner rhs (mixed)
  cpx<float>* xh_f;      // inner solution (mixed)
};

static int op_ncomp(const vd_grid* G, vd_op op) { return op == VD_OP_VELOCITY ? G->g.ndim : 1; }
static int op_tmp_fields(const vd_grid* G, vd_op op) {
  if (op == VD_OP_VELOCITY) return velocity_tmp_fields(G->g.ndim);
  if (op == VD_OP_KRHO) return krho_tmp_fields(G->g.ndim);
  return pressure_tmp_fields(G->g.ndim);
}
static int op_symbol(vd_op op) {
  return op == VD_OP_VELOCITY ? SYM_VELOCITY : (op == VD_OP_KRHO ? SYM_KLAP_INV : SYM_PRESSURE);
}

static SolveLayout solve_layout(const vd_grid* G, vd_op op, int solver, int restart, int maxit, int precision,
                                void* base, size_t* bytes) {
  const size_t nc = (size_t)G->g.ncplx;
  const int ncomp = op_ncomp(G, op);
  const size_t len = nc * ncomp;
  Carver c{(char*)base, 0, (size_t)-1};
  SolveLayout L;
  L.ks = c.take<KState>(sizeof(KState));
  L.partials = c.take<double>(sizeof(double) * kRedBlocks * 8);
  L.counter = c.take<unsigned>(sizeof(unsigned) * 4);
  L.hist = c.take<double>(sizeof(double) * (size_t)(std::max(maxit, 1) + 2));
  L.ost = c.take<OState>(sizeof(OState));
  L.removed = c.take<double>(sizeof(double) * 32);
  L.sym = c.take<double>(nc * 8);
  L.sym_f = nullptr;
  L.bh = c.take<cpx<double>>(len * 16);
  L.xh = c.take<cpx<double>>(len * 16);
  L.rh = c.take<cpx<double>>(len * 16);
  SpecSystem dummy{};
  dummy.len = (long long)len;
  const int tf = std::max(op_tmp_fields(G, op), 1);
  if (precision == VD_PREC_MIXED || precision == VD_PREC_MIXED_DD) {
    L.sym_f = c.take<float>(nc * 4);
    L.vecs = c.take<char>(krylov_vec_bytes<float>(dummy, solver, restart));
    L.bh_f = c.take<cpx<float>>(len * 8);
    L.xh_f = c.take<cpx<float>>(len * 8);
    L.tmp_f = c.take<cpx<float>>(nc * 8 * tf);
    // the double operator (true residual) needs its own temporaries and two vectors
    L.tmp = c.take<cpx<double>>(nc * 16 * tf);
  } else {
    L.vecs = c.take<char>(krylov_vec_bytes<double>(dummy, solver, restart));
    L.tmp = c.take<cpx<double>>(nc * 16 * tf);
    L.tmp_f = nullptr;
    L.bh_f = L.xh_f = nullptr;
  }
  *bytes = c.off;
  return L;
}

// operator callbacks ---------------------------------------------------------------------

template <typename T>
static void apply_cb(const SpecSystem& sys, const void* in, void* out, bool with_sym, const int* done,
                     cudaStream_t st) {
  const vd_grid* G = sys.G;
  const T* sym = with_sym ? (const T*)sys.sym : nullptr;
  if (sys.ctx[1] == (void*)2) {
    apply_krho_spec<T>(G, (const cpx<T>*)in, (cpx<T>*)out, sym, (const T*)sys.ctx[0], (cpx<T>*)sys.ctx[2], done, st,
                       sys.ctx[3]);
  } else if (sys.ncomp == 1 && sys.ctx[1] == nullptr) {
    apply_pressure_spec<T>(G, (const cpx<T>*)in, (cpx<T>*)out, sym, (const T*)sys.ctx[0], (cpx<T>*)sys.ctx[2], done,
                           st, sys.ctx[3]);
  } else {
    apply_velocity_spec<T>(G, (const cpx<T>*)in, (cpx<T>*)out, sym, sys.a, sys.inv_sc, (cpx<T>*)sys.ctx[2], done, st);
  }
}

// Density ratio above which the inner float operator of a mixed solve multiplies by 1/rho (or
// the K_rho coefficient) in float-pair arithmetic: the multiply by a coefficient spanning a
// wide range is kept at double-like accuracy while transforms and vectors stay float.
constexpr double kPairRatio = 10.0;

// Relative tolerance of the inner float solves of the refinement when the caller leaves it to
// the library.  At high density ratios a float CG can stall above it (near kappa times the
// float rounding; a ratio of 28.6 on a 512^2 slab stalled at 1.3e-5): the stall test of the
// guarded inner solves (KState::guard) then ends the sweep and the refinement goes on.
static double auto_inner_tol(const vd_grid*) { return 1e-5; }

static bool coef_in_pairs(const vd_grid* G, vd_op op, int coef_pair) {
  if (op == VD_OP_VELOCITY) return false;   // the velocity bracket multiplies by 1/rho in double
  if (coef_pair != 0) return coef_pair > 0;
  return G->rho_max > kPairRatio * G->rho_min;
}

template <typename T>
static SpecSystem make_system(const vd_grid* G, vd_op op, const vd_op_params* p, const void* sym, void* tmp,
                              int coef_pair = 0) {
  SpecSystem s{};
  s.G = G;
  s.ncomp = op_ncomp(G, op);
  s.len = (long long)G->g.ncplx * s.ncomp;
  s.h0 = G->g.h0;
  s.sym = sym;
  s.is_float = sizeof(T) == 4;
  s.apply = &apply_cb<T>;
  if (op == VD_OP_KRHO) {
    s.ctx[0] = (sizeof(T) == 8) ? (void*)G->kc_s : (void*)G->kc_f;
    s.ctx[1] = (void*)2;
  } else {
    s.ctx[0] = (sizeof(T) == 8) ? (void*)G->rinv_s : (void*)G->rinv_s_f;
    s.ctx[1] = (op == VD_OP_VELOCITY) ? (void*)1 : nullptr;
  }
  s.ctx[2] = tmp;
  s.ctx[3] = nullptr;
  if (sizeof(T) == 4 && coef_in_pairs(G, op, coef_pair))
    s.ctx[3] = (op == VD_OP_KRHO) ? (void*)G->kc_dd : (void*)G->rinv_s_dd;
  s.a = p ? p->a : 0.0;
  s.inv_sc = p ? p->inv_sc : 1.0;
  return s;
}

static vd_status check_op(const vd_grid* G, vd_op op, const vd_op_params* p) {
  if (!G) return fail(VD_ERR_INVALID_ARG, "null grid");
  if (op != VD_OP_PRESSURE && op != VD_OP_VELOCITY && op != VD_OP_KRHO)
    return fail(VD_ERR_INVALID_ARG, "unknown operator");
  if (!G->has_density) return fail(VD_ERR_NO_DENSITY, "vd_density_set has not been called");
  if (op == VD_OP_KRHO && !G->has_krho_data)
    return fail(VD_ERR_NO_DENSITY, "density was not set for the K_rho operator");
  if (op == VD_OP_VELOCITY) {
    if (!p) return fail(VD_ERR_INVALID_ARG, "velocity operator needs vd_op_params");
    if (!G->has_velocity_data) return fail(VD_ERR_NO_DENSITY, "density was set for the pressure operator only");
    if (!(p->a >= 0.0) || !std::isfinite(p->a) || !std::isfinite(p->inv_sc))
      return fail(VD_ERR_INVALID_ARG, "velocity parameters must be finite, a >= 0");
  }
  return VD_OK;
}

// forward transform of every component (physical double -> spectral double), one launch per
// pass for all components
static void fwd_all(const vd_grid* G, int ncomp, const double* in, cpx<double>* out, cudaStream_t st) {
  fwd_transform_n<double>(G, ncomp, in, out, st);
}
// inverse likewise; tmp: ncomp spectral fields (the operator's temporaries hold that many)
static void inv_all(const vd_grid* G, int ncomp, const cpx<double>* in, double* out, cpx<double>* tmp,
                    cudaStream_t st) {
  inv_transform_n<double>(G, ncomp, in, out, tmp, st);
}

// One FP64 solve as a capturable graph fragment on st (loop bodies captured on body_st):
// transforms, range projection, the Krylov loop as a conditional node, inverse transform,
// true residual and the result record info[0..4] (see krylov_graph_finish).
struct ResidCtx {
  const vd_grid* G;
  vd_op op;
  bool dd;
  const SpecSystem* sys64;
  void* tmp;
};
static void resid_cb(const void* c, const void* x, void* y, cudaStream_t st) {
  const ResidCtx& r = *static_cast<const ResidCtx*>(c);
  const cpx<double>* xi = (const cpx<double>*)x;
  cpx<double>* yo = (cpx<double>*)y;
  if (r.dd && r.op == VD_OP_KRHO) apply_krho_spec_dd(r.G, xi, yo, r.tmp, nullptr, st);
  else if (r.dd && r.op == VD_OP_VELOCITY) apply_velocity_spec_dd(r.G, xi, yo, r.sys64->a, r.sys64->inv_sc, r.tmp, nullptr, st);
  else if (r.dd) apply_pressure_spec_dd(r.G, xi, yo, r.tmp, nullptr, st);
  else r.sys64->apply(*r.sys64, xi, yo, false, nullptr, st);
}

vd_status enqueue_solve_graph(const vd_grid* G, vd_op op, vd_solver solver, const vd_op_params* opp, double tol,
                              int maxit, int restart, int precision, const double* b, double* x, void* ws,
                              size_t ws_bytes, double* info, cudaStream_t st, cudaStream_t const* body) {
  cudaStream_t body_st = body[0];
  vd_status e = check_op(G, op, opp);
  if (e != VD_OK) return e;
  if (op == VD_OP_KRHO) return fail(VD_ERR_INVALID_ARG, "graph solves cover the pressure and velocity operators");
  if (solver == VD_SOLVER_CG && op == VD_OP_VELOCITY)
    return fail(VD_ERR_INVALID_ARG, "CG needs a symmetric operator; V_rho is not symmetric");
  if (solver == VD_SOLVER_GMRES && restart > kMaxRestart) return fail(VD_ERR_INVALID_ARG, "GMRES restart must be <= 64");
  if (precision != VD_PREC_FP64 && precision != VD_PREC_MIXED && precision != VD_PREC_MIXED_DD)
    return fail(VD_ERR_INVALID_ARG, "unknown precision mode");
  size_t need = 0;
  SolveLayout L = solve_layout(G, op, solver, restart, maxit, precision, ws, &need);
  if (ws_bytes < need) return fail(VD_ERR_OOM, "workspace too small");
  const int ncomp = op_ncomp(G, op);
  const long long len = G->g.ncplx * ncomp;
  VD_CUDA(cudaMemsetAsync(L.counter, 0, sizeof(unsigned), st));
  // the double symbol serves only double Krylov iterations
  if (precision == VD_PREC_FP64) fill_symbol<double>(G, op_symbol(op), opp ? opp->a : 0.0, L.sym, st);
  const bool dd = precision == VD_PREC_MIXED_DD && op != VD_OP_VELOCITY;
  if (dd) fwd_transform_dd(G, b, L.bh, L.tmp, st);
  else fwd_all(G, ncomp, b, L.bh, st);
  if (op == VD_OP_PRESSURE) spec_project<double>(G, 1, L.bh, st);
  VD_CUDA(cudaMemsetAsync(L.xh, 0, sizeof(cpx<double>) * len, st));
  KWork kw{L.ks, L.partials, L.counter, L.hist};
  if (precision != VD_PREC_FP64) {
    fill_symbol<float>(G, op_symbol(op), opp ? opp->a : 0.0, L.sym_f, st);
    SpecSystem sys64 = make_system<double>(G, op, opp, L.sym, L.tmp);
    SpecSystem sys32 = make_system<float>(G, op, opp, L.sym_f, L.tmp_f);
    // the refinement residual in float pairs for every operator (the entry and exit transforms of
    // the velocity components stay double)
    ResidCtx rc{G, op, precision == VD_PREC_MIXED_DD, &sys64, L.tmp};
    SolveOpts si;
    si.solver = solver;
    si.tol = 0.0;
    si.maxit = maxit;
    si.restart = restart;
    si.check_every = 1;
    si.x_zero = 1;
    e = refine_enqueue_graph(sys64, sys32, &resid_cb, &rc, si, tol, auto_inner_tol(G), maxit, L.bh, L.xh, L.rh, L.bh_f, L.xh_f,
                             L.vecs, kw, L.ost, info, st, body[0], body[1], body[2]);
    if (e != VD_OK) return e;
    if (dd) inv_transform_dd(G, L.xh, x, L.tmp, st);
    else inv_all(G, ncomp, L.xh, x, L.tmp, st);
    VD_CUDA(cudaGetLastError());
    return VD_OK;
  }
  SolveOpts so;
  so.solver = solver;
  so.tol = tol;
  so.maxit = maxit;
  so.restart = restart;
  so.check_every = 1;
  so.x_zero = 1;
  SpecSystem sys = make_system<double>(G, op, opp, L.sym, L.tmp);
  if ((e = krylov_enqueue_graph<double>(sys, so, L.bh, L.xh, L.vecs, kw, st, body_st)) != VD_OK) return e;
  inv_all(G, ncomp, L.xh, x, L.tmp, st);
  return krylov_graph_finish<double>(sys, L.bh, L.xh, L.vecs, kw, info, st);
}

}  // namespace vd

extern "C" {

size_t vd_workspace_bytes(const vd_grid* G, vd_op op, vd_solver solver, const vd_solve_params* p) {
  if (!G) return 0;
  const int restart = p ? p->restart : 30;
  const int maxit = p ? p->max_it : 1000;
  const int prec = p ? p->precision : VD_PREC_FP64;
  size_t b = 0;
  solve_layout(G, op, solver, restart, maxit, prec, nullptr, &b);
  return b;
}

vd_status vd_apply_op(const vd_grid* G, vd_op op, const vd_op_params* p, const double* in, double* out, void* ws,
                      size_t ws_bytes, vd_stream stream) {
  vd_status e = check_op(G, op, p);
  if (e != VD_OK) return e;
  if (!in || !out || !ws) return fail(VD_ERR_INVALID_ARG, "null buffer");
  cudaStream_t st = (cudaStream_t)stream;
  size_t need = 0;
  SolveLayout L = solve_layout(G, op, VD_SOLVER_RMR, 1, 1, VD_PREC_FP64, ws, &need);
  if (ws_bytes < need) return fail(VD_ERR_OOM, "workspace too small");
  const int ncomp = op_ncomp(G, op);
  SpecSystem sys = make_system<double>(G, op, p, nullptr, L.tmp);
  fwd_all(G, ncomp, in, L.bh, st);
  sys.apply(sys, L.bh, L.xh, false, nullptr, st);
  inv_all(G, ncomp, L.xh, out, L.tmp, st);
  VD_CUDA(cudaGetLastError());
  return VD_OK;
}

vd_status vd_apply_precond(const vd_grid* G, vd_op op, const vd_op_params* p, const double* in, double* out,
                           void* ws, size_t ws_bytes, vd_stream stream) {
  if (!G) return fail(VD_ERR_INVALID_ARG, "null grid");
  if (op == VD_OP_VELOCITY && !p) return fail(VD_ERR_INVALID_ARG, "velocity preconditioner needs vd_op_params");
  if (!in || !out || !ws) return fail(VD_ERR_INVALID_ARG, "null buffer");
  cudaStream_t st = (cudaStream_t)stream;
  size_t need = 0;
  SolveLayout L = solve_layout(G, op, VD_SOLVER_RMR, 1, 1, VD_PREC_FP64, ws, &need);
  if (ws_bytes < need) return fail(VD_ERR_OOM, "workspace too small");
  const int ncomp = op_ncomp(G, op);
  if (op != VD_OP_PRESSURE && op != VD_OP_VELOCITY && op != VD_OP_KRHO)
    return fail(VD_ERR_INVALID_ARG, "unknown operator");
  fill_symbol<double>(G, op_symbol(op), p ? p->a : 0.0, L.sym, st);
  fwd_all(G, ncomp, in, L.bh, st);
  for (int c = 0; c < ncomp; ++c) {
    Mult m;
    m.sym = 1;
    m.symarr = L.sym;
    inv_transform<double>(G, L.bh + (size_t)c * G->g.ncplx, m, out + (size_t)c * G->g.nreal, L.tmp, st);
  }
  VD_CUDA(cudaGetLastError());
  return VD_OK;
}

size_t vd_transform_ws_bytes(const vd_grid* G, int prec) {
  if (!G) return 0;
  const size_t el = (prec == VD_PREC_MIXED) ? sizeof(cpx<float>) : sizeof(cpx<double>);
  return align256((size_t)G->g.ncplx * el);
}

vd_status vd_fft_r2c(const vd_grid* G, int prec, const void* in, void* out, void* ws, size_t ws_bytes,
                     vd_stream stream) {
  if (!G || !in || !out) return fail(VD_ERR_INVALID_ARG, "null argument");
  if (prec != VD_PREC_FP64 && prec != VD_PREC_MIXED && prec != VD_PREC_MIXED_DD)
    return fail(VD_ERR_INVALID_ARG, "unknown precision mode");
  if (in == out) return fail(VD_ERR_INVALID_ARG, "in and out must not alias");
  cudaStream_t st = (cudaStream_t)stream;
  if (prec == VD_PREC_FP64) {
    fwd_transform<double>(G, (const double*)in, (cpx<double>*)out, st);
  } else if (prec == VD_PREC_MIXED) {
    fwd_transform<float>(G, (const float*)in, (cpx<float>*)out, st);
  } else {
    if (!ws || ws_bytes < vd_transform_ws_bytes(G, prec)) return fail(VD_ERR_OOM, "transform workspace too small");
    fwd_transform_dd(G, (const double*)in, (cpx<double>*)out, ws, st);
  }
  VD_CUDA(cudaGetLastError());
  return VD_OK;
}

vd_status vd_fft_c2r(const vd_grid* G, int prec, const void* in, void* out, void* ws, size_t ws_bytes,
                     vd_stream stream) {
  if (!G || !in || !out) return fail(VD_ERR_INVALID_ARG, "null argument");
  if (prec != VD_PREC_FP64 && prec != VD_PREC_MIXED && prec != VD_PREC_MIXED_DD)
    return fail(VD_ERR_INVALID_ARG, "unknown precision mode");
  if (in == out) return fail(VD_ERR_INVALID_ARG, "in and out must not alias");
  if (G->g.ndim > 1 && (!ws || ws_bytes < vd_transform_ws_bytes(G, prec)))
    return fail(VD_ERR_OOM, "transform workspace too small");
  cudaStream_t st = (cudaStream_t)stream;
  Mult m;
  if (prec == VD_PREC_FP64) inv_transform<double>(G, (const cpx<double>*)in, m, (double*)out, (cpx<double>*)ws, st);
  else if (prec == VD_PREC_MIXED) inv_transform<float>(G, (const cpx<float>*)in, m, (float*)out, (cpx<float>*)ws, st);
  else inv_transform_dd(G, (const cpx<double>*)in, (double*)out, ws, st);
  VD_CUDA(cudaGetLastError());
  return VD_OK;
}

vd_status vd_divergence(const vd_grid* G, const double* u, double* out, void* ws, size_t ws_bytes, vd_stream stream) {
  if (!G || !u || !out || !ws) return fail(VD_ERR_INVALID_ARG, "null argument");
  cudaStream_t st = (cudaStream_t)stream;
  const GridDesc& g = G->g;
  const size_t need = align256((size_t)g.ncplx * 16 * 3);
  if (ws_bytes < need) return fail(VD_ERR_OOM, "workspace too small (3 spectral fields)");
  cpx<double>* a = (cpx<double>*)ws;
  cpx<double>* acc = a + g.ncplx;
  cpx<double>* tmp = acc + g.ncplx;
  // out = sum_j F^-1(i k_j F u_j): accumulate i k_j u^_j in spectral space via derivative transforms
  VD_CUDA(cudaMemsetAsync(out, 0, sizeof(double) * g.nreal, st));
  for (int j = 0; j < g.ndim; ++j) {
    fwd_transform<double>(G, u + (size_t)j * g.nreal, a, st);
    Mult m;
    m.deriv[j] = 1;
    inv_transform<double>(G, a, m, reinterpret_cast<double*>(acc), tmp, st);
    // out += acc (physical): reuse spectral axpy on reals viewed as complex pairs
    spec_axpy<double>(g.nreal / 2, 1.0, acc, out, st);
  }
  VD_CUDA(cudaGetLastError());
  return VD_OK;
}

vd_status vd_gradient(const vd_grid* G, const double* phi, double* out, void* ws, size_t ws_bytes, vd_stream stream) {
  if (!G || !phi || !out || !ws) return fail(VD_ERR_INVALID_ARG, "null argument");
  cudaStream_t st = (cudaStream_t)stream;
  const GridDesc& g = G->g;
  const size_t need = align256((size_t)g.ncplx * 16 * 3);
  if (ws_bytes < need) return fail(VD_ERR_OOM, "workspace too small (3 spectral fields)");
  cpx<double>* a = (cpx<double>*)ws;
  cpx<double>* tmp = a + g.ncplx;
  fwd_transform<double>(G, phi, a, st);
  for (int j = 0; j < g.ndim; ++j) {
    Mult m;
    m.deriv[j] = 1;
    inv_transform<double>(G, a, m, out + (size_t)j * g.nreal, tmp, st);
  }
  VD_CUDA(cudaGetLastError());
  return VD_OK;
}

vd_status vd_solve(const vd_grid* G, vd_op op, vd_solver solver, const vd_op_params* opp, const vd_solve_params* prm,
                   const double* b, double* x, vd_solve_info* info, void* ws, size_t ws_bytes, vd_stream stream) {
  vd_status e = check_op(G, op, opp);
  if (e != VD_OK) return e;
  if (!prm || !b || !x || !ws) return fail(VD_ERR_INVALID_ARG, "null argument");
  if (solver != VD_SOLVER_CG && solver != VD_SOLVER_GMRES && solver != VD_SOLVER_RMR)
    return fail(VD_ERR_INVALID_ARG, "unknown solver");
  if (solver == VD_SOLVER_CG && op == VD_OP_VELOCITY)
    return fail(VD_ERR_INVALID_ARG, "CG needs a symmetric operator; V_rho is not symmetric");
  if (!(prm->tol >= 0.0) || prm->max_it < 0) return fail(VD_ERR_INVALID_ARG, "tol must be >= 0 and max_it >= 0");
  if (prm->precision != VD_PREC_FP64 && prm->precision != VD_PREC_MIXED && prm->precision != VD_PREC_MIXED_DD)
    return fail(VD_ERR_INVALID_ARG, "unknown precision mode");
  if (solver == VD_SOLVER_GMRES && prm->restart > kMaxRestart)
    return fail(VD_ERR_INVALID_ARG, "GMRES restart must be <= 64");
  cudaStream_t st = (cudaStream_t)stream;
  const int restart = prm->restart > 0 ? prm->restart : 30;
  size_t need = 0;
  SolveLayout L = solve_layout(G, op, solver, restart, prm->max_it, prm->precision, ws, &need);
  if (ws_bytes < need) return fail(VD_ERR_OOM, "workspace too small");
  // small 1D pressure problems: the whole solve in one kernel launch (vd_small.cu)
  if (!(prm->range_tol > 0.0) && small_solve_eligible(G, op, solver, prm->precision, restart))
    return small_solve_1d(G, solver, prm, restart, b, x, info, L.ks, L.hist, std::max(prm->max_it, 1) + 2, st);
  const GridDesc& g = G->g;
  const int ncomp = op_ncomp(G, op);
  const long long len = g.ncplx * ncomp;
  const int symkind = op_symbol(op);
  // the reduction ticket counter must start at zero (the workspace is uninitialised memory)
  VD_CUDA(cudaMemsetAsync(L.counter, 0, sizeof(unsigned), st));
  // the double symbol serves only double Krylov iterations (the refinement applies A unpreconditioned)
  if (prm->precision == VD_PREC_FP64) fill_symbol<double>(G, symkind, opp ? opp->a : 0.0, L.sym, st);
  // spectral right-hand side and initial guess (float-pair transforms in VD_PREC_MIXED_DD
  // pressure solves, double otherwise)
  const bool dd_io = prm->precision == VD_PREC_MIXED_DD && op != VD_OP_VELOCITY;
  if (dd_io) fwd_transform_dd(G, b, L.bh, L.tmp, st);
  else fwd_all(G, ncomp, b, L.bh, st);
  // range projection (reading c4): the removed part's squared norm, in the weighted spectral
  // norm of the solver, is kept in removed2 (pressure: read back with the results)
  const int ncorner = 1 << g.ndim;
  double removed2 = 0.0;
  double removed_host[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  if (op == VD_OP_PRESSURE) spec_project<double>(G, 1, L.bh, st, L.removed);
  KWork kw{L.ks, L.partials, L.counter, L.hist};
  if (op == VD_OP_KRHO) {
    // remove the component along w = rho^-1/2 (the range of K~ is w-orthogonal)
    SpecSystem s1{};
    s1.G = G;
    s1.len = len;
    s1.h0 = g.h0;
    const double d = spec_dot_host<double>(s1, L.bh, G->kw_hat, kw, st);
    spec_axpy<double>(len, -d, G->kw_hat, L.bh, st);
    removed2 = d * d;   // w^ has unit weighted norm
  }
  SpecSystem sysn{};
  sysn.G = G;
  sysn.len = len;
  sysn.h0 = g.h0;
  if (prm->range_tol > 0.0 && op != VD_OP_VELOCITY) {
    if (op == VD_OP_PRESSURE) {
      VD_CUDA(cudaMemcpyAsync(removed_host, L.removed, sizeof(double) * ncorner, cudaMemcpyDeviceToHost, st));
      VD_CUDA(cudaStreamSynchronize(st));
      for (int k = 0; k < ncorner; ++k) removed2 += removed_host[k];
    }
    const double kept2 = spec_norm2_host<double>(sysn, L.bh, kw, st);
    if (removed2 > prm->range_tol * prm->range_tol * (kept2 + removed2)) {
      if (info) {
        info->iters = 0;
        info->outer_iters = 0;
        info->status = VD_ERR_RHS_NOT_IN_RANGE;
        info->relres = info->relres_true = 0.0;
        info->hist_len = 0;
        info->rhs_removed = std::sqrt(removed2 / (kept2 + removed2));
        info->coef_pair = 0;
      }
      char buf[160];
      std::snprintf(buf, sizeof buf, "right-hand side outside the range: ||Pi b - b|| / ||b|| = %.3e > range_tol",
                    std::sqrt(removed2 / (kept2 + removed2)));
      return fail(VD_ERR_RHS_NOT_IN_RANGE, buf);
    }
  }
  if (prm->use_x0) {
    if (dd_io) fwd_transform_dd(G, x, L.xh, L.tmp, st);
    else fwd_all(G, ncomp, x, L.xh, st);
    if (op == VD_OP_PRESSURE) spec_project<double>(G, 1, L.xh, st);
    if (op == VD_OP_KRHO) VD_CUDA(cudaMemsetAsync(L.xh, 0, sizeof(cpx<double>), st));   // zero mean
  } else {
    VD_CUDA(cudaMemsetAsync(L.xh, 0, sizeof(cpx<double>) * len, st));
  }
  SolveOpts so;
  so.solver = solver;
  so.tol = prm->tol;
  so.maxit = prm->max_it;
  so.restart = restart;
  so.check_every = prm->check_every > 0 ? prm->check_every : 1;
  so.x_zero = prm->use_x0 ? 0 : 1;
  SolveOut res{0, VD_ERR_NOT_CONVERGED, 0.0};
  double* hh = (info && info->hist && info->hist_cap > 0) ? info->hist : nullptr;
  // the device history buffer holds max_it + 2 entries
  const int hcap = hh ? std::min(info->hist_cap, prm->max_it + 2) : 0;
  SpecSystem sys64 = make_system<double>(G, op, opp, L.sym, L.tmp);
  bool x_phys_current = false;   // x already holds the inverse transform of the final L.xh
  bool coef_pair_used = false;
  int outer = 0;
  double relres_true = 0.0;
  if (prm->precision == VD_PREC_FP64) {
    e = krylov_solve<double>(sys64, so, L.bh, L.xh, L.vecs, kw, hh, hcap, &res, st);
    if (e != VD_OK) return e;
  } else {
    // iterative refinement: r = b - A64 x; inner float solve A32 d = r/|r|; x += |r| d
    fill_symbol<float>(G, symkind, opp ? opp->a : 0.0, L.sym_f, st);
    SpecSystem sys32 = make_system<float>(G, op, opp, L.sym_f, L.tmp_f, prm->coef_pair);
    coef_pair_used = sys32.ctx[3] != nullptr;
    // residual operator of the refinement: double, or float-pair transforms
    const bool use_dd = prm->precision == VD_PREC_MIXED_DD;
    // With want_phys the float-pair pressure residual also writes the physical-space iterate
    // into x (its fused x pass carries the inverse transform of the iterate); when the loop
    // ends right after such a residual the final inverse transform is skipped.  It is asked
    // for on a sweep expected to be the last: the outer residual it aims at (rel times the
    // inner tolerance) within a factor 10 of tol.  A wrong guess either way costs time only.
    auto resid_apply = [&](const cpx<double>* xin, cpx<double>* yout, bool want_phys) {
      if (use_dd && op == VD_OP_KRHO) {
        apply_krho_spec_dd(G, xin, yout, L.tmp, nullptr, st);
        x_phys_current = false;
      } else if (use_dd && op == VD_OP_VELOCITY) {
        apply_velocity_spec_dd(G, xin, yout, sys64.a, sys64.inv_sc, L.tmp, nullptr, st);
        x_phys_current = false;
      } else if (use_dd) {
        apply_pressure_spec_dd(G, xin, yout, L.tmp, nullptr, st, want_phys ? x : nullptr);
        x_phys_current = want_phys;
      } else {
        sys64.apply(sys64, xin, yout, false, nullptr, st);
      }
    };
    const double bb = spec_norm2_host<double>(sys64, L.bh, kw, st);
    const double bnorm = std::sqrt(bb);
    // r = b - A x0; with x0 = 0 the first sweep reads b itself and |r| = |b|
    const cpx<double>* r_cur = L.bh;
    double rnorm = bnorm;
    if (prm->use_x0) {
      resid_apply(L.xh, L.rh, false);
      rnorm = std::sqrt(spec_sub_norm2_host(sys64, L.bh, L.rh, L.rh, kw, st));
      r_cur = L.rh;
    }
    int total = 0;
    int hlen = 0;
    if (hh && hcap > 0) hh[hlen++] = bnorm > 0 ? rnorm / bnorm : 0.0;
    res.status = VD_ERR_NOT_CONVERGED;
    const double itol = prm->inner_tol > 0 ? prm->inner_tol : auto_inner_tol(G);
    const int max_outer = 20;
    for (;;) {
      // a non-finite norm is reported as such (NaN > 0 is false: it must not read as a zero rhs)
      const double rel = (!std::isfinite(bnorm) || !std::isfinite(rnorm))
                             ? std::numeric_limits<double>::quiet_NaN()
                             : (bnorm > 0 ? rnorm / bnorm : 0.0);
      res.relres = rel;
      if (!std::isfinite(rel)) {
        res.status = VD_ERR_NONFINITE;
        break;
      }
      if (rel <= prm->tol) {
        res.status = VD_OK;
        break;
      }
      if (total >= prm->max_it || outer >= max_outer) break;
      spec_d2f_scaled(len, r_cur, 1.0 / rnorm, L.bh_f, st);
      VD_CUDA(cudaMemsetAsync(L.xh_f, 0, sizeof(cpx<float>) * len, st));
      SolveOpts si = so;
      // ask the inner solve for a little more than needed so that the refined residual lands
      // below tol when it is the last sweep
      si.tol = std::max(itol, 0.5 * prm->tol / rel);
      si.maxit = prm->max_it - total;
      si.x_zero = 1;
      si.guard = kInnerGuard;
      SolveOut ri{0, 0, 0.0};
      std::vector<double> ih;
      const int icap = hh ? std::min(std::max(0, hcap - hlen) + 1, prm->max_it + 2) : 0;
      if (icap > 0) ih.resize(icap);
      {
        ProfSpan span(PC_INNER32, st);   // the whole inner solve, for the profiler's span mode
        e = krylov_solve<float>(sys32, si, L.bh_f, L.xh_f, L.vecs, kw, icap > 0 ? ih.data() : nullptr, icap, &ri, st);
      }
      if (e != VD_OK) return e;
      // history: inner residuals rescaled to the outer right-hand side
      for (int i = 1; i <= ri.iters && hlen < hcap && i < (int)ih.size(); ++i) hh[hlen++] = ih[i] * rel;
      total += ri.iters;
      ++outer;
      // x += rnorm * d  (d promoted to double)
      spec_axpy_f2d(len, rnorm, L.xh_f, L.xh, st);
      // true residual (double operator, or float-pair transforms in VD_PREC_MIXED_DD)
      resid_apply(L.xh, L.rh, rel * si.tol <= 10.0 * prm->tol);
      rnorm = std::sqrt(spec_sub_norm2_host(sys64, L.bh, L.rh, L.rh, kw, st));
      r_cur = L.rh;
      if (ri.status == VD_ERR_NONFINITE) {
        res.status = VD_ERR_NONFINITE;
        break;
      }
      if (ri.iters == 0 && ri.status != VD_OK) break;
    }
    res.iters = total;
    relres_true = bnorm > 0 ? rnorm / bnorm : 0.0;
    if (info) info->hist_len = hlen;
  }
  // back to physical space
  if (dd_io && !x_phys_current) inv_transform_dd(G, L.xh, x, L.tmp, st);
  else if (!dd_io) inv_all(G, ncomp, L.xh, x, L.tmp, st);
  if (prm->precision == VD_PREC_FP64) {
    // true residual of the returned iterate
    const double bb = spec_norm2_host<double>(sys64, L.bh, kw, st);
    sys64.apply(sys64, L.xh, L.rh, false, nullptr, st);
    spec_sub<double>(len, L.bh, L.rh, L.rh, st);
    const double rr = spec_norm2_host<double>(sys64, L.rh, kw, st);
    relres_true = bb > 0 ? std::sqrt(rr / bb) : 0.0;
    if (info) info->hist_len = hh ? std::min(hcap, res.iters + 1) : 0;
  }
  VD_CUDA(cudaGetLastError());
  if (op == VD_OP_PRESSURE && !(prm->range_tol > 0.0))
    VD_CUDA(cudaMemcpyAsync(removed_host, L.removed, sizeof(double) * ncorner, cudaMemcpyDeviceToHost, st));
  int dev_err = 0;
  if (g.dev_err) VD_CUDA(cudaMemcpyAsync(&dev_err, g.dev_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  VD_CUDA(cudaStreamSynchronize(st));
  if (dev_err) {
    VD_CUDA(cudaMemsetAsync(g.dev_err, 0, sizeof(int), st));
    VD_CUDA(cudaStreamSynchronize(st));
    return fail(VD_ERR_TIMEOUT, "a transform pass gave up waiting for its staged input (bounded wait); "
                                "the result is not valid");
  }
  if (op == VD_OP_PRESSURE && !(prm->range_tol > 0.0))
    for (int k = 0; k < ncorner; ++k) removed2 += removed_host[k];
  if (info) {
    info->iters = res.iters;
    info->outer_iters = outer;
    info->status = res.status;
    info->relres = res.relres;
    info->relres_true = relres_true;
    double kept2 = 0.0;
    if (removed2 > 0.0) kept2 = spec_norm2_host<double>(sysn, L.bh, kw, st);
    info->rhs_removed = removed2 > 0.0 ? std::sqrt(removed2 / (kept2 + removed2)) : 0.0;
    info->coef_pair = coef_pair_used ? 1 : 0;
  }
  if (res.status != VD_OK) {
    char buf[160];
    std::snprintf(buf, sizeof buf, "solve ended with status %d after %d iterations (relres %.3e)", res.status,
                  res.iters, res.relres);
    g_err = buf;
  }
  return (vd_status)res.status;
}

}  // extern "C"
