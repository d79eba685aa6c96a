// Pressure-operator apply that allocates no device memory.
//
// Some callers cannot call cudaMalloc: code that runs inside a host framework whose memory
// pool owns the whole device (raw allocations are forbidden or would fail), plugins that
// must not change the device memory footprint at run time, and latency-critical loops in
// which an allocation (which may synchronise the device) is not acceptable.  For them,
// vd_apply_pressure_noalloc computes out = L~_rho(in) with every intermediate (twiddle
// tables, 1/(N rho), spectral temporaries) kept in one file-scope device array of fixed size,
// so the call needs neither a grid object nor a workspace.  The caller passes only the grid
// description and its input/output buffers.
//
// The array is shared by every call of the process on a given device and keeps the last
// call's contents; nothing in it needs to start at zero except the density check flag, which
// each call clears.  Two calls whose kernels overlap on the GPU (different streams, or
// different host threads) race on the array: serialise them.
#include "vd_internal.h"
#include "vd_prof.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <mutex>

namespace vd {

// 32 MiB: enough for 3D grids up to 64^3, 2D up to 512 x 1024 and 1D lengths up to 1024 (the
// axis-length limit every entry point applies).
constexpr size_t kNoAllocScratchBytes = 32ull << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

static std::mutex g_na_mu;
static void* g_na_ptr[64] = {nullptr};

// device address of the scratch array on the current device, looked up once per device and
// kept for the life of the process (a cudaDeviceReset of that device would leave it stale:
// the entry point must not be used across one)
static vd_status noalloc_scratch(void** out) {
  int dev = 0;
  VD_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(VD_ERR_INVALID_ARG, "device index out of range for the no-allocation path");
  std::lock_guard<std::mutex> lk(g_na_mu);
  if (!g_na_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-allocation scratch)");
    g_na_ptr[dev] = p;
  }
  *out = g_na_ptr[dev];
  return VD_OK;
}

static bool na_plan(int n, FftPlan* p) {
  if (n < 2 || n > 4096) return false;
  int a = 0, b = 0, c = 0, r = n;
  while (r % 2 == 0) { r /= 2; ++a; }
  while (r % 3 == 0) { r /= 3; ++b; }
  while (r % 5 == 0) { r /= 5; ++c; }
  if (r != 1) return false;
  p->n = n;
  p->nst = 0;
  while (a >= 3) { p->rad[p->nst++] = 8; a -= 3; }
  if (a == 2) p->rad[p->nst++] = 4;
  if (a == 1) p->rad[p->nst++] = 2;
  while (b-- > 0) p->rad[p->nst++] = 3;
  while (c-- > 0) p->rad[p->nst++] = 5;
  return true;
}

// twiddles W_len^j = exp(-2 pi i j / len) for the four tables of a grid
__global__ void k_na_twiddles(GridDesc g, cpx<double>* tw) {
  const int m = g.n0 / 2;
  const int total = g.pk_off + m + 1;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    int j, len;
    if (t >= g.pk_off) {
      j = t - g.pk_off;
      len = g.n0;
    } else if (t >= g.pz.tw_off && g.ndim == 3) {
      j = t - g.pz.tw_off;
      len = g.pz.n;
    } else if (t >= g.py.tw_off && g.ndim >= 2) {
      j = t - g.py.tw_off;
      len = g.py.n;
    } else {
      j = t - g.px.tw_off;
      len = g.px.n;
    }
    double s, c;
    sincospi(2.0 * (double)j / (double)len, &s, &c);
    tw[t] = mk<double>(c, -s);
  }
}

__global__ void k_na_density(long long n, const double* __restrict__ rho, double invN, double* __restrict__ rinv,
                             int* bad) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const double r = rho[e];
    if (!(r > 0.0) || !isfinite(r)) *bad = 1;
    rinv[e] = invN / r;
  }
}

static size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace vd

using namespace vd;

extern "C" vd_status vd_apply_pressure_noalloc(int ndim, const int n[3], const double L[3], const double* rho,
                                               const double* in, double* out, vd_stream stream) {
  if (!n || !L || !rho || !in || !out) return fail(VD_ERR_INVALID_ARG, "null argument");
  if (ndim < 1 || ndim > 3) return fail(VD_ERR_INVALID_ARG, "ndim must be 1, 2 or 3");
  if (in == out) return fail(VD_ERR_INVALID_ARG, "in and out must not alias");
  // grid description on the stack (same plans and layout as vd_grid_create)
  vd_grid G;
  GridDesc& g = G.g;
  int nn[3] = {1, 1, 1};
  for (int j = 0; j < ndim; ++j) {
    if (n[j] < 4 || n[j] > 1024 || (n[j] % 2) != 0)
      return fail(VD_ERR_INVALID_ARG, "axis lengths must be even and in [4, 1024]");
    if (!(L[j] > 0.0) || !std::isfinite(L[j])) return fail(VD_ERR_INVALID_ARG, "box lengths must be positive");
    nn[j] = n[j];
  }
  g.ndim = ndim;
  g.n0 = nn[0];
  g.n1 = nn[1];
  g.n2 = nn[2];
  g.h0 = nn[0] / 2 + 1;
  g.nreal = (long long)nn[0] * nn[1] * nn[2];
  g.ncplx = (long long)g.h0 * nn[1] * nn[2];
  for (int j = 0; j < 3; ++j) {
    G.L[j] = (j < ndim) ? L[j] : 1.0;
    g.kfac[j] = 2.0 * 3.14159265358979323846 / G.L[j];
    g.kfac_dd[j][0] = (float)g.kfac[j];
    g.kfac_dd[j][1] = (float)(g.kfac[j] - (double)g.kfac_dd[j][0]);
    g.kfac_f[j] = (float)g.kfac[j];
  }
  bool ok = na_plan(nn[0] / 2, &g.px);
  int off = 0;
  g.px.tw_off = off;
  off += g.px.n;
  if (ndim >= 2) {
    ok = ok && na_plan(nn[1], &g.py);
    g.py.tw_off = off;
    off += g.py.n;
  } else {
    g.py = g.px;
  }
  if (ndim == 3) {
    ok = ok && na_plan(nn[2], &g.pz);
    g.pz.tw_off = off;
    off += g.pz.n;
  } else {
    g.pz = g.py;
  }
  if (!ok) return fail(VD_ERR_INVALID_ARG, "axis lengths must factor into 2, 3 and 5");
  g.pk_off = off;
  const size_t ntw = (size_t)off + g.n0 / 2 + 1;
  // scratch layout: flag | twiddles | 1/(N rho) | b^ | x^ | 3 temporaries
  const size_t fc = (size_t)g.ncplx * sizeof(cpx<double>);
  const size_t o_tw = 256;
  const size_t o_ri = a256(o_tw + ntw * sizeof(cpx<double>));
  const size_t o_b = a256(o_ri + (size_t)g.nreal * sizeof(double));
  const size_t o_x = a256(o_b + fc);
  const size_t o_t = a256(o_x + fc);
  const size_t need = a256(o_t + 3 * fc);
  if (need > kNoAllocScratchBytes) {
    char msg[200];
    std::snprintf(msg, sizeof msg,
                  "grid too large for the no-allocation path: needs %zu bytes of scratch, the fixed array holds %zu",
                  need, kNoAllocScratchBytes);
    return fail(VD_ERR_INVALID_ARG, msg);
  }
  void* base = nullptr;
  vd_status st0 = noalloc_scratch(&base);
  if (st0 != VD_OK) return st0;
  char* sb = static_cast<char*>(base);
  cudaStream_t st = (cudaStream_t)stream;
  int* bad = reinterpret_cast<int*>(sb);
  cpx<double>* tw = reinterpret_cast<cpx<double>*>(sb + o_tw);
  double* rinv = reinterpret_cast<double*>(sb + o_ri);
  cpx<double>* bh = reinterpret_cast<cpx<double>*>(sb + o_b);
  cpx<double>* xh = reinterpret_cast<cpx<double>*>(sb + o_x);
  cpx<double>* tmp = reinterpret_cast<cpx<double>*>(sb + o_t);
  G.tw_d = tw;
  G.tw_f = nullptr;
  G.rinv_s = rinv;
  G.has_density = 1;

  VD_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), st));
  { k_na_twiddles<<<(unsigned)((ntw + 255) / 256), 256, 0, st>>>(g, tw); count_launch(); }
  const int db = (int)std::min<long long>(1024, (g.nreal + 255) / 256);
  { k_na_density<<<db, 256, 0, st>>>(g.nreal, rho, 1.0 / (double)g.nreal, rinv, bad); count_launch(); }
  int hbad = 0;
  VD_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
  VD_CUDA(cudaStreamSynchronize(st));
  if (hbad) return fail(VD_ERR_INVALID_ARG, "density must be positive and finite");
  fwd_transform<double>(&G, in, bh, st);
  apply_pressure_spec<double>(&G, bh, xh, nullptr, rinv, tmp, nullptr, st);
  Mult m;
  inv_transform<double>(&G, xh, m, out, tmp, st);
  VD_CUDA(cudaGetLastError());
  return VD_OK;
}
