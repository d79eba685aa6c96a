// Launch-shape autotuner of the transform passes (not in the paper).
//
// For a grid and each requested arithmetic type, every pass the solver uses -- the y and z
// passes in both directions, and the x pass in its three forms (forward real-to-half-spectrum,
// inverse, and the fused inverse-weight-forward form of the operators) -- is timed with CUDA
// events (median of seven launches) for each candidate shape: the register-resident four-step
// kernel where one exists (float, lengths 128 and 256; x pass n0 = 128, 256, 512) and the
// Stockham engine with 1, 2, 4, ... lines per block up to the shared-memory limit.  A shape
// replaces the built-in choice only when it is at least 3% faster; the winner goes into the
// process-wide launch table that every later launch consults (and, with VD_TUNE_FILE set, into
// that file).  Shapes change only the work distribution, never the arithmetic of a line,
// except that the register kernel and the Stockham engine round differently (both are
// complete transforms; the parity tests hold for either).
#include "vd_internal.h"
#include "vd_dd.cuh"
#include "vd_passes.cuh"
#include "vd_prof.h"

#include <algorithm>
#include <vector>

namespace vd {

namespace {

constexpr size_t kSmemCap = 200 * 1024;

struct Timer {
  cudaEvent_t a = nullptr, b = nullptr;
  Timer() {
    cudaEventCreate(&a);
    cudaEventCreate(&b);
  }
  ~Timer() {
    cudaEventDestroy(a);
    cudaEventDestroy(b);
  }
};

// median of seven timed launches after two warm-ups (ms per launch)
template <typename F>
float time_it(F&& launch, cudaStream_t st, Timer& t) {
  launch();
  launch();
  float ms[7];
  for (int r = 0; r < 7; ++r) {
    cudaEventRecord(t.a, st);
    launch();
    cudaEventRecord(t.b, st);
    cudaEventSynchronize(t.b);
    cudaEventElapsedTime(&ms[r], t.a, t.b);
  }
  std::sort(ms, ms + 7);
  return ms[3];
}

// keep the built-in shape unless a candidate beats it clearly (timing noise must not flip it)
constexpr float kSwitchGain = 0.97f;

Xf plain_xf() {
  Xf x{};
  x.src = 0;
  x.dst = 0;
  x.first = 1;
  x.last = 1;
  x.scale = 1.0;
  return x;
}

template <typename T>
constexpr int tcode() {
  return std::is_same<T, dd>::value ? 2 : (sizeof(T) == 4 ? 1 : 0);
}

template <typename T>
vd_status tune_type(const vd_grid* G, const void* tw, void* a, void* b, cudaStream_t st, Timer& tm) {
  const GridDesc& g = G->g;
  const int type = tcode<T>();
  // y and z passes
  for (int axis = 1; axis <= 2; ++axis) {
    if (axis == 1 && g.ndim < 2) continue;
    if (axis == 2 && g.ndim < 3) continue;
    const int n = axis == 2 ? g.pz.n : g.py.n;
    const long long inner = axis == 2 ? (long long)g.n1 * g.h0 : g.h0;
    std::vector<int> cand;
    const bool reg = type == 1 && (n == 128 || n == 256);
    if (reg) cand.push_back(0);
    if (reg) cand.push_back(kChoiceStaged);
    for (int W = 1; W <= 64; W *= 2) {
      if (sizeof(cpx<T>) * (size_t)(n + 2 * W * n) > kSmemCap) break;
      if (W > 1 && W > 2 * inner) break;
      cand.push_back(W);
    }
    for (int dir = -1; dir <= 1; dir += 2) {
      AxisProg P{};
      P.nxf = 1;
      P.xf[0] = plain_xf();
      P.in[0] = a;
      P.out[0] = b;
      P.axis = axis;
      // the built-in shape first: the register kernel, else the heuristic tile width
      tune_set(0, type, n, axis, dir, -1);
      float tdef = time_it([&] { launch_axis<T>(P, dir, g, tw, st); }, st, tm);
      VD_CUDA(cudaGetLastError());
      int best = -1;
      float tbest = tdef * kSwitchGain;
      for (int c : cand) {
        tune_set(0, type, n, axis, dir, c);
        const float ms = time_it([&] { launch_axis<T>(P, dir, g, tw, st); }, st, tm);
        VD_CUDA(cudaGetLastError());
        if (ms < tbest) {
          tbest = ms;
          best = c;
        }
      }
      (void)reg;
      tune_set(0, type, n, axis, dir, best >= 0 ? best : default_shape(0, type, n, axis));
    }
  }
  // x pass: forward (mode 1), inverse (mode 2), fused (mode 0 with a weight field)
  const int m = g.n0 / 2;
  const long long nlines = (long long)g.n1 * g.n2;
  std::vector<int> cand;
  if (type == 1 && (m == 64 || m == 128 || m == 256)) cand.push_back(0);
  for (int L = 1; L <= 64; L *= 2) {
    if (sizeof(cpx<T>) * (size_t)(m + (m + 2) + 2 * L * (m + 1)) > kSmemCap) break;
    if (L > 1 && L > nlines) break;
    cand.push_back(L);
  }
  for (int mode = 0; mode <= 2; ++mode) {
    // the fused form can also stage its input lines with TMA (float register kernels)
    std::vector<int> cm = cand;
    if (mode == 0 && type == 1 && (m == 64 || m == 128 || m == 256) && nlines >= 2) cm.push_back(kChoiceStaged);
    XProg X{};
    X.ncomp = 1;
    X.mode = mode;
    X.in[0] = (mode == 2) ? (const void*)b : (mode == 1 ? (const void*)a : (const void*)b);
    X.out[0] = (mode == 2) ? a : b;
    X.wfield = (mode == 0) ? a : nullptr;
    X.scale = (mode == 2) ? 1.0 / (double)g.nreal : 0.5;
    tune_set(1, type, m, 0, mode, -1);
    const float tdef = time_it([&] { launch_xpass<T>(X, g, tw, st); }, st, tm);
    VD_CUDA(cudaGetLastError());
    int best = -1;
    float tbest = tdef * kSwitchGain;
    for (int c : cm) {
      tune_set(1, type, m, 0, mode, c);
      const float ms = time_it([&] { launch_xpass<T>(X, g, tw, st); }, st, tm);
      VD_CUDA(cudaGetLastError());
      if (ms < tbest) {
        tbest = ms;
        best = c;
      }
    }
    tune_set(1, type, m, 0, mode, best >= 0 ? best : default_shape(1, type, m));
  }
  return VD_OK;
}

}  // namespace

}  // namespace vd

extern "C" {

size_t vd_autotune_bytes(const vd_grid* G) {
  if (!G) return 0;
  return 2 * (size_t)G->g.ncplx * 16 + 256;
}

vd_status vd_autotune(const vd_grid* G, int precisions, void* scratch, size_t bytes, vd_stream stream) {
  using namespace vd;
  if (!G || !scratch) return fail(VD_ERR_INVALID_ARG, "null argument");
  if (precisions <= 0 || precisions > 7) return fail(VD_ERR_INVALID_ARG, "precisions: bit 0 double, 1 float, 2 float-pair");
  if (bytes < vd_autotune_bytes(G)) return fail(VD_ERR_OOM, "scratch smaller than vd_autotune_bytes");
  if (vd_profile_is_on()) return fail(VD_ERR_INVALID_ARG, "disable the profiler while tuning");
  cudaStream_t st = (cudaStream_t)stream;
  char* base = static_cast<char*>(scratch);
  void* a = base;
  void* b = base + (size_t)G->g.ncplx * 16;
  // defined data (zeros): timing on garbage could meet slow special values
  VD_CUDA(cudaMemsetAsync(scratch, 0, vd_autotune_bytes(G) - 256, st));
  Timer tm;
  vd_status e = VD_OK;
  if ((precisions & 1) && e == VD_OK) e = tune_type<double>(G, G->tw_d, a, b, st, tm);
  if ((precisions & 2) && e == VD_OK) e = tune_type<float>(G, G->tw_f, a, b, st, tm);
  if ((precisions & 4) && e == VD_OK) e = tune_type<dd>(G, G->tw_dd, a, b, st, tm);
  VD_CUDA(cudaStreamSynchronize(st));
  if (e == VD_OK) tune_save();
  return e;
}

int vd_autotune_table(int* out, int max) { return vd::tune_table(out, max); }

vd_status vd_autotune_set(int kind, int type, int n, int axis, int dir, int choice) {
  if (kind < 0 || kind > 1 || type < 0 || type > 2 || n <= 0) return vd::fail(VD_ERR_INVALID_ARG, "bad tuning key");
  if (choice != vd::kChoiceStaged && !(choice == vd::kChoiceUnpacked && type == 2) &&
      (choice > 64 || (choice > 0 && (choice & (choice - 1)))))
    return vd::fail(VD_ERR_INVALID_ARG, "bad choice");
  vd::tune_set(kind, type, n, axis, dir, choice);
  return VD_OK;
}

}  // extern "C"
