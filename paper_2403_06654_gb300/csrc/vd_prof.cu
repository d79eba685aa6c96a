// Launch counter and per-class event timing of the transform passes.
#include "vd_prof.h"
#include "vd_internal.h"
#include "vd_dd.cuh"

#include <algorithm>
#include <atomic>
#include <mutex>
#include <vector>

namespace vd {

static std::atomic<long long> g_launches{0};
static std::atomic<int> g_prof_on{0};

bool vd_profile_is_on() { return g_prof_on.load(std::memory_order_relaxed) != 0; }

struct Pending {
  int cls;
  cudaEvent_t a, b;
  double bytes, flops;
  cudaStream_t st;
  long long seq;
  bool dropped;
};
struct ClassTotals {
  long long launches = 0;
  double ms = 0.0, bytes = 0.0, flops = 0.0;
};

static std::mutex g_mu;
static std::vector<Pending> g_pending;
static std::vector<cudaEvent_t> g_free;
static ClassTotals g_tot[PC_N];
static long long g_seq = 0;   // sequence number of the next record

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

static cudaEvent_t get_event() {
  if (!g_free.empty()) {
    cudaEvent_t e = g_free.back();
    g_free.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

ProfScope::ProfScope(int c, cudaStream_t s, double by, double fl) : cls(c), st(s), bytes(by), flops(fl), slot(-1) {
  count_launch();
  const int mode = g_prof_on.load(std::memory_order_relaxed);
  if (!mode) return;
  std::lock_guard<std::mutex> lk(g_mu);
  Pending p;
  p.cls = c;
  p.a = nullptr;
  p.b = nullptr;
  p.bytes = by;
  p.flops = fl;
  p.st = s;
  p.seq = g_seq++;
  p.dropped = false;
  if (mode == 1) {
    p.a = get_event();
    p.b = get_event();
    cudaEventRecord(p.a, s);
  }
  g_pending.push_back(p);
  if (mode == 1) slot = (int)g_pending.size() - 1;
}

ProfSpan::ProfSpan(int c, cudaStream_t s) : cls(c), st(s), seq0(-1), a(nullptr) {
  if (g_prof_on.load(std::memory_order_relaxed) != 2) return;
  std::lock_guard<std::mutex> lk(g_mu);
  seq0 = g_seq;
  a = get_event();
  cudaEventRecord(a, s);
}

ProfSpan::~ProfSpan() {
  if (!a) return;
  std::lock_guard<std::mutex> lk(g_mu);
  Pending p;
  p.cls = cls;
  p.a = a;
  p.b = get_event();
  p.bytes = 0.0;
  p.flops = 0.0;
  for (const auto& q : g_pending)
    if (!q.a && q.seq >= seq0 && q.st == st && !q.dropped) {
      p.bytes += q.bytes;
      p.flops += q.flops;
    }
  p.st = st;
  p.seq = g_seq++;
  p.dropped = false;
  cudaEventRecord(p.b, st);
  g_pending.push_back(p);
}

ProfScope::~ProfScope() {
  if (slot < 0) return;
  std::lock_guard<std::mutex> lk(g_mu);
  cudaEventRecord(g_pending[slot].b, st);
}

static void collect_locked() {
  for (auto& p : g_pending) {
    if (!p.a) continue;   // span mode: a launch counted only inside its span
    cudaEventSynchronize(p.b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, p.a, p.b);
    if (!p.dropped) {
      ClassTotals& t = g_tot[p.cls];
      t.launches += 1;
      t.ms += ms;
      t.bytes += p.bytes;
      t.flops += p.flops;
    }
    g_free.push_back(p.a);
    g_free.push_back(p.b);
  }
  g_pending.clear();
}

long long prof_mark() {
  std::lock_guard<std::mutex> lk(g_mu);
  return g_seq;
}

void prof_discard(long long mark, cudaStream_t st) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto& p : g_pending)
    if (p.seq >= mark && p.st == st) p.dropped = true;
}

// ---------------------------------------------------------------------------------------
// arithmetic-rate microbenchmark (roofline denominators of the ALU-bound passes)
// ---------------------------------------------------------------------------------------

// written only when a chain ends on an impossible value, so that the chains stay live
static __device__ double g_alu_sink;

constexpr int kAluChains = 8;

// kAluChains independent chains a <- a * m + c per thread; values stay near 1 (m < 1, c small)
template <typename T>
__global__ void __launch_bounds__(256) k_alu_fma(int iters, T m, T c) {
  T a[kAluChains];
#pragma unroll
  for (int k = 0; k < kAluChains; ++k) a[k] = T(1) + T(threadIdx.x + k) * T(1e-3);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int k = 0; k < kAluChains; ++k) a[k] = fma(a[k], m, c);
  }
  T s = T(0);
#pragma unroll
  for (int k = 0; k < kAluChains; ++k) s += a[k];
  if (s == T(-1)) g_alu_sink = (double)s;
}

// the same chains in float-pair arithmetic (one float-pair multiply and one add per step)
__global__ void __launch_bounds__(256) k_alu_dd(int iters, float mh, float ml, float ch, float cl) {
  const dd m(mh, ml), c(ch, cl);
  dd a[kAluChains];
#pragma unroll
  for (int k = 0; k < kAluChains; ++k) a[k] = dd(1.0f + (float)(threadIdx.x + k) * 1e-3f, 0.0f);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int k = 0; k < kAluChains; ++k) a[k] = a[k] * m + c;
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < kAluChains; ++k) s += a[k].hi + a[k].lo;
  if (s == -1.0f) g_alu_sink = (double)s;
}

}  // namespace vd

using namespace vd;

extern "C" {

vd_status vd_alu_rate(int kind, double* flops_per_s, vd_stream stream) {
  if (kind < 0 || kind > 2 || !flops_per_s) return fail(VD_ERR_INVALID_ARG, "kind must be 0, 1 or 2");
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  VD_CUDA(cudaGetDevice(&dev));
  VD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = 8 * sms, threads = 256;
  // about 10-40 ms per launch on a GB300
  const int iters = (kind == 0) ? 512 : (kind == 1 ? 16384 : 2048);
  cudaEvent_t e0, e1;
  VD_CUDA(cudaEventCreate(&e0));
  VD_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {   // the first launch warms up
    VD_CUDA(cudaEventRecord(e0, st));
    if (kind == 0) k_alu_fma<double><<<blocks, threads, 0, st>>>(iters, 0.999999999, 1e-9);
    else if (kind == 1) k_alu_fma<float><<<blocks, threads, 0, st>>>(iters, 0.9999f, 1e-5f);
    else k_alu_dd<<<blocks, threads, 0, st>>>(iters, 0.9999f, 1e-12f, 1e-5f, 1e-13f);
    count_launch();
    VD_CUDA(cudaGetLastError());
    VD_CUDA(cudaEventRecord(e1, st));
    VD_CUDA(cudaEventSynchronize(e1));
    float ms = 0.0f;
    VD_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    if (rep > 0) best = std::min(best, ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const double steps = (double)blocks * threads * iters * 4.0 * kAluChains;
  *flops_per_s = 2.0 * steps / (best * 1e-3);
  return VD_OK;
}

long long vd_launch_count(void) { return g_launches.load(); }

vd_status vd_profile_enable(int on) {
  if (on < 0 || on > 2) return fail(VD_ERR_INVALID_ARG, "profile mode: 0 off, 1 every launch, 2 spans");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!on) collect_locked();
  g_prof_on.store(on);
  return VD_OK;
}

vd_status vd_profile_reset(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  collect_locked();
  for (auto& t : g_tot) t = ClassTotals();
  return VD_OK;
}

vd_status vd_profile_read(int cls, long long* launches, double* ms, double* alg_bytes, double* alg_flops) {
  if (cls < 0 || cls >= PC_N) return fail(VD_ERR_INVALID_ARG, "unknown profile class");
  std::lock_guard<std::mutex> lk(g_mu);
  collect_locked();
  const ClassTotals& t = g_tot[cls];
  if (launches) *launches = t.launches;
  if (ms) *ms = t.ms;
  if (alg_bytes) *alg_bytes = t.bytes;
  if (alg_flops) *alg_flops = t.flops;
  return VD_OK;
}

}  // extern "C"
