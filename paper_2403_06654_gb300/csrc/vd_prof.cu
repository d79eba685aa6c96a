// Launch counter and per-class event timing of the transform passes.
#include "vd_prof.h"
#include "vd_internal.h"

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

}  // namespace vd

using namespace vd;

extern "C" {

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
