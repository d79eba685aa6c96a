// Request server: continuous batching of variable-density solves on one GPU.
//
// Requests (grid, density, right-hand side, tolerance, solver) arrive at any time through
// vd_server_submit and wait in a FIFO queue.  A request is admitted as soon as an execution
// slot (worker) is idle and its device memory (density data + solve workspace, from the
// library's own workspace queries) fits in the server's HBM budget; admitted requests run
// concurrently, each on its worker's own non-blocking CUDA stream, so their kernels overlap
// on the device.  Krylov state lives in the request's device workspace for the whole solve.
// Memory is taken from the stream-ordered allocator of the worker's stream and returned when
// the request completes, which admits the next ones.  A request without an output buffer gets
// its solution in server memory that stays reserved until the caller fetches or releases it.
// Completions carry submit / start / done timestamps (host steady clock, seconds) for latency
// statistics.
//
// Every solve is deterministic (fixed launch shapes, fixed-order reductions) and never shares
// device data with another request, so a request's result does not depend on the mix it ran in.
#include "vd_internal.h"

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <tuple>
#include <vector>

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Job {
  vd_request r;
  double t_submit;
  size_t bytes;   // device bytes needed (density + workspace, plus a server-owned solution)
};

struct Owned {    // server-owned solution of a completed request
  void* p;
  size_t bytes;   // bytes it keeps reserved in the budget
  size_t size;    // bytes of the solution (n0 n1 n2 doubles)
};

size_t solution_size(const vd_request& r) {
  const long long n = (long long)r.n[0] * (r.ndim > 1 ? r.n[1] : 1) * (r.ndim > 2 ? r.n[2] : 1);
  return (size_t)n * sizeof(double);
}
size_t out_bytes(const vd_request& r) { return (solution_size(r) + 255) & ~(size_t)255; }

struct GridKey {
  int ndim, n0, n1, n2;
  double L0, L1, L2;
  bool operator<(const GridKey& o) const {
    return std::tie(ndim, n0, n1, n2, L0, L1, L2) < std::tie(o.ndim, o.n0, o.n1, o.n2, o.L0, o.L1, o.L2);
  }
};

}  // namespace

struct vd_server {
  vd_server_params p;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_work;   // workers wait for admitted jobs
  std::condition_variable cv_done;   // drain waits for completions
  std::deque<Job> queue;             // submitted, not admitted
  std::deque<Job> ready;             // admitted, waiting for a worker
  std::vector<vd_completion> done;   // completed, not yet polled
  std::map<unsigned long long, Owned> owned;   // server-owned solutions, by request id
  cudaStream_t aux = nullptr;        // stream of fetch copies and releases
  size_t reserved = 0;               // bytes held by admitted jobs and unreleased solutions
  size_t budget = 0;
  int idle = 0;                      // idle workers
  long long inflight = 0;            // admitted + running
  long long submitted = 0, completed = 0, cancelled = 0;
  bool stop = false;
  std::vector<std::thread> workers;

  // admit queued jobs while a worker is idle and memory fits (called with mu held)
  void admit_locked() {
    while (!queue.empty() && (long long)ready.size() < idle) {
      Job& j = queue.front();
      if (reserved + j.bytes > budget && reserved > 0) break;   // wait for memory (FIFO)
      reserved += j.bytes;
      ++inflight;
      ready.push_back(j);
      queue.pop_front();
      cv_work.notify_one();
    }
  }

  void worker_main() {
    cudaSetDevice(device);
    cudaStream_t st;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    std::map<GridKey, vd_grid*> grids;   // per-worker cache: grids carry per-request density
    for (;;) {
      Job j;
      {
        std::unique_lock<std::mutex> lk(mu);
        ++idle;
        admit_locked();
        cv_work.wait(lk, [&] { return stop || !ready.empty(); });
        --idle;
        if (ready.empty()) break;   // stop requested
        j = ready.front();
        ready.pop_front();
      }
      vd_completion c{};
      c.id = j.r.id;
      c.t_submit = j.t_submit;
      c.t_start = now_s();
      void* xo = nullptr;
      c.status = run(j, st, grids, &c, &xo);
      c.t_done = now_s();
      {
        std::lock_guard<std::mutex> lk(mu);
        size_t keep = 0;
        if (xo) {   // the solution stays reserved until the caller fetches or releases it
          keep = std::min(out_bytes(j.r), j.bytes);
          owned[j.r.id] = Owned{xo, keep, solution_size(j.r)};
        }
        reserved -= j.bytes - keep;
        --inflight;
        ++completed;
        done.push_back(c);
        admit_locked();
      }
      cv_done.notify_all();
    }
    for (auto& kv : grids) vd_grid_destroy(kv.second);
    cudaStreamDestroy(st);
  }

  int run(const Job& j, cudaStream_t st, std::map<GridKey, vd_grid*>& grids, vd_completion* c, void** xo) {
    const vd_request& r = j.r;
    GridKey key{r.ndim, r.n[0], r.ndim > 1 ? r.n[1] : 1, r.ndim > 2 ? r.n[2] : 1,
                r.L[0], r.ndim > 1 ? r.L[1] : 1.0, r.ndim > 2 ? r.L[2] : 1.0};
    vd_grid* G = nullptr;
    auto it = grids.find(key);
    if (it != grids.end()) {
      G = it->second;
    } else {
      vd_status e = vd_grid_create(r.ndim, r.n, r.L, &G);
      if (e != VD_OK) return e;
      grids[key] = G;
    }
    const size_t db = vd_density_bytes(G, VD_OP_PRESSURE);
    vd_solve_params sp = request_params(r);
    const size_t wb = vd_workspace_bytes(G, VD_OP_PRESSURE, (vd_solver)r.solver, &sp);
    double* x = r.x;
    if (!x) {
      if (cudaMallocAsync(xo, out_bytes(r), st) != cudaSuccess) {
        *xo = nullptr;
        cudaGetLastError();
        return VD_ERR_OOM;
      }
      x = static_cast<double*>(*xo);
    }
    c->x = x;
    void* mem = nullptr;
    if (cudaMallocAsync(&mem, db + wb + 256, st) != cudaSuccess) {
      cudaGetLastError();
      return VD_ERR_OOM;
    }
    char* base = static_cast<char*>(mem);
    vd_status e = vd_density_set(G, VD_OP_PRESSURE, r.rho, base, db, st);
    vd_solve_info info{};
    if (e == VD_OK)
      e = vd_solve(G, VD_OP_PRESSURE, (vd_solver)r.solver, nullptr, &sp, r.b, x, &info,
                   base + ((db + 255) & ~(size_t)255), wb, st);
    cudaFreeAsync(mem, st);
    cudaStreamSynchronize(st);
    c->iters = info.iters;
    c->relres_true = info.relres_true;
    return e;
  }

  // remove a server-owned solution (mu held); optionally copy it out first
  vd_status take_owned(unsigned long long id, double* dst, cudaStream_t st) {
    auto it = owned.find(id);
    if (it == owned.end()) return vd::fail(VD_ERR_INVALID_ARG, "no server-owned solution with this id");
    cudaStream_t fs = aux;
    if (dst) {   // the copy and the free are ordered on the caller's stream
      if (cudaMemcpyAsync(dst, it->second.p, it->second.size, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return vd::fail(VD_ERR_CUDA, "copy of the solution failed");
      fs = st;
    }
    cudaFreeAsync(it->second.p, fs);
    reserved -= it->second.bytes;
    owned.erase(it);
    admit_locked();
    return VD_OK;
  }

  static vd_solve_params request_params(const vd_request& r) {
    vd_solve_params sp{};
    sp.tol = r.tol;
    sp.max_it = r.max_it > 0 ? r.max_it : 500;
    sp.restart = r.restart > 0 ? r.restart : 30;
    sp.use_x0 = 0;
    sp.precision = r.precision;
    sp.inner_tol = 0.0;   // automatic
    sp.check_every = 1;
    return sp;
  }
};

extern "C" {

vd_status vd_server_create(const vd_server_params* p, vd_server** out) {
  if (!p || !out) return vd::fail(VD_ERR_INVALID_ARG, "null argument");
  if (p->max_inflight < 1 || p->max_inflight > 64) return vd::fail(VD_ERR_INVALID_ARG, "max_inflight in [1, 64]");
  vd_server* S = new vd_server();
  S->p = *p;
  cudaGetDevice(&S->device);
  size_t fr = 0, tot = 0;
  cudaMemGetInfo(&fr, &tot);
  S->budget = p->hbm_budget ? p->hbm_budget : (size_t)(0.8 * (double)fr);
  // keep freed request memory in the device pool (no return to the driver between requests)
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, S->device) == cudaSuccess) {
    unsigned long long thr = ~0ull;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  cudaStreamCreateWithFlags(&S->aux, cudaStreamNonBlocking);
  for (int i = 0; i < p->max_inflight; ++i) S->workers.emplace_back([S] { S->worker_main(); });
  *out = S;
  return VD_OK;
}

size_t vd_server_request_bytes(const vd_request* r) {
  if (!r) return 0;
  vd_grid G;   // host-only description: no device memory is touched
  if (!vd::grid_desc_only(r->ndim, r->n, r->L, &G)) return 0;
  vd_solve_params sp = vd_server::request_params(*r);
  return vd_density_bytes(&G, VD_OP_PRESSURE) + vd_workspace_bytes(&G, VD_OP_PRESSURE, (vd_solver)r->solver, &sp) +
         512 + (r->x ? 0 : out_bytes(*r));
}

vd_status vd_server_submit(vd_server* S, const vd_request* r, size_t bytes) {
  if (!S || !r || !r->rho || !r->b) return vd::fail(VD_ERR_INVALID_ARG, "null argument");
  if (r->solver < 0 || r->solver > 2) return vd::fail(VD_ERR_INVALID_ARG, "unknown solver");
  if (bytes == 0) return vd::fail(VD_ERR_INVALID_ARG, "request size unknown (use vd_server_request_bytes)");
  std::lock_guard<std::mutex> lk(S->mu);
  if (bytes > S->budget) return vd::fail(VD_ERR_OOM, "request larger than the server's HBM budget");
  S->queue.push_back(Job{*r, now_s(), bytes});
  ++S->submitted;
  S->admit_locked();
  return VD_OK;
}

vd_status vd_server_cancel(vd_server* S, unsigned long long id) {
  if (!S) return vd::fail(VD_ERR_INVALID_ARG, "null server");
  std::lock_guard<std::mutex> lk(S->mu);
  for (auto it = S->queue.begin(); it != S->queue.end(); ++it) {
    if (it->r.id == id) {
      S->queue.erase(it);
      ++S->cancelled;
      S->admit_locked();
      S->cv_done.notify_all();
      return VD_OK;
    }
  }
  return vd::fail(VD_ERR_INVALID_ARG, "no queued request with this id");
}

int vd_server_poll(vd_server* S, vd_completion* out, int max) {
  if (!S || !out || max <= 0) return 0;
  std::lock_guard<std::mutex> lk(S->mu);
  const int n = (int)std::min<size_t>(S->done.size(), (size_t)max);
  for (int i = 0; i < n; ++i) out[i] = S->done[i];
  S->done.erase(S->done.begin(), S->done.begin() + n);
  return n;
}

vd_status vd_server_fetch(vd_server* S, unsigned long long id, double* dst, vd_stream stream) {
  if (!S || !dst) return vd::fail(VD_ERR_INVALID_ARG, "null argument");
  std::lock_guard<std::mutex> lk(S->mu);
  return S->take_owned(id, dst, (cudaStream_t)stream);
}

vd_status vd_server_release(vd_server* S, unsigned long long id) {
  if (!S) return vd::fail(VD_ERR_INVALID_ARG, "null server");
  std::lock_guard<std::mutex> lk(S->mu);
  return S->take_owned(id, nullptr, nullptr);
}

vd_status vd_server_drain(vd_server* S) {
  if (!S) return vd::fail(VD_ERR_INVALID_ARG, "null server");
  std::unique_lock<std::mutex> lk(S->mu);
  S->cv_done.wait(lk, [&] { return S->completed + S->cancelled == S->submitted; });
  return VD_OK;
}

vd_status vd_server_stats(vd_server* S, long long* submitted, long long* completed, long long* inflight,
                          size_t* reserved, size_t* budget) {
  if (!S) return vd::fail(VD_ERR_INVALID_ARG, "null server");
  std::lock_guard<std::mutex> lk(S->mu);
  if (submitted) *submitted = S->submitted;
  if (completed) *completed = S->completed;
  if (inflight) *inflight = S->inflight;
  if (reserved) *reserved = S->reserved;
  if (budget) *budget = S->budget;
  return VD_OK;
}

vd_status vd_server_destroy(vd_server* S) {
  if (!S) return VD_OK;
  {
    std::unique_lock<std::mutex> lk(S->mu);
    S->cv_done.wait(lk, [&] { return S->completed + S->cancelled == S->submitted; });
    S->stop = true;
  }
  S->cv_work.notify_all();
  for (auto& t : S->workers) t.join();
  for (auto& kv : S->owned) cudaFreeAsync(kv.second.p, S->aux);
  cudaStreamSynchronize(S->aux);
  cudaStreamDestroy(S->aux);
  delete S;
  return VD_OK;
}

}  // extern "C"
