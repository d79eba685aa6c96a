// Batched solves of many uneven instances in one graph launch.
//
// vd_batch_create sets every instance's density, lays out every workspace in one caller
// buffer and records all solves into one CUDA graph.  Each instance is a branch of its own
// (forked from the capturing stream and joined at the end), so independent instances run
// concurrently; each solve in it is a conditional WHILE node whose body is one Krylov
// iteration (one restart cycle for GMRES) and whose condition is set on the device from the
// convergence flag.  vd_batch_run is one cudaGraphLaunch: no host synchronisation and no
// per-iteration launches from the host.  Results (iterations, status, residuals) are written
// to a device record per solve and read by vd_batch_info.
#include "vd_internal.h"
#include "vd_prof.h"

#include <algorithm>
#include <vector>

namespace {

struct Item {
  vd_batch_item in;
  vd_grid* G = nullptr;
  void* dens = nullptr;
  size_t dens_bytes = 0;
  void* ws_vel = nullptr;
  size_t ws_vel_bytes = 0;
  void* ws_pres = nullptr;
  size_t ws_pres_bytes = 0;
};

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

vd_solve_params solve_params(const vd_batch_params& p) {
  vd_solve_params s{};
  s.tol = p.tol;
  s.max_it = p.max_it;
  s.restart = p.restart > 0 ? p.restart : 30;
  s.precision = p.precision;
  return s;
}

// sizes of one item on a host-only grid description
bool item_sizes(const vd_batch_item& it, const vd_batch_params& p, size_t* dens, size_t* wv, size_t* wp) {
  vd_grid G;
  if (!vd::grid_desc_only(it.ndim, it.n, it.L, &G)) return false;
  const vd_op dop = it.b_vel ? VD_OP_VELOCITY : VD_OP_PRESSURE;
  const vd_solve_params sp = solve_params(p);
  *dens = a256(vd_density_bytes(&G, dop));
  *wv = it.b_vel ? a256(vd_workspace_bytes(&G, VD_OP_VELOCITY, (vd_solver)p.vel_solver, &sp)) : 0;
  *wp = it.b_pres ? a256(vd_workspace_bytes(&G, VD_OP_PRESSURE, (vd_solver)p.pres_solver, &sp)) : 0;
  return true;
}

constexpr int kInfo = 8;   // doubles per solve record

}  // namespace

struct vd_batch {
  std::vector<Item> items;
  vd_batch_params p{};
  double* info = nullptr;   // device: count x 2 records
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  size_t nodes = 0;
};

extern "C" {

size_t vd_batch_bytes(const vd_batch_item* items, int count, const vd_batch_params* params) {
  if (!items || !params || count <= 0) return 0;
  size_t total = a256((size_t)count * 2 * kInfo * sizeof(double));
  for (int i = 0; i < count; ++i) {
    size_t d, wv, wp;
    if (!item_sizes(items[i], *params, &d, &wv, &wp)) return 0;
    total += d + wv + wp;
  }
  return total;
}

vd_status vd_batch_create(const vd_batch_item* items, int count, const vd_batch_params* params, void* mem,
                          size_t bytes, vd_stream stream, vd_batch** out) {
  using namespace vd;
  if (!items || !params || !mem || !out || count <= 0) return fail(VD_ERR_INVALID_ARG, "null argument or empty batch");
  if (params->vel_solver == VD_SOLVER_CG) return fail(VD_ERR_INVALID_ARG, "V_rho is not symmetric: no CG");
  if (params->vel_solver < 0 || params->vel_solver > 2 || params->pres_solver < 0 || params->pres_solver > 2)
    return fail(VD_ERR_INVALID_ARG, "unknown solver");
  if (!(params->tol >= 0.0) || params->max_it < 0) return fail(VD_ERR_INVALID_ARG, "tol >= 0 and max_it >= 0");
  if (params->precision != VD_PREC_FP64 && params->precision != VD_PREC_MIXED && params->precision != VD_PREC_MIXED_DD)
    return fail(VD_ERR_INVALID_ARG, "unknown precision mode");
  if (vd_profile_is_on()) return fail(VD_ERR_INVALID_ARG, "disable the profiler while recording a batch");
  const size_t need = vd_batch_bytes(items, count, params);
  if (need == 0) return fail(VD_ERR_INVALID_ARG, "unsupported grid in the batch");
  if (bytes < need) return fail(VD_ERR_OOM, "batch memory smaller than vd_batch_bytes");
  cudaStream_t st = (cudaStream_t)stream;
  vd_batch* B = new vd_batch();
  B->p = *params;
  char* cur = static_cast<char*>(mem);
  B->info = reinterpret_cast<double*>(cur);
  cur += a256((size_t)count * 2 * kInfo * sizeof(double));
  auto cleanup = [&](vd_status e) {
    for (auto& it : B->items)
      if (it.G) vd_grid_destroy(it.G);
    delete B;
    return e;
  };
  // grids, densities, workspaces (outside the graph: densities are fixed for the batch)
  for (int i = 0; i < count; ++i) {
    Item it;
    it.in = items[i];
    if (!it.in.rho || (!it.in.b_vel && !it.in.b_pres) || (it.in.b_vel && !it.in.x_vel) ||
        (it.in.b_pres && !it.in.x_pres))
      return cleanup(fail(VD_ERR_INVALID_ARG, "item needs rho and at least one complete (b, x) pair"));
    size_t d, wv, wp;
    item_sizes(it.in, *params, &d, &wv, &wp);
    vd_status e = vd_grid_create(it.in.ndim, it.in.n, it.in.L, &it.G);
    if (e != VD_OK) return cleanup(e);
    it.dens = cur;
    it.dens_bytes = d;
    cur += d;
    it.ws_vel = wv ? cur : nullptr;
    it.ws_vel_bytes = wv;
    cur += wv;
    it.ws_pres = wp ? cur : nullptr;
    it.ws_pres_bytes = wp;
    cur += wp;
    B->items.push_back(it);
    e = vd_density_set(B->items.back().G, it.in.b_vel ? VD_OP_VELOCITY : VD_OP_PRESSURE, it.in.rho, it.dens, d,
                       stream);
    if (e != VD_OK) return cleanup(e);
  }
  VD_CUDA(cudaMemsetAsync(B->info, 0, (size_t)count * 2 * kInfo * sizeof(double), st));
  VD_CUDA(cudaStreamSynchronize(st));

  // record: fork one branch per item from the capturing stream, join them at the end
  cudaStream_t body[3] = {nullptr, nullptr, nullptr};
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> joins(2 * count, nullptr);
  std::vector<cudaStream_t> branches(2 * count, nullptr);   // one capture stream per system
  for (auto& s : branches) VD_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  for (auto& b : body) VD_CUDA(cudaStreamCreateWithFlags(&b, cudaStreamNonBlocking));
  VD_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
  for (auto& j : joins) VD_CUDA(cudaEventCreateWithFlags(&j, cudaEventDisableTiming));
  vd_status err = VD_OK;
  cudaStream_t cap = nullptr;
  VD_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
  VD_CUDA(cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed));
  VD_CUDA(cudaEventRecord(fork, cap));
  const vd_solve_params sp = solve_params(*params);
  for (int k = 0; k < 2 * count && err == VD_OK; ++k) {
    const int i = k / 2;
    const bool vel = (k % 2) == 0;
    Item& it = B->items[i];
    if (vel ? !it.in.b_vel : !it.in.b_pres) continue;
    cudaStream_t branch = branches[k];
    // the branch joins the capture through the fork event; its work is recorded in order
    if (cudaStreamWaitEvent(branch, fork, 0) != cudaSuccess) {
      err = fail(VD_ERR_CUDA, "fork of a batch branch failed");
      break;
    }
    double* rec = B->info + (size_t)i * 2 * kInfo;
    if (vel) {
      vd_op_params op{it.in.a, it.in.inv_sc};
      err = enqueue_solve_graph(it.G, VD_OP_VELOCITY, (vd_solver)params->vel_solver, &op, params->tol, sp.max_it,
                                sp.restart, sp.precision, it.in.b_vel, it.in.x_vel, it.ws_vel, it.ws_vel_bytes, rec,
                                branch, body);
    } else {
      err = enqueue_solve_graph(it.G, VD_OP_PRESSURE, (vd_solver)params->pres_solver, nullptr, params->tol, sp.max_it,
                                sp.restart, sp.precision, it.in.b_pres, it.in.x_pres, it.ws_pres, it.ws_pres_bytes,
                                rec + kInfo, branch, body);
    }
    if (err == VD_OK && cudaEventRecord(joins[k], branch) != cudaSuccess) err = fail(VD_ERR_CUDA, "join record");
    if (err == VD_OK && cudaStreamWaitEvent(cap, joins[k], 0) != cudaSuccess) err = fail(VD_ERR_CUDA, "join wait");
  }
  cudaGraph_t g = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(cap, &g);
  if (err == VD_OK && ce != cudaSuccess) err = cuda_fail(ce, "cudaStreamEndCapture");
  if (err == VD_OK) {
    const cudaError_t ie = cudaGraphInstantiate(&B->exec, g, 0);
    if (ie != cudaSuccess) err = cuda_fail(ie, "cudaGraphInstantiate");
  }
  if (err == VD_OK) {
    B->graph = g;
    cudaGraphGetNodes(g, nullptr, &B->nodes);
  } else if (g) {
    cudaGraphDestroy(g);
  }
  cudaStreamDestroy(cap);
  for (auto& s : branches) cudaStreamDestroy(s);
  for (auto& b : body) cudaStreamDestroy(b);
  cudaEventDestroy(fork);
  for (auto& j : joins) cudaEventDestroy(j);
  if (err != VD_OK) return cleanup(err);
  *out = B;
  return VD_OK;
}

vd_status vd_batch_run(vd_batch* B, vd_stream stream) {
  if (!B || !B->exec) return vd::fail(VD_ERR_INVALID_ARG, "null batch");
  VD_CUDA(cudaGraphLaunch(B->exec, (cudaStream_t)stream));
  return VD_OK;
}

vd_status vd_batch_info(vd_batch* B, int index, vd_solve_info* vel, vd_solve_info* pres) {
  if (!B || index < 0 || index >= (int)B->items.size()) return vd::fail(VD_ERR_INVALID_ARG, "bad batch index");
  double rec[2 * kInfo];
  // the graph may run on a non-blocking stream, which a legacy-stream copy does not wait for
  VD_CUDA(cudaDeviceSynchronize());
  VD_CUDA(cudaMemcpy(rec, B->info + (size_t)index * 2 * kInfo, sizeof rec, cudaMemcpyDeviceToHost));
  auto fill = [](const double* r, vd_solve_info* o) {
    if (!o) return;
    o->iters = (int)r[0];
    o->outer_iters = 0;
    o->status = (int)r[1];
    o->relres = r[2];
    o->relres_true = r[4];
    o->outer_iters = (int)r[5];
    o->hist_len = 0;
  };
  if (B->items[index].in.b_vel) fill(rec, vel);
  if (B->items[index].in.b_pres) fill(rec + kInfo, pres);
  return VD_OK;
}

size_t vd_batch_graph_nodes(const vd_batch* B) { return B ? B->nodes : 0; }

vd_status vd_batch_destroy(vd_batch* B) {
  if (!B) return VD_OK;
  if (B->exec) cudaGraphExecDestroy(B->exec);
  if (B->graph) cudaGraphDestroy(B->graph);
  for (auto& it : B->items)
    if (it.G) vd_grid_destroy(it.G);
  delete B;
  return VD_OK;
}

}  // extern "C"
