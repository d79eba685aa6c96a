// Krylov solvers in spectral space (device scalar state, host-driven iteration loop).
//
// The unknowns live in the half-spectrum representation: a real field is stored as its
// coefficients cpx[n2][n1][n0/2+1] (times ncomp components).  By Parseval the Euclidean
// inner product of two real fields is proportional to sum_k w(kx) Re(u_k conj(v_k)) with
// w = 1 on the kx = 0 and kx = n0/2 planes and w = 2 elsewhere, so CG, GMRES and RMR run on
// the spectral coefficients with that weighted inner product and produce the same iterates
// as on the physical grid.  The preconditioners are diagonal there (a symbol array).
#pragma once

#include "vd_internal.h"

namespace vd {

constexpr int kMaxRestart = 64;
constexpr int kRedBlocks = 608;   // fixed block count of every reduction (deterministic; 4 per SM on 152 SMs)
constexpr int kRedThreads = 256;
constexpr int kInnerGuard = 100;  // divergence guard of the inner float CG solves (see KState::guard)
constexpr int kStallWindow = 8;   // iterations without a halving of the residual that count as a stall

// device-resident scalar state of one solve
struct KState {
  double bb;       // ||b||^2
  double tol2bb;   // tol^2 ||b||^2
  double rr, rz, pq, alpha, beta, rw, ww;
  double best;     // best monitored relres so far
  double relres;
  int iters, maxit, status, done;
  int hist_cap;
  // GMRES (m, k, cycle_done); guard > 0 (the inner float CG solves of the refinement): past
  // its attainable accuracy a float CG stalls and then drifts away, so a guarded CG solve that
  // is below 1e-3 stops (status VD_ERR_DIVERGED, the refinement goes on) when its monitored
  // residual has not halved for kStallWindow iterations, or exceeds guard x its best value
  int m, k, cycle_done, guard;
  double beta0;
  double H[(kMaxRestart + 1) * kMaxRestart];   // column-major: H[i + j*(m+1)]
  double cs[kMaxRestart], sn[kMaxRestart], gv[kMaxRestart + 1], y[kMaxRestart];
  double h1[kMaxRestart + 1], h2[kMaxRestart + 1];
  double dtol;     // tolerance read by the epilogues when the launch passes a negative one
  double ref;      // guarded CG: residual at the last halving of the monitored residual ...
  int ref_it;      // ... and its iteration (stall test)
};

// device-resident state of an iterative-refinement loop recorded into a graph
struct OState {
  double bb, rr, rnorm, rel, tol, itol0, itol, scale;
  int total, outer, maxit, maxouter, done, status, force, pad;
};

struct KWork {
  KState* ks;
  double* partials;     // kRedBlocks * 8
  unsigned* counter;
  double* hist;         // hist_cap entries
};

// status codes stored in KState::status (mirror vd_status)
enum KStatus { KS_RUNNING = -1 };

struct Vec {
  void* p;        // cpx<T>*
  long long len;  // complex elements (ncomp * ncplx)
};

// Solve in spectral space.  Operator callbacks apply A (optionally right-preconditioned:
// with_sym = true means A S) on the stream.
struct SpecSystem {
  const vd_grid* G;
  int ncomp;
  long long len;            // ncomp * ncplx
  int h0;
  const void* sym;          // symbol array of the preconditioner (ncplx, type T)
  int is_float;             // vectors and transforms in float
  void (*apply)(const SpecSystem& sys, const void* in, void* out, bool with_sym, const int* done, cudaStream_t st);
  void* ctx[4];             // opaque per-operator data (rinv, tmp, params)
  double a, inv_sc;
};

struct SolveOpts {
  int solver;  // vd_solver
  double tol;
  int maxit;
  int restart;
  int check_every;
  int x_zero;   // x is known to be zero on entry: the first residual is b (no operator apply)
  int guard = 0;   // KState::guard of the solve
  const OState* dev_outer = nullptr;   // graph form: tolerance and iteration budget from the device
};

struct SolveOut {
  int iters;
  int status;
  double relres;
};

// x (in/out), b: spectral vectors of sys.len complex elements of type T.
// Workspace vectors: CG needs r,p,q (3 len); RMR r,w (2 len); GMRES V ((m+1) len) + w.
template <typename T>
vd_status krylov_solve(const SpecSystem& sys, const SolveOpts& o, const void* b, void* x, void* vecs,
                       const KWork& kw, double* host_hist, int host_hist_cap, SolveOut* out, cudaStream_t st);

template <typename T>
size_t krylov_vec_bytes(const SpecSystem& sys, int solver, int restart);

// The same solve as a capturable graph fragment: `st` must be capturing; the iteration loop
// becomes a conditional WHILE node (its body captured on body_st).  No host synchronisation:
// the result stays in the KState (iters, status, relres, done).
template <typename T>
vd_status krylov_enqueue_graph(const SpecSystem& sys, const SolveOpts& o, const void* b, void* x, void* vecs,
                               const KWork& kw, cudaStream_t st, cudaStream_t body_st);
// Iterative refinement as a graph fragment (see vd_krylov.cu): x += |r| d with the inner
// float solve A32 d = r/|r| and r = b - A x from `resid` (double or float-pair operator).
// bh, xh, rh: double spectral vectors (bh holds the projected rhs; xh is zeroed here);
// bh_f, xh_f, vecs: float inner vectors.  Streams: st capturing, s1..s3 for the bodies.
vd_status refine_enqueue_graph(const SpecSystem& sys64, const SpecSystem& sys32,
                               void (*resid)(const void* ctx, const void* x, void* y, cudaStream_t st),
                               const void* resid_ctx, const SolveOpts& inner, double tol, double itol0, int maxit,
                               void* bh, void* xh, void* rh, void* bh_f, void* xh_f, void* vecs, const KWork& kw,
                               OState* ost, double* info, cudaStream_t st, cudaStream_t s1, cudaStream_t s2,
                               cudaStream_t s3);

// After a graph solve: true residual of x and the result record info[0..4] (iterations,
// status, monitored relres, |b|^2, true relres), all on the device.  vecs: scratch.
template <typename T>
vd_status krylov_graph_finish(const SpecSystem& sys, const void* b, const void* x, void* vecs, const KWork& kw,
                              double* info, cudaStream_t st);

// helpers shared with the API layer
template <typename T>
void spec_copy_scale(long long len, const void* x, double s, void* y, cudaStream_t st);   // y = s x
template <typename T>
void spec_axpy(long long len, double a, const void* x, void* y, cudaStream_t st);         // y += a x
template <typename T>
void spec_sub(long long len, const void* b, const void* q, void* r, cudaStream_t st);     // r = b - q
// weighted norm^2 of a spectral vector -> host (synchronises)
template <typename T>
double spec_norm2_host(const SpecSystem& sys, const void* v, const KWork& kw, cudaStream_t st);
// weighted inner product (a, b) of two spectral vectors, returned to the host
template <typename T>
double spec_dot_host(const SpecSystem& sys, const void* a, const void* b, const KWork& kw, cudaStream_t st);
// zero the 2^d null-space coefficients of each component; removed (device, may be null,
// 2^d ncomp doubles) receives each removed coefficient's share of the squared weighted norm
template <typename T>
void spec_project(const vd_grid* G, int ncomp, void* v, cudaStream_t st, double* removed = nullptr);
// refinement steps on double vectors, each one pass: out = float(in * s) (narrowed right-hand
// side of the inner solve); y += a * double(xf) (correction); r = b - q returning |r|^2
// (weighted) to the host
void spec_d2f_scaled(long long len, const void* in, double s, void* out, cudaStream_t st);
void spec_axpy_f2d(long long len, double a, const void* xf, void* y, cudaStream_t st);
double spec_sub_norm2_host(const SpecSystem& sys, const void* b, const void* q, void* r, const KWork& kw,
                           cudaStream_t st);

}  // namespace vd
