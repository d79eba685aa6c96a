// Internal host-side structures of the library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "vd.h"
#include "vd_common.cuh"
#include "vd_passes.cuh"

struct vd_grid {
  vd::GridDesc g;
  double L[3];
  void* tw_d = nullptr;   // cpx<double> twiddle table (library-owned)
  void* tw_f = nullptr;   // cpx<float> copy
  void* tw_dd = nullptr;  // cpx<dd> copy (float-pair split of the extended-precision values)
  // density data (inside the caller's density workspace; set by vd_density_set)
  const double* rinv_s = nullptr;    // 1/(N rho), physical
  const float* rinv_s_f = nullptr;   // same, float
  const void* rinv_s_dd = nullptr;   // same, float-pair (dd per point)
  const double* grho[3] = {nullptr, nullptr, nullptr};     // D_j rho
  const double* hrho[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};  // D_i D_j rho (i<=j)
  const double* rho = nullptr;       // copy of rho
  // K_rho data (set by vd_density_set with VD_OP_KRHO): c/N with c = -Lap(w)/w, w = rho^-1/2,
  // and the spectrum of w normalised to unit Parseval norm
  const double* kc_s = nullptr;
  const float* kc_f = nullptr;
  const void* kc_dd = nullptr;
  const void* kw_hat = nullptr;      // cpx<double>, ncplx
  double rho_min = 0, rho_max = 0;
  int has_density = 0;
  int has_velocity_data = 0;
  int has_krho_data = 0;
};

namespace vd {

// fill the grid description (plans, sizes) of a stack/host vd_grid without device memory;
// enough for the size queries (vd_density_bytes, vd_workspace_bytes)
bool grid_desc_only(int ndim, const int n[3], const double L[3], vd_grid* G);

// set the thread-local error message and return the status
vd_status fail(vd_status st, const std::string& msg);
vd_status cuda_fail(cudaError_t e, const char* what);

#define VD_CUDA(call)                                   \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return vd::cuda_fail(e_, #call); \
  } while (0)

// index of the symmetric second-derivative pair (i <= j) in hrho[]
inline int hidx(int i, int j) {
  if (i > j) {
    int t = i;
    i = j;
    j = t;
  }
  static const int tab[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
  return tab[i][j];
}

// ------------------------------------------------------------------------------------
// generic transforms (vd_ops.cu).  Spectral fields hold g.ncplx elements, physical ones
// g.nreal.  deriv[j] in {0,1,2}: multiply by (i k~_j)^deriv[j]; sym/negk2 as MulFlags.
// ------------------------------------------------------------------------------------

struct Mult {
  int deriv[3] = {0, 0, 0};
  int sym = 0;          // multiply by symbol array
  int negk2 = 0;        // multiply by -|k~|^2
  const void* symarr = nullptr;
  double scale = 1.0;
};

// physical (T, nreal) -> spectral (cpx<T>, ncplx).  tmp: one spectral field.
template <typename T>
void fwd_transform(const vd_grid* G, const T* in, cpx<T>* out, cudaStream_t st);
// spectral -> physical with multiplier. tmp: one spectral field (2D/3D); `in` untouched.
template <typename T>
void inv_transform(const vd_grid* G, const cpx<T>* in, const Mult& m, T* out, cpx<T>* tmp, cudaStream_t st);
// the plain transforms of ncomp (<= 3) fields stored back to back, one launch per pass (each
// field's arithmetic as in fwd_transform / inv_transform; the inverse needs ncomp spectral tmp
// fields in 2D/3D)
template <typename T>
void fwd_transform_n(const vd_grid* G, int ncomp, const T* in, cpx<T>* out, cudaStream_t st);
template <typename T>
void inv_transform_n(const vd_grid* G, int ncomp, const cpx<T>* in, T* out, cpx<T>* tmp, cudaStream_t st);

// Pressure operator in spectral space: out = L~ (S in) with S = symarr (if non-null) else 1.
// tmp: 3 spectral fields (3D), 2 (2D), 0 (1D).  done: optional early-exit flag.
// wf_pair (float only, may be null): 1/(N rho) as float pairs, multiplied in float-pair
// arithmetic instead of rinv_s (the inner operator of mixed solves at high density ratios).
template <typename T>
void apply_pressure_spec(const vd_grid* G, const cpx<T>* in, cpx<T>* out, const T* symarr, const T* rinv_s,
                         cpx<T>* tmp, const int* done, cudaStream_t st, const void* wf_pair = nullptr);

// Pressure operator with float-pair transforms: double spectral fields in and out (no
// preconditioner), float-pair intermediates in tmp (3 spectral fields of 16 bytes per element).
// phys_out (may be null): also the inverse transform of `in` (real, n2 x n1 x n0 doubles),
// written by the fused x pass and equal bit for bit to inv_transform_dd of `in`
void apply_pressure_spec_dd(const vd_grid* G, const cpx<double>* in, cpx<double>* out, void* tmp, const int* done,
                            cudaStream_t st, double* phys_out = nullptr);

// Plain forward / inverse transforms with float-pair arithmetic (double fields in and out;
// tmp: one spectral field of 16-byte elements).
void fwd_transform_dd(const vd_grid* G, const double* in, cpx<double>* out, void* tmp, cudaStream_t st);
void inv_transform_dd(const vd_grid* G, const cpx<double>* in, double* out, void* tmp, cudaStream_t st);

// Velocity operator in spectral space: out_i = (S in)_i - a * F[rho^-1 (Lap u + Sc^-1 (...))]_i with u =
// F^-1 (S in).  ncomp = ndim components stored back to back.  tmp: see velocity_tmp_fields().
template <typename T>
void apply_velocity_spec(const vd_grid* G, const cpx<T>* in, cpx<T>* out, const T* symarr, double a,
                         double inv_sc, cpx<T>* tmp, const int* done, cudaStream_t st);
// the same without preconditioner in float-pair arithmetic, double fields in and out
void apply_velocity_spec_dd(const vd_grid* G, const cpx<double>* in, cpx<double>* out, double a, double inv_sc,
                            void* tmp, const int* done, cudaStream_t st);
int velocity_tmp_fields(int ndim);   // spectral-field-sized temporaries
int velocity_spec_tmps(int ndim);    // of which spectral scratch (the rest hold physical fields)
// grad[j] = F^-1(i k_j rh), hess[hidx(a, b)] = F^-1((i k_a)(i k_b) rh) in double; tmp: 3 spectral fields
void derivative_fields(const vd_grid* G, const cpx<double>* rh, double* const grad[3], double* const hess[6],
                       cpx<double>* tmp, cudaStream_t st);
int pressure_tmp_fields(int ndim);

// K_rho operator in spectral space: out = K~ (S in) = Lap S in + F(c F^-1(S in)); with S the
// pseudo-inverse of Lap (symarr non-null) the local term is the mean-free part of `in`.
// coef_s: c/N (physical, type T).  tmp: one spectral field (2D/3D), none (1D).
template <typename T>
void apply_krho_spec(const vd_grid* G, const cpx<T>* in, cpx<T>* out, const T* symarr, const T* coef_s,
                     cpx<T>* tmp, const int* done, cudaStream_t st, const void* wf_pair = nullptr);
// the same with float-pair transforms: double spectral fields in and out, no preconditioner
void apply_krho_spec_dd(const vd_grid* G, const cpx<double>* in, cpx<double>* out, void* tmp, const int* done,
                        cudaStream_t st);
int krho_tmp_fields(int ndim);

// symbol arrays (real, ncplx): pressure -1/|k~|^2 (0 on corners), velocity 1/(1+a|k~|^2),
// projection 1 / 0 on corners, K_rho preconditioner -1/|k|^2 (full k, 0 for the mean),
// full-wavenumber Laplacian -|k|^2
template <typename T>
void fill_symbol(const vd_grid* G, int kind, double a, T* out, cudaStream_t st);

// single-launch solves of 1D pressure problems in FP64 (vd_small.cu): eligibility, and the
// solve itself (out_dev: a result record in device memory, hist_dev: hist_cap doubles)
bool small_solve_eligible(const vd_grid* G, vd_op op, int solver, int precision, int restart);
vd_status small_solve_1d(const vd_grid* G, int solver, const vd_solve_params* prm, int restart, const double* b,
                         double* x, vd_solve_info* info, void* out_dev, double* hist_dev, int hist_cap,
                         cudaStream_t st);

// one solve recorded into the capture of st (see vd_api.cu); body: 3 streams for the
// conditional bodies (one is enough in FP64)
vd_status enqueue_solve_graph(const vd_grid* G, vd_op op, vd_solver solver, const vd_op_params* opp, double tol,
                              int maxit, int restart, int precision, const double* b, double* x, void* ws,
                              size_t ws_bytes, double* info, cudaStream_t st, cudaStream_t const* body);

}  // namespace vd
