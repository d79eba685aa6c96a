// Common device types for the variable-density spectral solver library.
//
// Layout (all fields row-major, x fastest):
//   physical real field  : T[n2][n1][n0]
//   half spectrum        : cpx<T>[n2][n1][h0],  h0 = n0/2 + 1
// Wavenumbers: k~_j = (2 pi / L_j) * f_j(m) with f(m) = m for m < n/2, m - n for m > n/2 and
// 0 at the Nyquist index m = n/2 (first derivatives of a real field stay real and
// skew-symmetric; the discrete Laplacian sum_j D_j D_j has symbol -|k~|^2).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace vd {

template <typename T>
struct __align__(2 * sizeof(T)) cpx {
  T x, y;
};

template <typename T>
__host__ __device__ __forceinline__ cpx<T> mk(T a, T b) {
  cpx<T> r;
  r.x = a;
  r.y = b;
  return r;
}
template <typename T>
__host__ __device__ __forceinline__ cpx<T> operator+(cpx<T> a, cpx<T> b) {
  return mk<T>(a.x + b.x, a.y + b.y);
}
template <typename T>
__host__ __device__ __forceinline__ cpx<T> operator-(cpx<T> a, cpx<T> b) {
  return mk<T>(a.x - b.x, a.y - b.y);
}
template <typename T>
__host__ __device__ __forceinline__ cpx<T> scal(cpx<T> a, T s) {
  return mk<T>(a.x * s, a.y * s);
}
// a * w (complex product)
template <typename T>
__host__ __device__ __forceinline__ cpx<T> cmul(cpx<T> a, cpx<T> w) {
  return mk<T>(a.x * w.x - a.y * w.y, a.x * w.y + a.y * w.x);
}
// a * conj(w)
template <typename T>
__host__ __device__ __forceinline__ cpx<T> cmulc(cpx<T> a, cpx<T> w) {
  return mk<T>(a.x * w.x + a.y * w.y, a.y * w.x - a.x * w.y);
}
template <typename T>
__host__ __device__ __forceinline__ cpx<T> conjg(cpx<T> a) {
  return mk<T>(a.x, -a.y);
}
// i * a
template <typename T>
__host__ __device__ __forceinline__ cpx<T> mul_i(cpx<T> a) {
  return mk<T>(-a.y, a.x);
}
// (i k) * a for real k
template <typename T>
__host__ __device__ __forceinline__ cpx<T> mul_ik(cpx<T> a, T k) {
  return mk<T>(-k * a.y, k * a.x);
}

// Maximum number of radix stages of one transform length.
constexpr int kMaxStages = 12;

// One complex FFT length n = prod(rad[0..nst-1]), radices in {2,3,4,5,8}; its twiddle table
// W_n^j = exp(-2 pi i j / n), j in [0, n), starts at element tw_off of the twiddle buffer.
struct FftPlan {
  int n;
  int nst;
  int rad[kMaxStages];
  int tw_off;
};

// Plans of one grid.  The x axis is transformed as a complex FFT of length m = n0/2 plus the
// real-data packing step, which needs W_{n0}^k for k in [0, m] (table at pk_off).
struct GridDesc {
  int ndim;
  int n0, n1, n2;
  int h0;
  long long nreal;   // n0 n1 n2
  long long ncplx;   // h0 n1 n2
  double kfac[3];    // 2 pi / L_j
  float kfac_dd[3][2];   // float-pair split of kfac (hi, lo)
  float kfac_f[3];       // kfac rounded to float (float kernels: no double -> float conversion on the device)
  FftPlan px;        // length n0/2
  FftPlan py;        // length n1 (ndim >= 2)
  FftPlan pz;        // length n2 (ndim == 3)
  int pk_off;        // packing twiddles W_{n0}^k, k = 0..n0/2
  int* dev_err = nullptr;   // device error word of the grid (a bounded wait gave up), or null
};

// signed integer frequency of index m on an axis of n points, with the Nyquist index -> 0
__host__ __device__ __forceinline__ int freq_tilde(int m, int n) {
  return (2 * m < n) ? m : ((2 * m == n) ? 0 : m - n);
}

// Diagonal symbols used as multipliers.
enum SymbolKind : int {
  SYM_NONE = 0,
  SYM_PRESSURE = 1,   // -1/|k~|^2, 0 where |k~| = 0   (pseudo-inverse of the Laplacian)
  SYM_VELOCITY = 2,   // 1/(1 + a |k~|^2)              (inverse of I - a Lap)
  SYM_PROJECT = 3,    // 1 except 0 on the 2^d corner modes (projection onto the range)
  SYM_KLAP_INV = 4,   // -1/|k|^2 with full wavenumbers, 0 for the mean only (K_rho preconditioner)
  SYM_KLAP = 5,       // -|k|^2 with full wavenumbers (Laplacian of the K_rho form)
};

// signed integer frequency of index m on an axis of n points (Nyquist index kept as -n/2)
__host__ __device__ __forceinline__ int freq_full(int m, int n) { return (2 * m < n) ? m : m - n; }

}  // namespace vd
