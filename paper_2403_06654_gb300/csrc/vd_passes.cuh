// Transform passes of the spectral operators (host-side declarations).
//
// A 3D operator apply in spectral space is a chain of passes, each reading and writing
// half-spectrum fields in HBM once:
//   z pass (lines along z) -> y pass (lines along y) -> fused x pass (inverse real
//   transform, pointwise physical-space work, forward real transform) -> y pass -> z pass.
// 2D chains drop the z passes and 1D chains are a single fused x pass.  Multipliers that
// are diagonal in Fourier space (derivatives i k~_j, -|k~|^2, preconditioner symbols)
// are applied while a pass loads or stores, so they cost no extra memory traffic.
#pragma once

#include "vd_common.cuh"

namespace vd {

// pre/post multiplier flags (combinable)
enum MulFlags : int {
  MUL_IK = 1,      // i k~ of the pass axis
  MUL_SYM = 2,     // the program's diagonal symbol (needs every axis in spectral space)
  MUL_NEGK2 = 4,   // -|k~|^2 (needs every axis in spectral space)
  MUL_IK2 = 8,     // (i k~)^2 = -k~^2 of the pass axis
};

constexpr int kMaxXf = 16;
constexpr int kMaxIO = 16;

// One transform of an axis pass: out[dst] (=|+=) scale * post( FFT( pre( in[src] ) ) ).
// Every transform writes out[dst] (an accumulating one adds to what an earlier transform of
// the same program wrote there), so a program must not read a buffer after one of its
// transforms has overwritten it; `last` is informative only.
// MUL_SYM reads the program's symbol array at the element's spectral index, so it is only
// meaningful where every axis is in spectral space (first inverse / last forward pass).
struct Xf {
  int8_t src, dst, pre, post;
  int8_t first;   // start a new accumulation for dst
  int8_t last;    // write dst after this transform
  int8_t nofft;   // skip the transform (pure diagonal multiply)
  int8_t pad;
  double scale;
  float scale_hi, scale_lo;   // float-pair split of scale (set on the host)
};

struct AxisProg {
  int nxf;
  Xf xf[kMaxXf];
  const void* in[kMaxIO];
  void* out[kMaxIO];
  const void* symarr;   // real symbol array (ncplx, same layout as the spectral fields)
  const int* done;      // if non-null and *done != 0 the kernel returns at once
  int axis;   // 1 = y, 2 = z
  int conv_in;          // float-pair kernels: bit i set -> in[i] holds doubles (split on load)
  int conv_out;         // float-pair kernels: bit i set -> out[i] holds doubles (summed on store)
};

// Fused x pass: for every component c, in[c] (half spectrum) -> pre -> inverse real FFT ->
// multiply by wfield (real, n0 per line; nullptr = 1) -> forward real FFT -> post -> out[c].
// mode 0: fused as described; mode 1: real in (in[c] is T*), forward only; mode 2: inverse
// only, real out (out[c] is T*).  scale multiplies the result.
constexpr int kMaxXComp = 6;

struct XProg {
  int ncomp;   // <= kMaxXComp
  int mode;
  const void* in[kMaxXComp];
  void* out[kMaxXComp];
  int pre[kMaxXComp];
  int post[kMaxXComp];
  const void* wfield;
  // float programs only: wfield holds a float pair (hi, lo) per real point, and the multiply
  // z * (hi + lo) is carried in float-pair arithmetic, rounded to float once
  int wf_dd;
  double scale;
  float scale_hi, scale_lo;   // float-pair split of scale (set by launch_xpass)
  const void* symarr;
  const int* done;
  int conv_in;          // float-pair kernels: bit c set -> in[c] holds doubles
  int conv_out;         // float-pair kernels: bit c set -> out[c] holds doubles
  // mode 0 only: if aux_out is set, component 0 is also transformed inverse-only (no pre
  // multiplier, as mode 2) into the real field aux_out, scaled by aux_scale (doubles when
  // aux_conv is set); that output equals a separate mode-2 pass over in[0] bit for bit
  void* aux_out;
  double aux_scale;
  float aux_scale_hi, aux_scale_lo;
  int aux_conv;
};

template <typename T>
void launch_axis(const AxisProg& P, int dir, const GridDesc& g, const void* tw, cudaStream_t st);

template <typename T>
void launch_xpass(const XProg& P, const GridDesc& g, const void* tw, cudaStream_t st);

// launch-shape table (vd_passes.cu).  kind 0: y/z pass (key: type, length, axis, direction);
// kind 1: x pass (key: type, n0/2, axis 0, mode).  type: 0 double, 1 float, 2 float-pair.
// choice: 0 register four-step kernel, > 0 lines per block, < 0 (get) absent / (set) erase.
// kind 0 choice kChoiceStaged: the register kernel with TMA-staged input (float y/z passes of
// length 128 / 256).  Type 2 choice kChoiceUnpacked (either kind): the Stockham engine on
// unpacked float pairs with the default lines per block, instead of the packed engine that the
// float-pair passes use for lengths whose radices are 2, 4 and 8 (same results, bit for bit).
constexpr int kChoiceStaged = 128;
constexpr int kChoiceUnpacked = 256;
int tune_get(int kind, int type, int n, int axis, int dir);
void tune_set(int kind, int type, int n, int axis, int dir, int choice);
int tune_table(int* out, int max);   // 6 ints per entry; returns the entry count
int default_shape(int kind, int type, int n, int axis = 0);   // the built-in choice (kind 1: n = n0/2)
void tune_save();                    // write the table to $VD_TUNE_FILE (if set)

// shared memory footprint (bytes) of the pass kernels, for the attribute setup
template <typename T>
size_t axis_smem_bytes(const GridDesc& g, int axis);
template <typename T>
size_t xpass_smem_bytes(const GridDesc& g);

}  // namespace vd
