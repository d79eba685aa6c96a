// Launch counting and optional per-kernel-class event timing.
//
// Every kernel launch of the library increments a process-wide counter.  When profiling is
// enabled, the transform-pass launches are bracketed by CUDA events recorded on the launching
// stream, and the algorithmic bytes (each input/output field once) and flops (5 n log2 n per
// complex line transform of length n) of the launch are accumulated per class.
#pragma once

#include <cuda_runtime.h>

namespace vd {

enum ProfClass : int {
  PC_AXIS64 = 0,   // strided y/z pass, double
  PC_AXIS32 = 1,   // strided y/z pass, float
  PC_XPASS64 = 2,  // contiguous x pass, double
  PC_XPASS32 = 3,  // contiguous x pass, float
  PC_OTHER = 4,    // reductions, vector updates, pointwise kernels
  PC_AXISDD = 5,   // strided y/z pass, float-pair
  PC_XPASSDD = 6,  // contiguous x pass, float-pair
  PC_VEC32 = 7,    // Krylov vector kernels on float vectors
  PC_VEC64 = 8,    // Krylov vector kernels on double vectors
  PC_INNER32 = 9,  // a whole inner float Krylov solve (span mode only)
  PC_N = 10
};

void count_launch();
bool vd_profile_is_on();   // event timing enabled (events cannot be recorded into a graph)

// Launches enqueued past convergence (they return at once) must not add their algorithmic
// bytes: prof_mark() before enqueuing such a batch, prof_discard(mark, st) once it is known
// to have been speculative drops the records of that stream from the mark on.
long long prof_mark();
void prof_discard(long long mark, cudaStream_t st);

// RAII bracket of a stretch of work (span mode, vd_profile_enable(2)): two events around it
// on its stream and the algorithmic bytes and flops of the launches issued inside it on that
// stream; the launches themselves are not bracketed in this mode
struct ProfSpan {
  ProfSpan(int cls, cudaStream_t st);
  ~ProfSpan();
  int cls;
  cudaStream_t st;
  long long seq0;
  cudaEvent_t a;
};

// RAII bracket of one launch; records events only when profiling is on (mode 1)
struct ProfScope {
  ProfScope(int cls, cudaStream_t st, double bytes, double flops);
  ~ProfScope();
  int cls;
  cudaStream_t st;
  double bytes, flops;
  int slot;
};

}  // namespace vd
