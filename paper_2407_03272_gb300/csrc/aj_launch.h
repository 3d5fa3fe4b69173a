// aj_launch.h -- type-erased launch interface between the host API and the
// per-precision kernel translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace aj {

struct RhsState;

// Untyped mirror of IterArgs<P>; the pointer types follow the precision.
struct IterLaunch {
  int n;
  const int* row_ptr;
  const int* col;
  const void* val;
  const void* b;
  const void* jinv;
  void* x[3];
  void* u[2];  // stored sweep form only
  double* partials;
  unsigned long long* bar;
  int* err;
  RhsState* state;
  long long* rlog;
  int rlog_cap;
  double* trace;
  long long trace_cap;
  long long maxit;
  int stop;
  int restart;
  int momentum;
  double tol;
  double fstar;
  double fscale;
  long long max_sweeps;
  int qx;  // 1: stored sweep form (u = Q x kept), 0: lazy form (two row sums)
};

// Cooperative launch of the persistent kernel for precision `pol`
// (0 F64, 1 DF64, 2 F32, 3 BF16), nrhs in [1, 4] and the sweep form L.qx.
cudaError_t launch_persistent(int pol, int nrhs, const IterLaunch& L, int grid, cudaStream_t s);
// Co-resident CTAs per SM of that kernel (0 on error).
int persistent_blocks_per_sm(int pol, int nrhs, int qx);

cudaError_t launch_persistent_f64(int nrhs, const IterLaunch& L, int grid, cudaStream_t s);
cudaError_t launch_persistent_df64(int nrhs, const IterLaunch& L, int grid, cudaStream_t s);
cudaError_t launch_persistent_f32(int nrhs, const IterLaunch& L, int grid, cudaStream_t s);
cudaError_t launch_persistent_b16(int nrhs, const IterLaunch& L, int grid, cudaStream_t s);
int blocks_per_sm_f64(int nrhs, int qx);
int blocks_per_sm_df64(int nrhs, int qx);
int blocks_per_sm_f32(int nrhs, int qx);
int blocks_per_sm_b16(int nrhs, int qx);

}  // namespace aj
