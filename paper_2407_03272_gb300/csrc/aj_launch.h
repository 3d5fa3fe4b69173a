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
  int nrhs;  // right-hand sides, 1..4
  const int* row_ptr;
  const int* col;
  const void* val;
  int fmt;  // 0 CSR, 1 SELL-C-sigma (fields below), 2 constant-coefficient stencil
  int sdim, sN, sdiag_at, soff_at;  // stencil: 2 or 3 dimensions, grid side, entries of val
  unsigned long long smag;          // stencil: q / N = (q * smag) >> sshift for 0 <= q < 2^31
  int sshift;
  int jblk;                         // rows per block of J (1: diagonal)
  int short_rows;                   // 1: no row has more than 32 entries (zero: not known)
  int nsell;
  int sell_cl;  // log2 of the SELL slice height
  int ntiles_sell;
  int nltiles;
  const int* perm;
  const int* rlen;
  const int* sptr;
  const int* scol;
  const void* sval;
  const int* long_rows;
  const int* ltp;
  int nhuge;
  const int* huge_rows;
  const void* b;
  const void* jinv;
  void* x[3];
  void* u[2];  // stored sweep forms only
  void* dl;    // difference sweep form only: x^t - x^{t-1}
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
  unsigned long long bar_timeout_ns;  // limit of each grid-barrier wait (0: the default, 4 s)
  int bar_withhold;                   // failure-detection tests: CTA index + 1 that withholds its
                                      // first barrier arrival (0: none), see grid_sync
  int qx;  // sweep form: 0 lazy (two row sums), 1 stored (u = Q x kept), 2 stored + difference
};

// Untyped mirror of LockArgs<P>: many systems in lockstep in one launch.
// `sys` is a device array of per-system kernel arguments packed with
// pack_iter_args (the layout is the same for every precision policy).
struct LockLaunch {
  const void* sys;
  const int* unit_sys;
  const int* sys_u0;
  const int* sys_nu;
  const int* cta_u0;
  RhsState* st2;
  RhsState* st_out;
  int nu;
  long long sweeps;
  unsigned long long* bar;
  int* err;
};

// Size in bytes of one packed per-system argument block, and the packing.
size_t iter_args_bytes();
void pack_iter_args(int pol, const IterLaunch& L, void* dst);
// Cooperative launch of the lockstep kernel (systems of any right-hand-side
// count) and its co-resident CTAs per SM.
cudaError_t launch_lockstep(int pol, int qx, const LockLaunch& B, int grid, cudaStream_t s);
int lockstep_blocks_per_sm(int pol, int qx);

// Cooperative launch of the persistent kernel for precision `pol`
// (0 F64, 1 DF64, 2 F32, 3 BF16), nrhs in [1, 4] and the sweep form L.qx.
cudaError_t launch_persistent(int pol, int nrhs, const IterLaunch& L, int grid, cudaStream_t s);
// Co-resident CTAs per SM of that kernel for formats fm (0 CSR only, 1 any,
// 2 stencil only, 3 SELL-32 only, 4 SELL-16/8 only; fm < 0: the smallest over
// them), 0 on error.
int persistent_blocks_per_sm(int pol, int nrhs, int qx, int fm = -1);

cudaError_t launch_persistent_f64(int nrhs, const IterLaunch& L, int grid, cudaStream_t s);
cudaError_t launch_persistent_df64(int nrhs, const IterLaunch& L, int grid, cudaStream_t s);
cudaError_t launch_persistent_f32(int nrhs, const IterLaunch& L, int grid, cudaStream_t s);
cudaError_t launch_persistent_b16(int nrhs, const IterLaunch& L, int grid, cudaStream_t s);
int blocks_per_sm_f64(int nrhs, int qx, int fm = -1);
int blocks_per_sm_df64(int nrhs, int qx, int fm = -1);
int blocks_per_sm_f32(int nrhs, int qx, int fm = -1);
int blocks_per_sm_b16(int nrhs, int qx, int fm = -1);

#define AJ_DECLARE_BATCHED(suf)                                                              \
  void pack_iter_args_##suf(const IterLaunch& L, void* dst);                                 \
  cudaError_t launch_lockstep_##suf(int qx, const LockLaunch& B, int grid, cudaStream_t s);  \
  int lockstep_blocks_per_sm_##suf(int qx);
AJ_DECLARE_BATCHED(f64)
AJ_DECLARE_BATCHED(df64)
AJ_DECLARE_BATCHED(f32)
AJ_DECLARE_BATCHED(b16)
#undef AJ_DECLARE_BATCHED

}  // namespace aj
