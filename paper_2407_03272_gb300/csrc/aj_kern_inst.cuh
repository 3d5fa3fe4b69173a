// aj_kern_inst.cuh -- instantiates the persistent and batched kernels of one
// precision policy (one right-hand side, and 2..4 with lanes per row).  Included once per translation unit with
// AJ_POL (policy type) and AJ_SUFFIX (name suffix) defined.
#include <string.h>

#include <algorithm>
#include <type_traits>

#include "aj_core.cuh"
#include "aj_launch.h"

#define AJ_CAT2(a, b) a##b
#define AJ_CAT(a, b) AJ_CAT2(a, b)

namespace aj {

template <class P>
static IterArgs<P> typed_args(const IterLaunch& L) {
  IterArgs<P> a;
  a.n = L.n;
  a.nrhs = L.nrhs;
  a.lgr = lanes_log2(L.nrhs);
  a.row_ptr = L.row_ptr;
  a.col = L.col;
  a.val = static_cast<const typename P::V*>(L.val);
  a.fmt = L.fmt;
  a.sdim = L.sdim;
  a.sN = L.sN;
  a.sdiag_at = L.sdiag_at;
  a.soff_at = L.soff_at;
  a.smag = L.smag;
  a.sshift = L.sshift;
  a.jblk = L.jblk < 1 ? 1 : L.jblk;
  a.short_rows = L.short_rows;
  a.nsell = L.nsell;
  a.sell_cl = L.sell_cl ? L.sell_cl : 5;
  a.ntiles_sell = L.ntiles_sell;
  a.nltiles = L.nltiles;
  a.perm = L.perm;
  a.rlen = L.rlen;
  a.sptr = L.sptr;
  a.scol = L.scol;
  a.sval = static_cast<const typename P::V*>(L.sval);
  a.long_rows = L.long_rows;
  a.ltp = L.ltp;
  a.nhuge = L.nhuge;
  a.huge_rows = L.huge_rows;
  a.b = static_cast<const typename P::X*>(L.b);
  a.jinv = static_cast<const typename P::X*>(L.jinv);
  for (int k = 0; k < 3; k++) a.x[k] = static_cast<typename P::X*>(L.x[k]);
  for (int k = 0; k < 2; k++) a.u[k] = static_cast<typename P::X*>(L.u[k]);
  a.dl = static_cast<typename P::X*>(L.dl);
  a.partials = L.partials;
  a.bar = L.bar;
  a.err = L.err;
  a.state = L.state;
  a.rlog = L.rlog;
  a.rlog_cap = L.rlog_cap;
  a.trace = L.trace;
  a.trace_cap = L.trace_cap;
  a.maxit = L.maxit;
  a.stop = L.stop;
  a.restart = L.restart;
  a.momentum = L.momentum;
  a.tol = L.tol;
  a.fstar = L.fstar;
  a.fscale = L.fscale;
  a.max_sweeps = L.max_sweeps;
  a.bar_timeout_ns = L.bar_timeout_ns ? L.bar_timeout_ns : kBarrierTimeoutNs;
  a.bar_withhold_cta = L.bar_withhold - 1;
  return a;
}

// The difference sweep form (SF = 2) is built for FP64 only, the policy whose
// FP64 issue rate it relieves.
template <class P>
constexpr bool kHasDelta = std::is_same<P, PolF64>::value;

template <class P>
static cudaError_t launch_lockstep_p(int qx, const LockLaunch& B, int grid, cudaStream_t s) {
  LockArgs<P> b;
  b.sys = static_cast<const IterArgs<P>*>(B.sys);
  b.unit_sys = B.unit_sys;
  b.sys_u0 = B.sys_u0;
  b.sys_nu = B.sys_nu;
  b.cta_u0 = B.cta_u0;
  b.st2 = B.st2;
  b.st_out = B.st_out;
  b.nu = B.nu;
  b.sweeps = B.sweeps;
  b.bar = B.bar;
  b.err = B.err;
  void* args[] = {&b};
  const void* k = nullptr;
  if (qx == 0) k = (const void*)aj_lockstep_kernel<P, 0>;
  else if (qx == 1) k = (const void*)aj_lockstep_kernel<P, 1>;
  else if (qx == 3) k = (const void*)aj_lockstep_kernel<P, 3>;
  else if constexpr (kHasDelta<P>) {
    if (qx == 2) k = (const void*)aj_lockstep_kernel<P, 2>;
  }
  if (!k) return cudaErrorInvalidValue;
  return cudaLaunchCooperativeKernel(k, dim3(grid), dim3(kThreads), args, 0, s);
}

// Co-resident CTAs per SM of kernel k.  Kernels with stage buffers in shared
// memory (the staged stencil sweep) ask for the largest shared-memory
// carveout first, so that their CTAs per SM are limited by registers, not by
// the L1 / shared split; the others keep the default split (their gathers
// use L1).
static int occ_of(const void* k) {
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, k) == cudaSuccess && fa.sharedSizeBytes > 8192)
    cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
  cudaGetLastError();
  int nb = 0;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, kThreads, 0) == cudaSuccess ? nb : 0;
}

// The persistent kernel for sweep form sf and formats fm (0 CSR only, 1
// any, 2 stencil only, 3 SELL-32 only, 4 SELL-16/8 only).
template <class P, int SF, bool MULTI>
static const void* persistent_fm(int fm) {
  return fm == 0   ? (const void*)aj_persistent_kernel<P, SF, 0, MULTI>
         : fm == 1 ? (const void*)aj_persistent_kernel<P, SF, 1, MULTI>
         : fm == 2 ? (const void*)aj_persistent_kernel<P, SF, 2, MULTI>
         : fm == 3 ? (const void*)aj_persistent_kernel<P, SF, 3, MULTI>
                   : (const void*)aj_persistent_kernel<P, SF, 4, MULTI>;
}

template <class P, bool MULTI>
static const void* persistent_fn(int sf, int fm) {
  if (sf == 0) return persistent_fm<P, 0, MULTI>(fm);
  if (sf == 1) return persistent_fm<P, 1, MULTI>(fm);
  if (sf == 3) return persistent_fm<P, 3, MULTI>(fm);
  if constexpr (kHasDelta<P>)
    if (sf == 2) return persistent_fm<P, 2, MULTI>(fm);
  return nullptr;
}

// The instantiation a launch needs: the stencil rows alone, SELL alone, CSR
// alone, or any (the block-diagonal J).
static int launch_fm(const IterLaunch& L) {
  return L.fmt == 2 ? 2 : L.jblk > 1 ? 1
         : L.fmt == 1 ? (L.sell_cl && L.sell_cl < 5 ? 4 : AJ_SELL_FM) : 0;
}

template <class P, bool MULTI>
static cudaError_t launch_m(const IterLaunch& L, int grid, cudaStream_t s) {
  IterArgs<P> a = typed_args<P>(L);
  void* args[] = {&a};
  const void* k = persistent_fn<P, MULTI>(L.qx, launch_fm(L));
  if (!k) return cudaErrorInvalidValue;
  return cudaLaunchCooperativeKernel(k, dim3(grid), dim3(kThreads), args, 0, s);
}

// Co-resident CTAs of the persistent kernel for formats fm (0 CSR only, 1
// any, 2 stencil only, 3 and 4 SELL only), or with fm < 0 the smallest over them, so that
// a grid sized by it fits any of them.
template <class P, bool MULTI>
static int occ_m(int qx, int fm) {
  if (fm >= 0) {
    const void* k = persistent_fn<P, MULTI>(qx, fm);
    return k ? occ_of(k) : 0;
  }
  int occ = 1 << 30;
  for (int f = 0; f < 5; f++) {
    const void* k = persistent_fn<P, MULTI>(qx, f);
    if (!k) return 0;
    occ = std::min(occ, occ_of(k));
  }
  return occ;
}

cudaError_t AJ_CAT(launch_persistent_, AJ_SUFFIX)(int nrhs, const IterLaunch& L, int grid,
                                                  cudaStream_t s) {
  if (nrhs < 1 || nrhs > kMaxRhs || L.nrhs != nrhs) return cudaErrorInvalidValue;
  return nrhs == 1 ? launch_m<AJ_POL, false>(L, grid, s) : launch_m<AJ_POL, true>(L, grid, s);
}

int AJ_CAT(blocks_per_sm_, AJ_SUFFIX)(int nrhs, int qx, int fm) {
  if (nrhs < 1 || nrhs > kMaxRhs) return 0;
  return nrhs == 1 ? occ_m<AJ_POL, false>(qx, fm) : occ_m<AJ_POL, true>(qx, fm);
}

void AJ_CAT(pack_iter_args_, AJ_SUFFIX)(const IterLaunch& L, void* dst) {
  static_assert(sizeof(IterArgs<AJ_POL>) == sizeof(IterArgs<PolF64>), "one packed layout");
  IterArgs<AJ_POL> a = typed_args<AJ_POL>(L);
  memcpy(dst, &a, sizeof(a));
}

cudaError_t AJ_CAT(launch_lockstep_, AJ_SUFFIX)(int qx, const LockLaunch& B, int grid, cudaStream_t s) {
  return launch_lockstep_p<AJ_POL>(qx, B, grid, s);
}

int AJ_CAT(lockstep_blocks_per_sm_, AJ_SUFFIX)(int qx) {
  if (qx == 0) return occ_of((const void*)aj_lockstep_kernel<AJ_POL, 0>);
  if (qx == 1) return occ_of((const void*)aj_lockstep_kernel<AJ_POL, 1>);
  if (qx == 3) return occ_of((const void*)aj_lockstep_kernel<AJ_POL, 3>);
  if constexpr (kHasDelta<AJ_POL>)
    if (qx == 2) return occ_of((const void*)aj_lockstep_kernel<AJ_POL, 2>);
  return 0;
}

}  // namespace aj
