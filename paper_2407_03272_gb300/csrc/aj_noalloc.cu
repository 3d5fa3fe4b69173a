// aj_noalloc.cu -- aj_solve_noalloc: the FP64 fused AJ solve for one
// right-hand side, with every scratch buffer in one fixed device array of this
// file instead of memory allocated per call.
//
// Some callers must not allocate device memory: a latency-critical server whose
// other streams would stall on the implicit device synchronisation of
// cudaMalloc / cudaFree; a process whose device memory is all reserved up front
// by a framework's caching allocator, so that a foreign cudaMalloc can fail at
// run time; embedded or certified deployments that fix every device buffer at
// load time.  This entry point serves them.  The caller passes the matrix, b
// and the output on the device; the library supplies J^{-1}, the three iterate
// buffers, the two Q x buffers of the stored sweep form, the per-CTA partial
// sums, the grid-barrier counter, the error word and the solver state from the
// array below.  Nothing here calls cudaMalloc,
// cudaFree or an allocating library routine.
//
// The array is a host-side stand-in in host code: its device address comes
// from cudaGetSymbolAddress, taken once per device with that device current.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>

#include "aj.h"
#include "aj_core.cuh"
#include "aj_launch.h"

namespace {

using namespace aj;

constexpr long long kNaMaxN = AJ_NOALLOC_MAX_N;
constexpr int kNaMaxTiles = (int)((kNaMaxN + kThreads - 1) / kThreads);  // largest useful grid
constexpr int kNaRlogCap = 64;
constexpr int kNaThreads = 256;
constexpr int kNaMaxDevices = 64;

// Layout of the scratch array (byte offsets, each 256-byte aligned).
constexpr size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }
constexpr size_t kOffJinv = 0;
constexpr size_t kOffX0 = align256(kOffJinv + (size_t)kNaMaxN * 8);
constexpr size_t kVecBytes = align256((size_t)kNaMaxN * 8);
constexpr size_t kOffU0 = kOffX0 + 3 * kVecBytes;
constexpr size_t kOffPart = kOffU0 + 2 * kVecBytes;
constexpr size_t kOffState = align256(kOffPart + (size_t)2 * kNaMaxTiles * kNRed * 8);
constexpr size_t kOffRlog = align256(kOffState + sizeof(RhsState));
constexpr size_t kOffBar = align256(kOffRlog + (size_t)kNaRlogCap * 8);
constexpr size_t kOffErr = kOffBar + 64;
constexpr size_t kOffFlags = kOffErr + 64;
constexpr size_t kOffBpart = kOffFlags + 64;  // per-block partial sums of ||b||^2
constexpr size_t kScratchBytes = align256(kOffBpart + (size_t)kNaMaxTiles * 8);

// The fixed scratch: about 6.1 MB, held by every GPU that loads libaj.
static __device__ __align__(256) unsigned char g_na_scratch[kScratchBytes];

struct NaDevice {
  bool ready = false;
  unsigned char* base = nullptr;  // device address of g_na_scratch on this device
  int grid_cap = 0;               // co-resident CTAs of the FP64 persistent kernel
};
NaDevice g_na_dev[kNaMaxDevices];
std::mutex g_na_mu;

// Validation of the caller's CSR (each thread checks its own row's bounds
// before it reads the row), diag and J^{-1} (eq. J-diag or J = L D, the same
// summation order as aj_set), in one pass.  flags gets the error bits.
__global__ void k_na_prepare(int n, long long nnz, const int* rp, const int* ci, const double* val,
                             int policy, double L, double* jinv, int* flags) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int a = rp[i], e = rp[i + 1];
  int f = 0;
  if (a < 0 || e < a || (long long)e > nnz) f |= 1;
  if (i == 0 && a != 0) f |= 1;
  if (i == n - 1 && (long long)e != nnz) f |= 1;
  if (f) {
    atomicOr(flags, f);
    return;
  }
  double d = 0.0;
  bool off_nonzero = false;
  for (int q = a; q < e; q++) {
    const int c = ci[q];
    const double v = val[q];
    if (c < 0 || c >= n) f |= 2;
    if (!isfinite(v)) f |= 4;
    if (c == i) d += v;
    else if (v != 0.0) off_nonzero = true;
  }
  if (d < 0.0) f |= 8;
  if (d == 0.0 && off_nonzero) f |= 16;
  if (f) {
    atomicOr(flags, f);
    return;
  }
  double j;
  if (policy == AJ_J_ABSROWSUM) {
    double off = 0.0;
    for (int q = a; q < e; q++)
      if (ci[q] != i) off += fabs(val[q]);
    j = d + off;
  } else {
    j = L * d;
  }
  if (j == 0.0) j = 1.0;
  jinv[i] = 1.0 / j;
}

// ||b||^2 in the order aj_create forms it, so that the stop test sees the
// same bits: per block of 256 entries, the squares summed by a xor tree over
// each warp's lanes and then the 8 warps in order (one partial per block,
// into bpart); k_na_init then adds the partials in block order.  A
// non-finite entry sets flag bit 32.
__global__ void k_na_bnorm2(int n, const double* b, double* bpart, int* flags) {
  __shared__ double sm[kNaThreads / 32];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double v = 0.0;
  if (i < n) {
    const double bi = b[i];
    if (!isfinite(bi)) atomicOr(flags, 32);
    v = __dmul_rn(bi, bi);
  }
  for (int m = 16; m >= 1; m >>= 1) v = __dadd_rn(v, __shfl_xor_sync(0xffffffffu, v, m));
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < kNaThreads / 32; k++) s = __dadd_rn(s, sm[k]);
    bpart[blockIdx.x] = s;
  }
}

// x^0 into iterate buffer 0; clears the barrier counter, the error word and
// the restart log; block 0 thread 0 also adds the block partials of ||b||^2
// (k_na_bnorm2) in block order and writes the initial solver state.
__global__ void k_na_init(int n, const double* x0, const double* bpart, int nbpart, long long K0,
                          double* x, RhsState* st, long long* rlog, unsigned long long* bar,
                          int* err) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = x0 ? x0[i] : 0.0;
  if (i < kNaRlogCap) rlog[i] = -1;
  if (i == 0) {
    *bar = 0ull;
    *err = 0;
    double s = 0.0;
    for (int k = 0; k < nbpart; k++) s = __dadd_rn(s, bpart[k]);
    RhsState q;
    memset(&q, 0, sizeof(q));
    q.alpha = 1.0;
    q.beta = 0.0;
    q.bnorm2 = s;
    q.K = K0;
    q.cur = 0;
    q.prev = 0;
    q.nxt = 1;
    *st = q;
  }
}

// x_out = the buffer that holds the returned iterate.
__global__ void k_na_finish(int n, const RhsState* st, const double* x0, const double* x1,
                            const double* x2, double* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int k = st->cur;
  const double* src = k == 0 ? x0 : (k == 1 ? x1 : x2);
  out[i] = src[i];
}

// Device address of the scratch array and the grid cap on the current
// device, taken once per device.
aj_status na_setup(NaDevice** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return AJ_ECUDA;
  }
  if (dev < 0 || dev >= kNaMaxDevices) return AJ_ECUDA;
  std::lock_guard<std::mutex> lk(g_na_mu);
  NaDevice& d = g_na_dev[dev];
  if (!d.ready) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_na_scratch) != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return AJ_ECUDA;
    }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      return AJ_ECUDA;
    }
    const int bps = blocks_per_sm_f64(1, 1);
    if (bps < 1 || sms < 1) return AJ_ECUDA;
    d.base = (unsigned char*)p;
    d.grid_cap = bps * sms;
    d.ready = true;
  }
  *out = &d;
  return AJ_OK;
}

aj_status na_status(int s) {
  switch (s) {
    case kOk: return AJ_OK;
    case kEMaxit: return AJ_EMAXIT;
    case kEDiverged: return AJ_EDIVERGED;
    case kENonfinite: return AJ_ENONFINITE;
    case kETimeout: return AJ_ETIMEOUT;
  }
  return AJ_ECUDA;
}

}  // namespace

#define NA_CK(expr)                 \
  do {                              \
    if ((expr) != cudaSuccess) {    \
      cudaGetLastError();           \
      return AJ_ECUDA;              \
    }                               \
  } while (0)

extern "C" aj_status aj_solve_noalloc(const aj_csr* Q, const double* b, const aj_params* p,
                                      double* x_out, aj_info* info, void* cuda_stream) {
  const auto t0 = std::chrono::steady_clock::now();
  if (info) std::memset(info, 0, sizeof(*info));
  if (!Q || !p) return AJ_EINVAL;
  if (Q->n < 0 || Q->nnz < 0 || Q->nnz >= (1ll << 31) - 1) return AJ_EINVAL;
  if (Q->n > kNaMaxN) return AJ_ENOMEM;
  if (Q->n > 0 && (!Q->on_device || !Q->row_ptr || !b || !x_out)) return AJ_EINVAL;
  if (Q->nnz > 0 && (!Q->col || !Q->val)) return AJ_EINVAL;
  if (p->precision != AJ_FP64) return AJ_EINVAL;
  if (p->j_policy != AJ_J_ABSROWSUM && !(p->j_policy == AJ_J_SCALED_DIAG && p->L > 0.0))
    return AJ_EINVAL;
  if (p->restart != AJ_RESTART_NONE && p->restart != AJ_RESTART_ADAPTIVE) return AJ_EINVAL;
  if (p->K0 < 2 || p->maxit < 0 || !(p->tol >= 0.0)) return AJ_EINVAL;
  if (p->stop < AJ_STOP_RELRES || p->stop > AJ_STOP_NONE) return AJ_EINVAL;
  if (p->x0 && !p->x0_on_device) return AJ_EINVAL;
  const int n = (int)Q->n;
  if (n == 0) {
    if (info) info->status = AJ_OK;
    return AJ_OK;
  }
  NaDevice* d = nullptr;
  aj_status e = na_setup(&d);
  if (e != AJ_OK) return e;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  unsigned char* base = d->base;
  double* jinv = (double*)(base + kOffJinv);
  double* xb[3];
  for (int k = 0; k < 3; k++) xb[k] = (double*)(base + kOffX0 + k * kVecBytes);
  double* ub[2];
  for (int k = 0; k < 2; k++) ub[k] = (double*)(base + kOffU0 + k * kVecBytes);
  double* part = (double*)(base + kOffPart);
  RhsState* st = (RhsState*)(base + kOffState);
  long long* rlog = (long long*)(base + kOffRlog);
  unsigned long long* bar = (unsigned long long*)(base + kOffBar);
  int* err = (int*)(base + kOffErr);
  int* flags = (int*)(base + kOffFlags);
  double* bpart = (double*)(base + kOffBpart);
  const unsigned blocks = (unsigned)((n + kNaThreads - 1) / kNaThreads);
  int launches = 0;

  // setup: validate, J^{-1}, x^0, state
  NA_CK(cudaMemsetAsync(flags, 0, sizeof(int), s));
  k_na_prepare<<<blocks, kNaThreads, 0, s>>>(n, Q->nnz, Q->row_ptr, Q->col, Q->val, p->j_policy,
                                             p->L, jinv, flags);
  k_na_bnorm2<<<blocks, kNaThreads, 0, s>>>(n, b, bpart, flags);
  k_na_init<<<blocks, kNaThreads, 0, s>>>(n, p->x0, bpart, (int)blocks, p->K0, xb[0], st, rlog, bar, err);
  launches += 3;
  NA_CK(cudaGetLastError());
  int hflags = 0;
  NA_CK(cudaMemcpyAsync(&hflags, flags, sizeof(int), cudaMemcpyDeviceToHost, s));
  NA_CK(cudaStreamSynchronize(s));
  if (hflags) return AJ_EINVAL;

  // the fused persistent kernel
  const int ntiles = (n + kThreads - 1) / kThreads;
  int grid = std::min(d->grid_cap, ntiles);
  if (p->grid_ctas > 0) grid = std::min(grid, p->grid_ctas);
  if (grid < 1) grid = 1;
  IterLaunch L;
  std::memset(&L, 0, sizeof(L));
  L.n = n;
  L.nrhs = 1;
  L.row_ptr = Q->row_ptr;
  L.col = Q->col;
  L.val = Q->val;
  L.b = b;
  L.jinv = jinv;
  for (int k = 0; k < 3; k++) L.x[k] = xb[k];
  for (int k = 0; k < 2; k++) L.u[k] = ub[k];
  // the stored sweep form: the same iterates, bit for bit, as the difference
  // form, with one n-vector less of scratch
  L.qx = 1;
  L.partials = part;
  L.bar = bar;
  L.err = err;
  L.state = st;
  L.rlog = rlog;
  L.rlog_cap = kNaRlogCap;
  L.maxit = p->maxit;
  L.stop = p->stop;
  L.restart = p->restart == AJ_RESTART_ADAPTIVE;
  L.momentum = p->momentum != 0;
  L.tol = p->tol;
  L.fstar = p->fstar;
  L.fscale = 1.0;
  L.max_sweeps = p->maxit + 2;
  NA_CK(launch_persistent_f64(1, L, grid, s));
  k_na_finish<<<blocks, kNaThreads, 0, s>>>(n, st, xb[0], xb[1], xb[2], x_out);
  launches += 2;
  NA_CK(cudaGetLastError());
  RhsState hs;
  int herr = 0;
  NA_CK(cudaMemcpyAsync(&hs, st, sizeof(hs), cudaMemcpyDeviceToHost, s));
  NA_CK(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  NA_CK(cudaStreamSynchronize(s));
  if (herr != 0) return herr == kETimeout ? AJ_ETIMEOUT : AJ_ECUDA;
  const aj_status status = na_status(hs.status);
  if (info) {
    const double ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    info->iters = hs.t_final;
    info->restarts = hs.ell;
    info->sweeps = hs.t_final + 1;
    info->outer = 0;
    info->relres = hs.relres;
    info->objgap = p->stop == AJ_STOP_OBJGAP
                       ? std::fabs(hs.fval - p->fstar) / (1.0 + std::fabs(p->fstar))
                       : 0.0;
    info->L_used = p->j_policy == AJ_J_SCALED_DIAG ? p->L : 0.0;
    info->ms = ms;
    info->kernel_ms = ms;
    info->launches = launches;
    info->status = status;
  }
  return status;
}
