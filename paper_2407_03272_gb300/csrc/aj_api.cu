// aj_api.cu -- host implementation of the libaj C ABI (include/aj.h).
//
// A context owns a device copy of Q (CSR, FP64 master values plus, when the
// precision asks for it, an FP32 / BF16 / double-float copy), the right-hand
// sides, J^{-1}, three iterate buffers and the small workspaces of the
// persistent kernel.  aj_solve runs the persistent fused kernel (FP64 and
// DF64 directly; FP32 and BF16 as the inner solver of an FP64 iterative
// refinement loop) and reports the FP64 residual of what it returns.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <climits>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <tuple>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "aj.h"
#include "aj_core.cuh"
#include "aj_launch.h"
#include "aj_pcg.cuh"
#include "aj_setup.cuh"

using namespace aj;

namespace {

inline unsigned grid1d(long long m) { return (unsigned)((m + kSetupThreads - 1) / kSetupThreads); }

std::atomic<unsigned long long> g_launches{0};
thread_local long long t_launches = 0;  // launches of the solve running on this thread
inline void counted() {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  t_launches++;
}

// Failure-detection test hooks (aj_test_barrier_stall, aj_test_alloc_fail):
// a CTA of the next persistent launch that withholds its first barrier
// arrival, with the barrier's wait limit for that launch; and a device
// allocation that fails after `g_alloc_fail_after` more successful ones.
std::atomic<int> g_stall_cta{-1};
std::atomic<long long> g_stall_timeout_ns{0};
std::atomic<long long> g_alloc_fail_after{-1};

// Hits and misses of the process-wide caches (aj_cache_stats): the ordering
// cache of aj_set's locality test and the autotuner's choices.
std::atomic<unsigned long long> g_order_hits{0}, g_order_misses{0}, g_tune_hits{0}, g_tune_misses{0};

bool alloc_hook_fails() {
  long long v = g_alloc_fail_after.load();
  while (v >= 0) {
    const long long nv = v == 0 ? -1 : v - 1;
    if (g_alloc_fail_after.compare_exchange_weak(v, nv)) return v == 0;
  }
  return false;
}

// Device memory of the library comes from one memory pool per device, in
// stream order: cudaMallocFromPoolAsync and cudaFreeAsync neither
// synchronise the device nor hand memory back to the driver (the pool's
// release threshold is "never"), so contexts and server requests that come
// and go reuse blocks for the price of a pool lookup instead of paying
// cudaMalloc / cudaFree every time.  If the pool cannot be created, plain
// cudaMalloc / cudaFree are used.
cudaMemPool_t device_pool() {
  static std::mutex mu;
  static std::map<int, cudaMemPool_t> pools;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  std::lock_guard<std::mutex> lk(mu);
  auto it = pools.find(dev);
  if (it != pools.end()) return it->second;
  cudaMemPoolProps props;
  std::memset(&props, 0, sizeof(props));
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  cudaMemPool_t pool = nullptr;
  if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
    cudaGetLastError();
    pool = nullptr;
  } else {
    uint64_t never = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &never);
  }
  pools[dev] = pool;
  return pool;
}

// Allocations of one owner, made and freed in the order of the owner's stream
// (*stream; the legacy default stream when null).  Work that uses them on
// another stream must be ordered after that stream first.
struct Workspace {
  std::vector<std::pair<void*, bool>> ptrs;  // (pointer, from the pool)
  size_t bytes = 0;
  const cudaStream_t* stream = nullptr;
  cudaStream_t st() const { return stream ? *stream : nullptr; }
  void* alloc(size_t b) {
    void* p = nullptr;
    if (b == 0) b = 16;
    if (alloc_hook_fails()) return nullptr;
    cudaMemPool_t pool = device_pool();
    const cudaError_t e = pool ? cudaMallocFromPoolAsync(&p, b, pool, st()) : cudaMalloc(&p, b);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    ptrs.push_back({p, pool != nullptr});
    bytes += b;
    return p;
  }
  void release() {
    for (auto& q : ptrs) {
      if (q.second) cudaFreeAsync(q.first, st());
      else cudaFree(q.first);
    }
    ptrs.clear();
    bytes = 0;
  }
};

size_t xelem_bytes(int pol) {
  switch (pol) {
    case AJ_FP64: return 8;
    case AJ_DF64: return 8;
    default: return 4;
  }
}
size_t velem_bytes(int pol) {
  switch (pol) {
    case AJ_FP64: return 8;
    case AJ_DF64: return 8;
    case AJ_FP32_IR: return 4;
    default: return 2;
  }
}
// kernel policy id: 0 F64, 1 DF64, 2 F32, 3 BF16
int kernel_pol(int precision) { return precision; }

double pow2_near(double v) {
  // a power of two s with s * v in [1, 2) (v > 0); 1 for v = 0 or non-finite
  if (!(v > 0.0) || !std::isfinite(v)) return 1.0;
  int e = 0;
  std::frexp(v, &e);  // v = m * 2^e, m in [0.5, 1)
  return std::ldexp(1.0, 1 - e);
}

}  // namespace

namespace aj {
cudaError_t launch_persistent(int pol, int nrhs, const IterLaunch& L, int grid, cudaStream_t s) {
  switch (pol) {
    case 0: return launch_persistent_f64(nrhs, L, grid, s);
    case 1: return launch_persistent_df64(nrhs, L, grid, s);
    case 2: return launch_persistent_f32(nrhs, L, grid, s);
    case 3: return launch_persistent_b16(nrhs, L, grid, s);
  }
  return cudaErrorInvalidValue;
}
size_t iter_args_bytes() { return sizeof(IterArgs<PolF64>); }
void pack_iter_args(int pol, const IterLaunch& L, void* dst) {
  switch (pol) {
    case 0: pack_iter_args_f64(L, dst); break;
    case 1: pack_iter_args_df64(L, dst); break;
    case 2: pack_iter_args_f32(L, dst); break;
    case 3: pack_iter_args_b16(L, dst); break;
  }
}
cudaError_t launch_lockstep(int pol, int qx, const LockLaunch& B, int grid, cudaStream_t s) {
  switch (pol) {
    case 0: return launch_lockstep_f64(qx, B, grid, s);
    case 1: return launch_lockstep_df64(qx, B, grid, s);
    case 2: return launch_lockstep_f32(qx, B, grid, s);
    case 3: return launch_lockstep_b16(qx, B, grid, s);
  }
  return cudaErrorInvalidValue;
}
int lockstep_blocks_per_sm(int pol, int qx) {
  switch (pol) {
    case 0: return lockstep_blocks_per_sm_f64(qx);
    case 1: return lockstep_blocks_per_sm_df64(qx);
    case 2: return lockstep_blocks_per_sm_f32(qx);
    case 3: return lockstep_blocks_per_sm_b16(qx);
  }
  return 0;
}
int persistent_blocks_per_sm(int pol, int nrhs, int qx, int fm) {
  switch (pol) {
    case 0: return blocks_per_sm_f64(nrhs, qx, fm);
    case 1: return blocks_per_sm_df64(nrhs, qx, fm);
    case 2: return blocks_per_sm_f32(nrhs, qx, fm);
    case 3: return blocks_per_sm_b16(nrhs, qx, fm);
  }
  return 0;
}
}  // namespace aj

struct aj_ctx {
  int dev = 0;
  cudaStream_t stream = nullptr;
  int sm_count = 0;
  int64_t n = 0, nnz = 0;
  int nrhs = 1;
  Workspace base;  // lifetime of the context
  Workspace pws;   // rebuilt by aj_set
  int* rp = nullptr;
  int* ci = nullptr;
  double* val64 = nullptr;
  double* diag = nullptr;
  double* b64 = nullptr;  // interleaved
  double* jinv64 = nullptr;
  double bnorm2[kMaxRhs] = {0, 0, 0, 0};
  aj_params prm;
  bool have_prm = false;
  int pol = -1;
  void* valp = nullptr;
  void* bp = nullptr;
  void* jinvp = nullptr;
  void* x[3] = {nullptr, nullptr, nullptr};
  void* u[2] = {nullptr, nullptr};  // Q x^t, Q x^{t-1} (stored sweep forms); y^t, y^{t+1} (explicit y)
  void* dl = nullptr;               // x^t - x^{t-1} (difference sweep form)
  // SELL-C-sigma copy of Q (fmt = 1), rebuilt by aj_set
  Workspace sws;
  int fmt = 0, sell_sigma = 0, sell_lmax = 0, sell_cl = 5;
  int ctas_cap = 0;   // CTAs per SM the autotuner chose (0: the kernel's occupancy)
  int tuned = 0;      // 1 when the format and grid came from timing (or its cache)
  int sdim = 0, sN = 0;  // stencil format (fmt = 2): dimensions and grid side
  // block-diagonal J (eq. J-blkdiag, jblk > 1 rows per block): row k of each
  // block's inverse in FP64 and in the iteration precision, rebuilt by aj_set
  Workspace bws;
  int jblk = 1;
  double* jb64 = nullptr;
  void* jbp = nullptr;
  double fill = 1.0;
  int nsell = 0, ntiles_sell = 0, nltiles = 0, nhuge = 0;
  int *d_perm = nullptr, *d_rlen = nullptr, *d_sptr = nullptr, *d_scol = nullptr;
  int *d_long = nullptr, *d_ltp = nullptr, *d_huge = nullptr;
  void* d_sval = nullptr;
  int qx = 0;                       // sweep form in use: 0 lazy, 1 stored, 2 difference, 3 explicit y
  double sQ = 1.0;
  double sb[kMaxRhs] = {1, 1, 1, 1};
  double L_used = 0.0;
  int grid = 1;
  int part_cap = 0;  // CTAs the partial-sum buffer holds
  double* partials = nullptr;
  unsigned long long* bar = nullptr;
  int* err = nullptr;
  RhsState* state = nullptr;
  long long* rlog = nullptr;
  int rlog_cap = 64;
  double* part_small = nullptr;
  int part_small_n = 0;
  double* x64 = nullptr;
  double* r64 = nullptr;
  double* tmp64 = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr, kev0 = nullptr, kev1 = nullptr;
  double kernel_ms = 0.0;  // fused-kernel device time of the current solve
  bool resume = false;
  std::vector<RhsState> st_h;
  std::vector<std::vector<long long>> rlog_h;
  // locality ordering (aj_set, AJ_REORDER_*): while `ordered`, rp, ci, val64,
  // diag and b64 point at renumbered copies in ows; the caller's order stays
  // in rp0 .. b0
  Workspace ows;
  int ordered = 0;
  bool order_tried = false;  // AUTO already evaluated for this matrix
  double span0 = 0.0, span1 = 0.0;
  int* rp0 = nullptr;
  int* ci0 = nullptr;
  double* val0 = nullptr;
  double* diag0 = nullptr;
  double* b0 = nullptr;
  int* perm = nullptr;      // device [n]: new row -> caller's row
  std::vector<int> perm_h;  // host copy
  // rows longer than kResidLong entries, in the run's order, for the FP64
  // residual's warp-per-row pass (rebuilt when the order changes)
  int maxlen = 0;
  Workspace rws;
  int* d_resid_long = nullptr;
  int n_resid_long = 0;
  double* part_long = nullptr;
  int resid_long_order = -1;  // `ordered` the list was built for
};

static const int kResidLong = 32;
// eq. J-blkdiag: longest row accepted (the setup thread of a block scans its
// entries once per neighbouring block)
static const int kBlkMaxRow = 1024;

static aj_status cuda_fail(cudaError_t e) {
  (void)e;
  cudaGetLastError();
  return AJ_ECUDA;
}
#define CK(expr)                                      \
  do {                                                \
    cudaError_t _e = (expr);                          \
    if (_e != cudaSuccess) return cuda_fail(_e);      \
  } while (0)

extern "C" void aj_params_default(aj_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->j_policy = AJ_J_ABSROWSUM;
  p->L = 0.0;
  p->L_margin = 0.02;
  p->restart = AJ_RESTART_ADAPTIVE;
  p->momentum = 1;
  p->K0 = 2;
  p->tol = 1e-8;
  p->stop = AJ_STOP_RELRES;
  p->fstar = 0.0;
  p->maxit = 100000;
  p->precision = AJ_FP64;
  p->format = AJ_FMT_AUTO;
  p->x0 = nullptr;
  p->x0_on_device = 0;
  p->inner_tol = 1e-4;
  p->max_outer = 30;
  p->grid_ctas = 0;
  p->sweep_form = AJ_SWEEP_AUTO;
  p->sell_sigma = 0;
  p->sell_lmax = 0;
}

extern "C" const char* aj_strerror(aj_status s) {
  switch (s) {
    case AJ_OK: return "ok";
    case AJ_EINVAL: return "invalid argument or matrix";
    case AJ_ENOMEM: return "out of memory";
    case AJ_ECUDA: return "CUDA runtime error";
    case AJ_EMAXIT: return "iteration limit reached";
    case AJ_EDIVERGED: return "diverged (S = J - Q not positive semidefinite?)";
    case AJ_ENONFINITE: return "non-finite value in a reduction";
    case AJ_ETIMEOUT: return "device barrier timed out";
    case AJ_EBUSY: return "request larger than the server budget";
    case AJ_PENDING: return "pending";
  }
  return "unknown status";
}

extern "C" void aj_destroy(aj_ctx* c) {
  if (!c) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(c->dev);
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  c->sws.release();
  c->bws.release();
  c->pws.release();
  c->ows.release();
  c->rws.release();
  c->base.release();
  // the frees above are stream-ordered: wait for them, so that the pool can
  // hand the memory to the next allocation on any stream at once instead of
  // mapping new memory (aj_create of a 256^3 system took 41-51 ms instead of
  // 9 ms when it followed a context freed on the legacy stream)
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  if (c->kev0) cudaEventDestroy(c->kev0);
  if (c->kev1) cudaEventDestroy(c->kev1);
  cudaSetDevice(cur);
  delete c;
}

// Sum the first `blocks` rows of a [blocks][w] partial array on the host (fixed order).
static aj_status host_sum_parts(aj_ctx* c, const double* dpart, int blocks, int w, double* out) {
  std::vector<double> h((size_t)blocks * w);
  CK(cudaMemcpyAsync(h.data(), dpart, h.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  for (int k = 0; k < w; k++) out[k] = 0.0;
  for (int b = 0; b < blocks; b++)
    for (int k = 0; k < w; k++) out[k] += h[(size_t)b * w + k];
  return AJ_OK;
}

// 1: aj_create prints the host time of its phases to stderr (a diagnostic build)
#ifndef AJ_TRACE_CREATE
#define AJ_TRACE_CREATE 0
#endif
static double trace_now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

extern "C" aj_status aj_create(const aj_csr* Q, const double* b, int nrhs, aj_ctx** out) {
  if (!out) return AJ_EINVAL;
  const double tr0 = AJ_TRACE_CREATE ? trace_now_ms() : 0.0;
  *out = nullptr;
  if (!Q || nrhs < 1 || nrhs > kMaxRhs || Q->n < 0 || Q->nnz < 0) return AJ_EINVAL;
  if (Q->n >= (1ll << 31) - 1 || Q->nnz >= (1ll << 31) - 1) return AJ_EINVAL;
  if (Q->n > 0 && (!Q->row_ptr || !b)) return AJ_EINVAL;
  if (Q->nnz > 0 && (!Q->col || !Q->val)) return AJ_EINVAL;
  aj_ctx* c = new aj_ctx();
  aj_params_default(&c->prm);
  c->base.stream = c->pws.stream = c->sws.stream = c->ows.stream = c->rws.stream = c->bws.stream = &c->stream;
  cudaGetDevice(&c->dev);
  cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->dev);
  c->n = Q->n;
  c->nnz = Q->nnz;
  c->nrhs = nrhs;
  const int n = (int)Q->n;
  const long long nnz = Q->nnz;
  const long long m = (long long)n * nrhs;
  // One pool allocation holds all of them, each array 256-byte aligned: the
  // next context of the same size then reuses this one freed block (nine
  // separate blocks left the pool mapping new memory for most of them, 23-58
  // ms of a 256^3 system's creation against 9 ms).  Matrix arrays are padded
  // by 16 entries so 16-byte vector reads never leave them.
  c->part_small_n = std::max<int>(1, (int)grid1d(std::max<long long>(n, 1)));
  size_t off = 0;
  auto carve = [&](size_t bytes) {
    const size_t o = off;
    off += (bytes + 255) & ~(size_t)255;
    return o;
  };
  const size_t o_rp = carve((size_t)(n + 1 + 16) * 4);
  const size_t o_ci = carve((size_t)(nnz + 16) * 4);
  const size_t o_val = carve((size_t)(nnz + 16) * 8);
  const size_t o_diag = carve((size_t)(n + 1) * 8);
  const size_t o_b = carve((size_t)(m + 1) * 8);
  const size_t o_jinv = carve((size_t)(n + 1) * 8);
  const size_t o_tmp = carve((size_t)(m + 1) * 8);
  const size_t o_part = carve((size_t)c->part_small_n * kMaxRhs * 3 * 8);
  const size_t o_err = carve(64);
  char* blk = (char*)c->base.alloc(off);
  if (!blk) {
    aj_destroy(c);
    return AJ_ENOMEM;
  }
  if (AJ_TRACE_CREATE) {
    cudaStreamSynchronize(c->stream);
    fprintf(stderr, "aj_create alloc %.2f ms\n", trace_now_ms() - tr0);
  }
  c->rp = (int*)(blk + o_rp);
  c->ci = (int*)(blk + o_ci);
  c->val64 = (double*)(blk + o_val);
  c->diag = (double*)(blk + o_diag);
  c->b64 = (double*)(blk + o_b);
  c->jinv64 = (double*)(blk + o_jinv);
  c->tmp64 = (double*)(blk + o_tmp);
  c->part_small = (double*)(blk + o_part);
  c->err = (int*)(blk + o_err);
  if (cudaEventCreate(&c->ev0) != cudaSuccess || cudaEventCreate(&c->ev1) != cudaSuccess ||
      cudaEventCreate(&c->kev0) != cudaSuccess || cudaEventCreate(&c->kev1) != cudaSuccess) {
    aj_destroy(c);
    return AJ_ECUDA;
  }
  const cudaMemcpyKind kind = Q->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  cudaStream_t s = c->stream;
  aj_status st = AJ_OK;
  do {
    if (cudaMemcpyAsync(c->rp, Q->row_ptr, (size_t)(n + 1) * 4, kind, s) != cudaSuccess ||
        (nnz > 0 && cudaMemcpyAsync(c->ci, Q->col, (size_t)nnz * 4, kind, s) != cudaSuccess) ||
        (nnz > 0 && cudaMemcpyAsync(c->val64, Q->val, (size_t)nnz * 8, kind, s) != cudaSuccess) ||
        cudaMemsetAsync(c->ci + nnz, 0, 16 * 4, s) != cudaSuccess ||
        cudaMemsetAsync(c->val64 + nnz, 0, 16 * 8, s) != cudaSuccess ||
        cudaMemcpyAsync(c->tmp64, b, (size_t)m * 8, kind, s) != cudaSuccess ||
        cudaMemsetAsync(c->err, 0, 64, s) != cudaSuccess) {
      st = cuda_fail(cudaGetLastError());
      break;
    }
    if (AJ_TRACE_CREATE) {
      cudaStreamSynchronize(s);
      fprintf(stderr, "aj_create copies %.2f ms\n", trace_now_ms() - tr0);
    }
    k_check_rowptr<<<grid1d((long long)n + 1), kSetupThreads, 0, s>>>(n, nnz, c->rp, c->err);
    counted();
    int flags = 0;
    if (cudaMemcpyAsync(&flags, c->err, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      st = cuda_fail(cudaGetLastError());
      break;
    }
    if (flags) { st = AJ_EINVAL; break; }
    if (n > 0) {
      k_check_rows<<<grid1d(n), kSetupThreads, 0, s>>>(n, c->rp, c->ci, c->val64, c->diag, c->err);
      counted();
    }
    if (m > 0) {
      k_interleave<<<grid1d(m), kSetupThreads, 0, s>>>(n, nrhs, c->tmp64, c->b64);
      counted();
    }
    if (cudaMemcpyAsync(&flags, c->err, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      st = cuda_fail(cudaGetLastError());
      break;
    }
    if (flags) { st = AJ_EINVAL; break; }
    // longest row (c->err is zero again: flags was 0)
    if (n > 0) {
      k_max_row_len<<<std::min<unsigned>(grid1d(n), 4096), kSetupThreads, 0, s>>>(n, c->rp, c->err);
      counted();
      if (cudaMemcpyAsync(&c->maxlen, c->err, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
          cudaMemsetAsync(c->err, 0, 4, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
        st = cuda_fail(cudaGetLastError());
        break;
      }
    }
    // ||b_r||^2 in FP64 and b finite, on the device (c->err is zero here)
    if (n > 0) {
      const int blocks = (int)grid1d(n);
      k_bnorm2<<<blocks, kSetupThreads, 0, s>>>(n, nrhs, c->b64, c->part_small, c->err);
      counted();
      int bad = 0;
      double sums[kMaxRhs] = {0.0, 0.0, 0.0, 0.0};
      if (cudaGetLastError() != cudaSuccess || cudaMemcpyAsync(&bad, c->err, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
          cudaMemsetAsync(c->err, 0, 4, s) != cudaSuccess || host_sum_parts(c, c->part_small, blocks, nrhs, sums) != AJ_OK) {
        st = cuda_fail(cudaGetLastError());
        break;
      }
      if (bad) { st = AJ_EINVAL; break; }
      for (int r = 0; r < nrhs; r++) c->bnorm2[r] = sums[r];
    }
  } while (0);
  if (st != AJ_OK) {
    aj_destroy(c);
    return st;
  }
  c->rp0 = c->rp;
  c->ci0 = c->ci;
  c->val0 = c->val64;
  c->diag0 = c->diag;
  c->b0 = c->b64;
  if (AJ_TRACE_CREATE) fprintf(stderr, "aj_create done %.2f ms\n", trace_now_ms() - tr0);
  *out = c;
  return AJ_OK;
}

extern "C" aj_status aj_set_stream(aj_ctx* c, void* stream) {
  if (!c) return AJ_EINVAL;
  // the context's memory was allocated in the order of its old stream
  if (c->stream != (cudaStream_t)stream && cudaStreamSynchronize(c->stream) != cudaSuccess)
    return cuda_fail(cudaGetLastError());
  c->stream = (cudaStream_t)stream;
  return AJ_OK;
}

// Power iteration for lambda_max(D^-1/2 Q D^-1/2) in FP64 (setup step; a few
// hundred kernel launches at most).
static aj_status estimate_L(aj_ctx* c, double* L_out) {
  const int n = (int)c->n;
  cudaStream_t s = c->stream;
  if (n == 0) { *L_out = 1.0; return AJ_OK; }
  double* v = c->tmp64;
  double* w = c->jinv64;  // scratch: J^{-1} is rebuilt after the estimate
  // deterministic start vector: 1 + small index-dependent perturbation
  std::vector<double> h(n);
  for (int i = 0; i < n; i++) h[i] = 1.0 + 0.25 * std::sin(0.7 * i + 0.3);
  CK(cudaMemcpyAsync(v, h.data(), (size_t)n * 8, cudaMemcpyHostToDevice, s));
  double nv = 0.0;
  for (double q : h) nv += q * q;
  k_scale<<<grid1d(n), kSetupThreads, 0, s>>>(n, v, 1.0 / std::sqrt(nv));
  counted();
  const int blocks = (int)grid1d(n);
  double lam = 0.0;
  for (int it = 0; it < 300; it++) {
    k_normalized_spmv<<<blocks, kSetupThreads, 0, s>>>(n, c->rp, c->ci, c->val64, c->diag, v, w,
                                                       c->part_small);
    counted();
    double sums[2];
    aj_status st = host_sum_parts(c, c->part_small, blocks, 2, sums);
    if (st != AJ_OK) return st;
    const double lam_new = sums[0];  // Rayleigh quotient with ||v|| = 1
    const double wn = std::sqrt(sums[1]);
    if (!(wn > 0.0) || !std::isfinite(wn)) break;
    std::swap(v, w);
    k_scale<<<grid1d(n), kSetupThreads, 0, s>>>(n, v, 1.0 / wn);
    counted();
    const bool conv = it > 10 && std::fabs(lam_new - lam) <= 1e-7 * std::fabs(lam_new);
    lam = lam_new;
    if (conv) break;
  }
  // a Gershgorin bound is always safe; never exceed it
  k_gershgorin<<<blocks, kSetupThreads, 0, s>>>(n, c->rp, c->ci, c->val64, c->diag, c->part_small);
  counted();
  std::vector<double> hg(blocks);
  CK(cudaMemcpyAsync(hg.data(), c->part_small, (size_t)blocks * 8, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  double gb = 0.0;
  for (double g : hg) gb = std::max(gb, g);
  double L = (1.0 + c->prm.L_margin) * lam;
  if (gb > 0.0) L = std::min(L, gb);
  if (!(L > 0.0)) L = gb > 0.0 ? gb : 1.0;
  *L_out = L;
  return AJ_OK;
}

// ---------------------------------------------------------------- locality ordering
// Reverse Cuthill-McKee order of the graph of Q (rows as vertices, stored
// entries as edges; George and Liu 1981): in each connected component a
// breadth-first search starts from a pseudo-peripheral vertex (repeat the
// search from a least-degree vertex of the last level while the depth
// grows), visits the neighbours of each vertex by increasing degree, and the
// whole order is reversed.  perm[new] = old.
static void rcm_order(int n, const std::vector<int>& rp, const std::vector<int>& ci, std::vector<int>& perm) {
  std::vector<int> deg(n), mark(n, -1), queue;
  for (int i = 0; i < n; i++) deg[i] = rp[i + 1] - rp[i];
  queue.reserve(n);
  int stamp = 0;
  // levels of a BFS from r (marks vertices with this stamp); returns depth and last level
  auto bfs_levels = [&](int r, std::vector<int>& last) {
    const int st = stamp++;
    std::vector<int> cur(1, r), nxt;
    mark[r] = st;
    int depth = 0;
    for (;;) {
      nxt.clear();
      for (int v : cur)
        for (int q = rp[v]; q < rp[v + 1]; q++) {
          const int u = ci[q];
          if (mark[u] != st) { mark[u] = st; nxt.push_back(u); }
        }
      if (nxt.empty()) break;
      cur.swap(nxt);
      depth++;
    }
    last = cur;
    return depth;
  };
  std::vector<char> done(n, 0);
  std::vector<int> order, last, nb;
  order.reserve(n);
  for (int s0 = 0; s0 < n; s0++) {
    if (done[s0]) continue;
    int root = s0, ecc = -1;
    for (int it = 0; it < 6; it++) {
      const int d = bfs_levels(root, last);
      if (d <= ecc) break;
      ecc = d;
      int best = last[0];
      for (int v : last) if (deg[v] < deg[best] || (deg[v] == deg[best] && v < best)) best = v;
      root = best;
    }
    // Cuthill-McKee from root
    size_t head = order.size();
    order.push_back(root);
    done[root] = 1;
    while (head < order.size()) {
      const int v = order[head++];
      nb.clear();
      for (int q = rp[v]; q < rp[v + 1]; q++) {
        const int u = ci[q];
        if (!done[u]) { done[u] = 1; nb.push_back(u); }
      }
      std::sort(nb.begin(), nb.end(), [&](int x, int y) { return deg[x] < deg[y] || (deg[x] == deg[y] && x < y); });
      order.insert(order.end(), nb.begin(), nb.end());
    }
  }
  perm.assign(order.rbegin(), order.rend());
}

// Summed row spans (largest minus smallest column) with columns renamed by
// iperm (identity when empty).
static double row_spans(int n, const std::vector<int>& rp, const std::vector<int>& ci, const std::vector<int>& iperm) {
  double tot = 0.0;
  for (int i = 0; i < n; i++) {
    int lo = INT_MAX, hi = -1;
    for (int q = rp[i]; q < rp[i + 1]; q++) {
      const int c = iperm.empty() ? ci[q] : iperm[ci[q]];
      lo = std::min(lo, c);
      hi = std::max(hi, c);
    }
    if (hi >= lo) tot += (double)(hi - lo);
  }
  return tot;
}

// Orderings already computed, keyed by the matrix's pattern (n, nnz and a
// 64-bit hash of row_ptr and col), so that a server that sees the same
// operator again, or a caller that builds several contexts of one matrix,
// skips the host-side search.  Any permutation of the rows is a valid
// ordering, so a hash collision could cost locality but never accuracy.
struct OrderEntry {
  bool use = false;  // AUTO's decision
  double span0 = 0.0, span1 = 0.0;
  std::vector<int> perm;
};
static std::map<std::tuple<int64_t, int64_t, uint64_t>, OrderEntry> g_order;
static std::deque<std::tuple<int64_t, int64_t, uint64_t>> g_order_fifo;
static std::mutex g_order_mu;
static const size_t kOrderCacheEntries = 64;

static uint64_t pattern_hash(const std::vector<int>& rp, const std::vector<int>& ci) {
  uint64_t h = 0x9e3779b97f4a7c15ull;
  auto mix = [&](uint64_t v) {
    h ^= v + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2);
    h *= 0xbf58476d1ce4e5b9ull;
    h ^= h >> 31;
  };
  for (int v : rp) mix((uint32_t)v);
  for (int v : ci) mix((uint32_t)v);
  return h;
}

// Back to the caller's row order.
static void order_drop(aj_ctx* c) {
  c->rp = c->rp0;
  c->ci = c->ci0;
  c->val64 = c->val0;
  c->diag = c->diag0;
  c->b64 = c->b0;
  c->ows.release();
  c->perm = nullptr;
  c->perm_h.clear();
  c->ordered = 0;
}

// Renumbered copies of the matrix, its diagonal and b for perm (host, new ->
// old); the context then runs in that order.
static aj_status order_apply(aj_ctx* c, const std::vector<int>& perm, const std::vector<int>& rp) {
  const int n = (int)c->n;
  const long long nnz = c->nnz;
  const int nrhs = c->nrhs;
  cudaStream_t s = c->stream;
  order_drop(c);
  std::vector<int> iperm(n), rp1((size_t)n + 1);
  rp1[0] = 0;
  for (int i = 0; i < n; i++) {
    iperm[perm[i]] = i;
    rp1[i + 1] = rp1[i] + (rp[perm[i] + 1] - rp[perm[i]]);
  }
  int* d_perm = (int*)c->ows.alloc((size_t)(n + 1) * 4);
  int* d_iperm = (int*)c->ows.alloc((size_t)(n + 1) * 4);
  int* rp_o = (int*)c->ows.alloc((size_t)(n + 1 + 16) * 4);
  int* ci_o = (int*)c->ows.alloc((size_t)(nnz + 16) * 4);
  double* val_o = (double*)c->ows.alloc((size_t)(nnz + 16) * 8);
  double* diag_o = (double*)c->ows.alloc((size_t)(n + 1) * 8);
  double* b_o = (double*)c->ows.alloc((size_t)((long long)n * nrhs + 1) * 8);
  if (!d_perm || !d_iperm || !rp_o || !ci_o || !val_o || !diag_o || !b_o) {
    c->ows.release();
    return AJ_ENOMEM;
  }
  CK(cudaMemcpyAsync(d_perm, perm.data(), (size_t)n * 4, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(d_iperm, iperm.data(), (size_t)n * 4, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(rp_o, rp1.data(), (size_t)(n + 1) * 4, cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(ci_o + nnz, 0, 16 * 4, s));
  CK(cudaMemsetAsync(val_o + nnz, 0, 16 * 8, s));
  if (n > 0) {
    k_permute_csr<<<(unsigned)(((long long)n * 32 + kSetupThreads - 1) / kSetupThreads), kSetupThreads, 0, s>>>(
        n, d_perm, d_iperm, c->rp0, c->ci0, c->val0, rp_o, ci_o, val_o);
    counted();
    k_gather_rows<<<grid1d(n), kSetupThreads, 0, s>>>(n, 1, d_perm, c->diag0, diag_o);
    counted();
    k_gather_rows<<<grid1d((long long)n * nrhs), kSetupThreads, 0, s>>>(n, nrhs, d_perm, c->b0, b_o);
    counted();
  }
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  c->rp = rp_o;
  c->ci = ci_o;
  c->val64 = val_o;
  c->diag = diag_o;
  c->b64 = b_o;
  c->perm = d_perm;
  c->perm_h = perm;
  c->ordered = 1;
  return AJ_OK;
}

// The row order aj_set asks for (see AJ_REORDER_* in aj.h).
static aj_status choose_order(aj_ctx* c, int mode) {
  if (mode == AJ_REORDER_NONE) {
    if (c->ordered) order_drop(c);
    return AJ_OK;
  }
  if (c->ordered) return AJ_OK;                          // already renumbered
  if (mode == AJ_REORDER_AUTO && c->order_tried) return AJ_OK;  // evaluated before: keep the caller's order
  const int n = (int)c->n;
  if (n < 2 || c->nnz == 0) return AJ_OK;
  cudaStream_t s = c->stream;
  if (mode == AJ_REORDER_AUTO) {
    c->order_tried = true;
    const double mean = (double)c->nnz / n;
    if (n < 16384 || c->maxlen > 16.0 * mean + 16.0) return AJ_OK;
    // rows that already gather from a small part of x on average (a natural
    // stencil order spans 2 N^(d-1) of n = N^d) keep the caller's order; the
    // summed spans come from a device pass, so such matrices cost no copy
    const int blocks = (int)grid1d(n);
    Workspace tmp;
    tmp.stream = &c->stream;
    double* part = (double*)tmp.alloc((size_t)blocks * 8);
    if (!part) return AJ_ENOMEM;
    k_row_spans<<<blocks, kSetupThreads, 0, s>>>(n, c->rp0, c->ci0, part);
    counted();
    double span = 0.0;
    aj_status e = host_sum_parts(c, part, blocks, 1, &span);
    tmp.release();
    if (e != AJ_OK) return e;
    c->span0 = c->span1 = span;
    if (span <= (double)n * (n / 8.0)) return AJ_OK;
  }
  std::vector<int> rp((size_t)n + 1);
  CK(cudaMemcpyAsync(rp.data(), c->rp0, rp.size() * 4, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  std::vector<int> ci((size_t)c->nnz);
  CK(cudaMemcpyAsync(ci.data(), c->ci0, ci.size() * 4, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  const auto key = std::make_tuple(c->n, c->nnz, pattern_hash(rp, ci));
  OrderEntry ent;
  bool hit = false;
  {
    std::lock_guard<std::mutex> lk(g_order_mu);
    auto it = g_order.find(key);
    if (it != g_order.end() && (it->second.use || mode == AJ_REORDER_AUTO)) {
      ent = it->second;
      hit = true;
    }
  }
  (hit ? g_order_hits : g_order_misses).fetch_add(1);
  if (!hit) {
    const std::vector<int> none;
    ent.span0 = ent.span1 = row_spans(n, rp, ci, none);
    if (mode == AJ_REORDER_RCM || ent.span0 > (double)n * (n / 8.0)) {
      rcm_order(n, rp, ci, ent.perm);
      std::vector<int> iperm(n);
      for (int i = 0; i < n; i++) iperm[ent.perm[i]] = i;
      ent.span1 = row_spans(n, rp, ci, iperm);
      ent.use = ent.span1 * 4.0 <= ent.span0;
    }
    std::lock_guard<std::mutex> lk(g_order_mu);
    if (!g_order.count(key)) {
      if (g_order_fifo.size() >= kOrderCacheEntries) {
        g_order.erase(g_order_fifo.front());
        g_order_fifo.pop_front();
      }
      g_order_fifo.push_back(key);
    }
    g_order[key] = ent;
  }
  c->span0 = ent.span0;
  c->span1 = ent.span1;
  if (mode == AJ_REORDER_AUTO && !ent.use) return AJ_OK;
  return order_apply(c, ent.perm, rp);
}

extern "C" aj_status aj_get_order(aj_ctx* c, int* reordered, double* span_before, double* span_after) {
  if (!c) return AJ_EINVAL;
  if (reordered) *reordered = c->ordered;
  if (span_before) *span_before = c->span0;
  if (span_after) *span_after = c->span1;
  return AJ_OK;
}

static aj_status choose_format(aj_ctx* c, const aj_params* p);

// The persistent grid for the current format and sweep form: one CTA per
// tile up to the co-resident limit (SELL counts its sliced, long-row and
// huge-row tiles), or the caller's grid_ctas.
static void size_grid(aj_ctx* c) {
  // the instantiation the launch takes: the stencil rows alone, CSR alone, or any
  const int fm = c->fmt == 2 ? 2 : c->jblk > 1 ? 1 : c->fmt == 1 ? (c->sell_cl < 5 ? 4 : AJ_SELL_FM) : 0;
  int bps = std::max(1, persistent_blocks_per_sm(kernel_pol(c->pol), c->nrhs, c->qx, fm));
  if (c->ctas_cap > 0) bps = std::min(bps, c->ctas_cap);
  const long long rpt = kThreads >> lanes_log2(c->nrhs);
  const long long ntiles = c->fmt == 1 ? (long long)c->ntiles_sell + c->nltiles + c->nhuge
                                       : (c->n + rpt - 1) / rpt;
  long long g = std::min<long long>((long long)bps * c->sm_count, std::max<long long>(1, ntiles));
  if (c->prm.grid_ctas > 0) g = std::min<long long>(c->prm.grid_ctas, (long long)bps * c->sm_count);
  c->grid = (int)std::max<long long>(1, g);
}

// (Re)build everything that depends on the parameters.
extern "C" aj_status aj_set(aj_ctx* c, const aj_params* p) {
  if (!c || !p) return AJ_EINVAL;
  if (p->j_policy != AJ_J_ABSROWSUM && p->j_policy != AJ_J_SCALED_DIAG && p->j_policy != AJ_J_BLKDIAG)
    return AJ_EINVAL;
  const int jblk = p->j_policy != AJ_J_BLKDIAG ? 1 : p->j_block == 0 ? 4 : p->j_block;
  if (p->j_policy == AJ_J_BLKDIAG && jblk != 1 && jblk != 2 && jblk != 4 && jblk != 8) return AJ_EINVAL;
  if (jblk > 1 && (p->format == AJ_FMT_SELL || p->reorder == AJ_REORDER_RCM)) return AJ_EINVAL;
  if (p->restart != AJ_RESTART_NONE && p->restart != AJ_RESTART_ADAPTIVE) return AJ_EINVAL;
  if (p->K0 < 2 || p->maxit < 0 || !(p->tol >= 0.0) || p->L < 0.0 || !(p->L_margin >= 0.0))
    return AJ_EINVAL;
  if (p->stop < AJ_STOP_RELRES || p->stop > AJ_STOP_NONE) return AJ_EINVAL;
  if (p->precision < AJ_FP64 || p->precision > AJ_BF16_IR) return AJ_EINVAL;
  if (p->format < AJ_FMT_AUTO || p->format > AJ_FMT_STENCIL) return AJ_EINVAL;
  if (p->grid_ctas < 0) return AJ_EINVAL;
  if (p->sweep_form < AJ_SWEEP_AUTO || p->sweep_form > AJ_SWEEP_Y) return AJ_EINVAL;
  if (p->sweep_form == AJ_SWEEP_DELTA && p->precision != AJ_FP64) return AJ_EINVAL;
  if (p->sweep_form == AJ_SWEEP_Y && p->stop == AJ_STOP_OBJGAP) return AJ_EINVAL;
  if (p->sell_sigma < 0 || p->sell_lmax < 0) return AJ_EINVAL;
  if (p->sell_c != 0 && p->sell_c != 8 && p->sell_c != 16 && p->sell_c != 32) return AJ_EINVAL;
  if (p->reorder < AJ_REORDER_AUTO || p->reorder > AJ_REORDER_RCM) return AJ_EINVAL;
  if ((p->precision == AJ_FP32_IR || p->precision == AJ_BF16_IR) &&
      (!(p->inner_tol > 0.0) || p->max_outer < 1))
    return AJ_EINVAL;
  const int old_pol = c->pol;
  c->prm = *p;
  // until this call succeeds the context counts as never set: a solve then
  // runs aj_set with the defaults first, as on a fresh context
  c->have_prm = false;
  c->resume = false;
  const int n = (int)c->n;
  const long long nnz = c->nnz;
  const int nrhs = c->nrhs;
  const long long m = (long long)n * nrhs;
  cudaStream_t s = c->stream;
  // --- row order (before anything is derived from the matrix)
  {
    const int was = c->ordered;
    aj_status st = choose_order(c, jblk > 1 ? AJ_REORDER_NONE : p->reorder);
    if (st != AJ_OK) return st;
    if (was != c->ordered) c->sws.release(), c->fmt = 0;
  }
  // --- J^{-1} in FP64
  double L = 0.0;
  if (p->j_policy == AJ_J_SCALED_DIAG) {
    L = p->L;
    if (L == 0.0) {
      aj_status st = estimate_L(c, &L);
      if (st != AJ_OK) return st;
    }
  }
  c->L_used = L;
  if (n > 0) {
    k_jinv<<<grid1d(n), kSetupThreads, 0, s>>>(n, c->rp, c->ci, c->val64, c->diag,
                                               p->j_policy == AJ_J_SCALED_DIAG ? 1 : 0, L, c->jinv64);
    counted();
  }
  CK(cudaGetLastError());
  // --- eq. J-blkdiag: the inverse of every block (eq. J-diag's inverse in
  // jinv64 stands in for blocks whose J^{ii} is singular)
  c->bws.release();
  c->jb64 = nullptr;
  c->jbp = nullptr;
  c->jblk = 1;
  if (jblk > 1 && n > 0) {
    if (c->maxlen > kBlkMaxRow) return AJ_EINVAL;
    const long long nblk = ((long long)n + jblk - 1) / jblk;
    c->jb64 = (double*)c->bws.alloc((size_t)(nblk * jblk * jblk + 16) * 8);
    if (!c->jb64) return AJ_ENOMEM;
    CK(cudaMemsetAsync(c->err, 0, 4, s));
    k_jblk<<<(unsigned)std::min<long long>((nblk + 127) / 128, 65535), 128, 0, s>>>(
        n, jblk, c->rp, c->ci, c->val64, c->jinv64, c->jb64, c->err);
    counted();
    int bad = 0;
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(&bad, c->err, 4, cudaMemcpyDeviceToHost, s));
    CK(cudaMemsetAsync(c->err, 0, 4, s));
    CK(cudaStreamSynchronize(s));
    if (bad) return AJ_EINVAL;
    c->jblk = jblk;
  }
  // --- precision-specific arrays
  const int pol = p->precision;
  if (pol != old_pol) {
    c->pws.release();
    c->pol = -1;  // set again once every array of the new precision exists
    c->valp = c->bp = c->jinvp = nullptr;
    c->x[0] = c->x[1] = c->x[2] = nullptr;
    c->u[0] = c->u[1] = nullptr;
    c->dl = nullptr;
    c->partials = nullptr;
    c->bar = nullptr;
    c->state = nullptr;
    c->rlog = nullptr;
    c->x64 = c->r64 = nullptr;
    const size_t xe = xelem_bytes(pol);
    if (pol != AJ_FP64) {
      c->valp = c->pws.alloc((size_t)(nnz + 16) * velem_bytes(pol));
      c->bp = c->pws.alloc((size_t)(m + 1) * xe);
      c->jinvp = c->pws.alloc((size_t)(n + 1) * xe);
      if (!c->valp || !c->bp || !c->jinvp) return AJ_ENOMEM;
    }
    for (int k = 0; k < 3; k++) {
      c->x[k] = c->pws.alloc((size_t)(m + 1) * xe);
      if (!c->x[k]) return AJ_ENOMEM;
    }
    for (int k = 0; k < 2; k++) {
      c->u[k] = c->pws.alloc((size_t)(m + 1) * xe);
      if (!c->u[k]) return AJ_ENOMEM;
    }
    c->dl = c->pws.alloc((size_t)(m + 1) * xe);
    if (!c->dl) return AJ_ENOMEM;
    c->x64 = (double*)c->pws.alloc((size_t)(m + 1) * 8);
    c->r64 = (double*)c->pws.alloc((size_t)(m + 1) * 8);
    if (!c->x64 || !c->r64) return AJ_ENOMEM;
    const int kp = kernel_pol(pol);
    int bps = 1;  // the largest grid any sweep form and format may take
    for (int q = 0; q < 4; q++)
      for (int f = 0; f < 5; f++) bps = std::max(bps, persistent_blocks_per_sm(kp, nrhs, q, f));
    const int maxg = bps * c->sm_count;
    c->partials = (double*)c->pws.alloc((size_t)2 * maxg * nrhs * kNRed * 8);
    c->part_cap = maxg;
    c->bar = (unsigned long long*)c->pws.alloc(64);
    c->state = (RhsState*)c->pws.alloc(sizeof(RhsState) * kMaxRhs);
    c->rlog = (long long*)c->pws.alloc((size_t)kMaxRhs * c->rlog_cap * 8);
    if (!c->partials || !c->bar || !c->state || !c->rlog) return AJ_ENOMEM;
    c->pol = pol;
  }
  // --- sweep form and grid: a multiple of the SM count when the problem is large enough
  // AUTO: for FP64 the explicit-y form with one right-hand side (the fewest
  // FP64 instructions per row: 256^3 Poisson 0.480 ms per sweep against 0.553
  // in the difference form), the difference form with several or with the
  // objective-gap stop; for the other precisions the stored form while the
  // format is chosen, then the lazy form on CSR (see the end of aj_set)
  const bool auto_y = p->precision == AJ_FP64 && p->stop != AJ_STOP_OBJGAP && nrhs == 1;
  c->qx = p->sweep_form == AJ_SWEEP_LAZY     ? 0
          : p->sweep_form == AJ_SWEEP_STORED ? 1
          : p->sweep_form == AJ_SWEEP_DELTA  ? 2
          : p->sweep_form == AJ_SWEEP_Y      ? 3
          : (p->precision == AJ_FP64 ? (auto_y ? 3 : 2) : 1);
  size_grid(c);
  // --- scaled copies for the non-FP64 policies (powers of two: exact)
  if (pol != AJ_FP64) {
    // max |Q_ij| via the diagonal bound: for SPSD Q, |Q_ij| <= sqrt(Q_ii Q_jj) <= max diag
    // (the diagonal is non-negative: aj_create rejects a negative one)
    double vmax = 0.0;
    if (n > 0) {
      unsigned long long* dm = (unsigned long long*)c->part_small;
      unsigned long long bits = 0ull;
      CK(cudaMemsetAsync(dm, 0, 8, s));
      k_max_nonneg<<<std::min<unsigned>(grid1d(n), 4096), kSetupThreads, 0, s>>>(n, c->diag, dm);
      counted();
      CK(cudaGetLastError());
      CK(cudaMemcpyAsync(&bits, dm, 8, cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      std::memcpy(&vmax, &bits, 8);
    }
    c->sQ = pow2_near(vmax);
    if (pol == AJ_DF64) {
      if (nnz > 0) {
        k_to_dw<<<grid1d(nnz), kSetupThreads, 0, s>>>(nnz, c->val64, c->sQ, (float2*)c->valp);
        counted();
      }
      if (n > 0) {
        k_to_dw<<<grid1d(n), kSetupThreads, 0, s>>>(n, c->jinv64, 1.0 / c->sQ, (float2*)c->jinvp);
        counted();
      }
      if (c->jblk > 1) {
        const long long nb = ((long long)n + c->jblk - 1) / c->jblk * c->jblk * c->jblk;
        c->jbp = c->bws.alloc((size_t)(nb + 16) * sizeof(float2));
        if (!c->jbp) return AJ_ENOMEM;
        k_to_dw<<<grid1d(nb), kSetupThreads, 0, s>>>(nb, c->jb64, 1.0 / c->sQ, (float2*)c->jbp);
        counted();
      }
    } else if (pol == AJ_FP32_IR) {
      if (nnz > 0) {
        k_to_f32<<<grid1d(nnz), kSetupThreads, 0, s>>>(nnz, c->val64, c->sQ, (float*)c->valp);
        counted();
      }
      if (n > 0) {
        k_to_f32<<<grid1d(n), kSetupThreads, 0, s>>>(n, c->jinv64, 1.0 / c->sQ, (float*)c->jinvp);
        counted();
      }
    } else {
      if (nnz > 0) {
        k_to_b16<<<grid1d(nnz), kSetupThreads, 0, s>>>(nnz, c->val64, c->sQ, (__nv_bfloat16*)c->valp);
        counted();
      }
      if (n > 0) {
        k_to_f32<<<grid1d(n), kSetupThreads, 0, s>>>(n, c->jinv64, 1.0 / c->sQ, (float*)c->jinvp);
        counted();
      }
    }
    CK(cudaGetLastError());
  } else {
    c->sQ = 1.0;
  }
  if (pol != AJ_FP64 && pol != AJ_DF64 && c->jblk > 1) {
    // FP32 and BF16 values: J^{-1} in FP32
    const long long nb = ((long long)n + c->jblk - 1) / c->jblk * c->jblk * c->jblk;
    c->jbp = c->bws.alloc((size_t)(nb + 16) * sizeof(float));
    if (!c->jbp) return AJ_ENOMEM;
    k_to_f32<<<grid1d(nb), kSetupThreads, 0, s>>>(nb, c->jb64, 1.0 / c->sQ, (float*)c->jbp);
    counted();
    CK(cudaGetLastError());
  }
  CK(cudaStreamSynchronize(s));
  aj_status fe = choose_format(c, p);
  if (fe != AJ_OK) return fe;
  // AUTO sweep form: the difference form for FP64 (one FMA per entry and one
  // FP64 instruction less per row: FP64 issue binds), stored for SELL
  // (irregular rows: one random gather per entry instead of two), lazy for
  // the other precisions on CSR, where the second row sum gathers from the
  // same cached lines and saves two n-vectors of traffic
  // (FP32 values in the stencil format: the explicit-y form, 0.187 against
  // 0.213 ms per 256^3 sweep lazy; it gathers one vector instead of two)
  if (p->sweep_form == AJ_SWEEP_AUTO && p->precision != AJ_FP64 && c->fmt != 1)
    c->qx = (c->fmt == 2 && p->precision == AJ_FP32_IR && c->nrhs == 1 && p->stop != AJ_STOP_OBJGAP) ? 3 : 0;
  size_grid(c);
  c->have_prm = true;
  return AJ_OK;
}

// Load interleaved FP64 data, scaled per right-hand side, into an
// iteration-precision buffer.
static void to_policy(aj_ctx* c, const double* src_il, void* dst, const double* scale_per_rhs) {
  const long long m = (long long)c->n * c->nrhs;
  if (m == 0) return;
  RhsMap mp;
  for (int r = 0; r < kMaxRhs; r++) {
    mp.s[r] = r < c->nrhs ? scale_per_rhs[r] : 1.0;
    mp.cur[r] = 0;
  }
  cudaStream_t s = c->stream;
  switch (c->pol) {
    case AJ_FP64: k_to_policy<double><<<grid1d(m), kSetupThreads, 0, s>>>(m, c->nrhs, src_il, mp, (double*)dst); counted(); break;
    case AJ_DF64: k_to_policy<float2><<<grid1d(m), kSetupThreads, 0, s>>>(m, c->nrhs, src_il, mp, (float2*)dst); counted(); break;
    default: k_to_policy<float><<<grid1d(m), kSetupThreads, 0, s>>>(m, c->nrhs, src_il, mp, (float*)dst); counted(); break;
  }
}

// Buffer cur[r] of each right-hand side, times scale[r], into an interleaved
// FP64 vector.
static aj_status from_policy(aj_ctx* c, const int* cur, const double* scale, double* dst_il) {
  const long long m = (long long)c->n * c->nrhs;
  if (m == 0) return AJ_OK;
  RhsMap mp;
  for (int r = 0; r < kMaxRhs; r++) {
    mp.s[r] = r < c->nrhs ? scale[r] : 1.0;
    mp.cur[r] = r < c->nrhs ? cur[r] : 0;
  }
  cudaStream_t s = c->stream;
  switch (c->pol) {
    case AJ_FP64:
      k_from_policy<double><<<grid1d(m), kSetupThreads, 0, s>>>(
          m, c->nrhs, (const double*)c->x[0], (const double*)c->x[1], (const double*)c->x[2], mp, dst_il);
      counted();
      break;
    case AJ_DF64:
      k_from_policy<float2><<<grid1d(m), kSetupThreads, 0, s>>>(
          m, c->nrhs, (const float2*)c->x[0], (const float2*)c->x[1], (const float2*)c->x[2], mp, dst_il);
      counted();
      break;
    default:
      k_from_policy<float><<<grid1d(m), kSetupThreads, 0, s>>>(
          m, c->nrhs, (const float*)c->x[0], (const float*)c->x[1], (const float*)c->x[2], mp, dst_il);
      counted();
      break;
  }
  CK(cudaGetLastError());
  return AJ_OK;
}

static void init_state(aj_ctx* c, RhsState* st, const double* bn2) {
  for (int r = 0; r < c->nrhs; r++) {
    RhsState& q = st[r];
    std::memset(&q, 0, sizeof(q));
    q.alpha = 1.0;
    q.beta = 0.0;
    q.bnorm2 = bn2[r];
    q.t = 0;
    q.ell = 0;
    q.K = c->prm.K0;
    q.Kre = 0;
    q.cur = 0;
    q.prev = 0;
    q.nxt = 1;
    q.done = 0;
    q.status = 0;
  }
}

// Run the persistent kernel to completion from state st (host copy, in/out).
// Kernel arguments of one context's persistent solve.
static IterLaunch make_launch(aj_ctx* c, const void* bvec, long long maxit, int stop, double tol,
                              double fstar, double fscale) {
  IterLaunch L;
  std::memset(&L, 0, sizeof(L));
  L.n = (int)c->n;
  L.nrhs = c->nrhs;
  L.row_ptr = c->rp;
  L.col = c->ci;
  L.val = c->pol == AJ_FP64 ? (const void*)c->val64 : c->valp;
  L.fmt = c->fmt;
  if (c->fmt == 2) {
    L.sdim = c->sdim;
    L.sN = c->sN;
    L.sdiag_at = 0;
    L.soff_at = 1;
    // division by N as a multiply and shift (Granlund and Montgomery, PLDI
    // 1994, Thm. 4.2 with 31-bit numerators): l = ceil(log2 N),
    // m = floor(2^(31+l) / N) + 1, then q / N = (q m) >> (31 + l)
    int l = 0;
    while ((1ll << l) < c->sN) l++;
    L.smag = (unsigned long long)((1ull << (31 + l)) / (unsigned long long)c->sN) + 1ull;
    L.sshift = 31 + l;
  }
  if (c->fmt == 1) {
    L.nsell = c->nsell;
    L.sell_cl = c->sell_cl;
    L.ntiles_sell = c->ntiles_sell;
    L.nltiles = c->nltiles;
    L.perm = c->d_perm;
    L.rlen = c->d_rlen;
    L.sptr = c->d_sptr;
    L.scol = c->d_scol;
    L.sval = c->d_sval;
    L.long_rows = c->d_long;
    L.ltp = c->d_ltp;
    L.nhuge = c->nhuge;
    L.huge_rows = c->d_huge;
  }
  L.b = bvec;
  L.jinv = c->pol == AJ_FP64 ? (const void*)c->jinv64 : c->jinvp;
  if (c->jblk > 1) L.jinv = c->pol == AJ_FP64 ? (const void*)c->jb64 : c->jbp;
  L.jblk = c->jblk;
  L.short_rows = c->maxlen <= kLongRow ? 1 : 0;
  for (int k = 0; k < 3; k++) L.x[k] = c->x[k];
  for (int k = 0; k < 2; k++) L.u[k] = c->u[k];
  L.dl = c->dl;
  L.qx = c->qx;
  L.partials = c->partials;
  L.bar = c->bar;
  L.err = c->err;
  L.state = c->state;
  L.rlog = c->rlog;
  L.rlog_cap = c->rlog_cap;
  L.trace = nullptr;
  L.trace_cap = 0;
  L.maxit = maxit;
  L.stop = stop;
  L.restart = c->prm.restart == AJ_RESTART_ADAPTIVE;
  L.momentum = c->prm.momentum != 0;
  L.tol = tol;
  L.fstar = fstar;
  L.fscale = fscale;
  L.max_sweeps = maxit + 2;
  return L;
}

// Upload the state of a run and clear its barrier, error word and restart log.
static aj_status stage_state(aj_ctx* c, const std::vector<RhsState>& st, bool log_restarts) {
  cudaStream_t s = c->stream;
  CK(cudaMemcpyAsync(c->state, st.data(), sizeof(RhsState) * c->nrhs, cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(c->bar, 0, 64, s));
  CK(cudaMemsetAsync(c->err, 0, 64, s));
  if (log_restarts) CK(cudaMemsetAsync(c->rlog, 0xff, (size_t)kMaxRhs * c->rlog_cap * 8, s));
  return AJ_OK;
}

// Run the persistent kernel to completion from state st (host copy, in/out).
static aj_status run_persistent(aj_ctx* c, std::vector<RhsState>& st, const void* bvec,
                                long long maxit, int stop, double tol, double fstar,
                                double fscale, bool log_restarts) {
  cudaStream_t s = c->stream;
  IterLaunch L = make_launch(c, bvec, maxit, stop, tol, fstar, fscale);
  const int stall = g_stall_cta.exchange(-1);
  if (stall >= 0) {
    L.bar_withhold = stall + 1;
    L.bar_timeout_ns = (unsigned long long)g_stall_timeout_ns.load();
  }
  aj_status e = stage_state(c, st, log_restarts);
  if (e != AJ_OK) return e;
  CK(cudaEventRecord(c->kev0, s));
  CK(launch_persistent(kernel_pol(c->pol), c->nrhs, L, c->grid, s));
  counted();
  CK(cudaEventRecord(c->kev1, s));
  int err = 0;
  CK(cudaMemcpyAsync(&err, c->err, 4, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(st.data(), c->state, sizeof(RhsState) * c->nrhs, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  float kms = 0.f;
  cudaEventElapsedTime(&kms, c->kev0, c->kev1);
  c->kernel_ms += kms;
  if (err != 0) return err == kETimeout ? AJ_ETIMEOUT : AJ_ECUDA;
  return AJ_OK;
}

// ---------------------------------------------------------------- matrix format
// SELL-C-sigma (C = 32) from the CSR arrays: rows longer than kHugeRow get a
// whole CTA each; rows longer than lmax go to the long-row bucket, sorted by
// length (longest first) and cut into tiles of at most 256 rows and
// kLongTileEntries entries, summed a warp per row; the others are sorted by
// length, longest first, within windows of sigma rows and sliced.
static const long long kLongTileEntries = 32768;
static const int kHugeRow = 4096;

template <class T>
static void sell_fill(aj_ctx* c, const void* val) {
  k_sell_fill<T><<<grid1d(c->nsell), kSetupThreads, 0, c->stream>>>(
      c->nsell, c->sell_cl, c->d_perm, c->d_rlen, c->d_sptr, c->rp, c->ci, (const T*)val, c->d_scol,
      (T*)c->d_sval);
  counted();
}

static aj_status build_sell(aj_ctx* c, int sigma, int lmax, int cl = 5) {
  c->sws.release();
  c->fmt = 0;
  c->fill = 1.0;
  if (c->nrhs > 1) cl = 5;  // several right-hand sides take the lanes of a row
  const int n = (int)c->n;
  const int rpt = kThreads >> lanes_log2(c->nrhs);  // rows per tile
  const int C = 1 << cl;                            // slice height
  const int rpt_sell = cl < 5 ? (kWarps << cl) : rpt;  // rows per sliced tile
  cudaStream_t s = c->stream;
  std::vector<int> rp((size_t)n + 1);
  CK(cudaMemcpyAsync(rp.data(), c->rp, rp.size() * 4, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  auto len = [&](int i) { return rp[i + 1] - rp[i]; };
  std::vector<int> rows, lng, hug;
  rows.reserve(n);
  for (int i = 0; i < n; i++) {
    const int l = len(i);
    (l > kHugeRow ? hug : l > lmax ? lng : rows).push_back(i);
  }
  std::stable_sort(lng.begin(), lng.end(), [&](int x, int y) { return len(x) > len(y); });
  for (size_t w0 = 0; w0 < rows.size(); w0 += (size_t)sigma) {
    auto b = rows.begin() + w0, e = rows.begin() + std::min(rows.size(), w0 + (size_t)sigma);
    std::stable_sort(b, e, [&](int x, int y) { return len(x) > len(y); });
  }
  const int nsell = (int)rows.size();
  const int nslices = (nsell + C - 1) / C;
  std::vector<int> rlen(nsell), sptr((size_t)nslices + 1);
  long long tot = 0;
  for (int sl = 0; sl < nslices; sl++) {
    int w = 0;
    for (int p = sl * C; p < std::min(nsell, sl * C + C); p++) {
      rlen[p] = len(rows[p]);
      w = std::max(w, rlen[p]);
    }
    sptr[sl] = (int)tot;
    tot += (long long)C * w;
    if (tot > (1ll << 31) - 64) return AJ_ENOMEM;
  }
  sptr[nslices] = (int)tot;
  std::vector<int> ltp(1, 0);
  // long-row tiles hold at most kLongTileEntries entries, fewer when that
  // would leave fewer tiles than SMs (a few rows of many entries): then
  // about eight tiles per SM, at least 4096 entries each
  long long long_total = 0;
  for (int r : lng) long_total += len(r);
  long long tile_cap = kLongTileEntries;
  if (long_total / kLongTileEntries < c->sm_count)
    tile_cap = std::max<long long>(4096, long_total / (8ll * c->sm_count));
  long long acc = 0, long_entries = 0;
  int cnt = 0;
  for (int j = 0; j < (int)lng.size(); j++) {
    const int l = len(lng[j]);
    if (cnt > 0 && (cnt == rpt || acc + l > tile_cap)) {
      ltp.push_back(j);
      acc = 0;
      cnt = 0;
    }
    acc += l;
    cnt++;
    long_entries += l;
  }
  if (!lng.empty()) ltp.push_back((int)lng.size());
  // the huge rows sorted longest first (one tile each); the long rows are
  // sorted longest first already
  std::stable_sort(hug.begin(), hug.end(), [&](int x, int y) { return len(x) > len(y); });
  const int ntsell = (nsell + rpt_sell - 1) / rpt_sell;
  const size_t vb = velem_bytes(c->pol);
  c->d_perm = (int*)c->sws.alloc(((size_t)nsell + 1) * 4);
  c->d_rlen = (int*)c->sws.alloc(((size_t)nsell + 1) * 4);
  c->d_sptr = (int*)c->sws.alloc(sptr.size() * 4);
  c->d_scol = (int*)c->sws.alloc(((size_t)tot + 32) * 4);
  c->d_sval = c->sws.alloc(((size_t)tot + 32) * vb);
  c->d_long = (int*)c->sws.alloc((lng.size() + 1) * 4);
  c->d_ltp = (int*)c->sws.alloc(ltp.size() * 4);
  c->d_huge = (int*)c->sws.alloc((hug.size() + 1) * 4);
  if (!c->d_perm || !c->d_rlen || !c->d_sptr || !c->d_scol || !c->d_sval || !c->d_long || !c->d_ltp ||
      !c->d_huge) {
    c->sws.release();
    return AJ_ENOMEM;
  }
  if (nsell) {
    CK(cudaMemcpyAsync(c->d_perm, rows.data(), (size_t)nsell * 4, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(c->d_rlen, rlen.data(), (size_t)nsell * 4, cudaMemcpyHostToDevice, s));
  }
  CK(cudaMemcpyAsync(c->d_sptr, sptr.data(), sptr.size() * 4, cudaMemcpyHostToDevice, s));
  if (!lng.empty()) CK(cudaMemcpyAsync(c->d_long, lng.data(), lng.size() * 4, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(c->d_ltp, ltp.data(), ltp.size() * 4, cudaMemcpyHostToDevice, s));
  if (!hug.empty()) CK(cudaMemcpyAsync(c->d_huge, hug.data(), hug.size() * 4, cudaMemcpyHostToDevice, s));
  for (int h : hug) long_entries += len(h);
  CK(cudaMemsetAsync(c->d_scol, 0, ((size_t)tot + 32) * 4, s));
  CK(cudaMemsetAsync(c->d_sval, 0, ((size_t)tot + 32) * vb, s));
  c->nsell = nsell;
  c->sell_cl = cl;
  c->ntiles_sell = ntsell;
  c->nltiles = (int)ltp.size() - 1;
  c->nhuge = (int)hug.size();
  if (nsell) {
    const void* val = c->pol == AJ_FP64 ? (const void*)c->val64 : c->valp;
    switch (c->pol) {
      case AJ_FP64: sell_fill<double>(c, val); break;
      case AJ_DF64: sell_fill<float2>(c, val); break;
      case AJ_FP32_IR: sell_fill<float>(c, val); break;
      default: sell_fill<__nv_bfloat16>(c, val); break;
    }
  }
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  c->fmt = 1;
  c->sell_sigma = sigma;
  c->sell_lmax = lmax;
  c->fill = c->nnz > 0 ? (double)(tot + long_entries) / (double)c->nnz : 1.0;
  return AJ_OK;
}

// Device time per sweep of the current format: a few sweeps from x = 0 with
// b = 0 (every load and multiply-add still runs).
static aj_status time_sweeps(aj_ctx* c, double* ms_per_sweep) {
  size_grid(c);
  const long long m = (long long)c->n * c->nrhs;
  cudaStream_t s = c->stream;
  const void* bvec = c->pol == AJ_FP64 ? (const void*)c->tmp64 : c->bp;
  CK(cudaMemsetAsync((void*)bvec, 0, (size_t)(m + 1) * xelem_bytes(c->pol), s));
  double best = 1e300;
  for (int rep = 0; rep < 2; rep++) {
    CK(cudaMemsetAsync(c->x[0], 0, (size_t)(m + 1) * xelem_bytes(c->pol), s));
    std::vector<RhsState> st(c->nrhs);
    double one[kMaxRhs] = {1, 1, 1, 1};
    init_state(c, st.data(), one);
    const double k0 = c->kernel_ms;
    const long long T = 8;
    aj_status e = run_persistent(c, st, bvec, T, AJ_STOP_NONE, 0.0, 0.0, 1.0, false);
    if (e != AJ_OK) return e;
    best = std::min(best, (c->kernel_ms - k0) / (double)(T + 1));
  }
  *ms_per_sweep = best;
  return AJ_OK;
}

struct TuneKey {
  int64_t n, nnz, sumsq, maxlen;
  int pol, nrhs, qx, ordered;
  bool operator<(const TuneKey& o) const {
    return std::tie(n, nnz, sumsq, maxlen, pol, nrhs, qx, ordered) <
           std::tie(o.n, o.nnz, o.sumsq, o.maxlen, o.pol, o.nrhs, o.qx, o.ordered);
  }
};
// the autotuner's choice: format (0 CSR, 1 SELL), sigma, lmax, log2 of the
// SELL slice height, CTAs per SM
struct TuneVal {
  int fmt, sigma, lmax, cl, ctas;
};
static std::map<TuneKey, TuneVal> g_tune;
static std::mutex g_tune_mu;

// The constant-coefficient stencil format: Q in natural row order is the
// 5-point (N x N) or 7-point (N^3) stencil with one diagonal and one
// off-diagonal value (a Dirichlet Laplacian, Sec. 4's grid problems).  The
// sweep then computes each row's columns and values instead of loading them,
// in the same ascending order and with the same values as the CSR rows, so
// its iterates are the CSR iterates bit for bit.  *is says whether Q is one.
static aj_status detect_stencil(aj_ctx* c, bool* is) {
  *is = false;
  const long long n = c->n, nnz = c->nnz;
  if (c->ordered || n < 4 || c->maxlen > 7) return AJ_OK;
  int dim = 0, N = 0;
  for (int d = 2; d <= 3 && !dim; d++) {
    const long long r = (long long)std::llround(std::pow((double)n, 1.0 / d));
    for (long long g = std::max(2ll, r - 1); g <= r + 1; g++) {
      const long long gd = d == 2 ? g * g : g * g * g;
      const long long want = d == 2 ? 5 * n - 4 * g : 7 * n - 6 * g * g;
      if (gd == n && nnz == want) { dim = d; N = (int)g; break; }
    }
  }
  if (!dim) return AJ_OK;
  cudaStream_t s = c->stream;
  // row 0 (a corner): the diagonal first, then the off-diagonal of column 1
  int c01[2];
  double v01[2];
  CK(cudaMemcpyAsync(c01, c->ci, 8, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(v01, c->val64, 16, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (c01[0] != 0 || c01[1] != 1) return AJ_OK;
  CK(cudaMemsetAsync(c->err, 0, 4, s));
  k_check_stencil<<<std::min<unsigned>(grid1d(n), 4096), kSetupThreads, 0, s>>>(
      (int)n, N, dim, c->rp, c->ci, c->val64, v01[0], v01[1], c->err);
  counted();
  int bad = 0;
  CK(cudaMemcpyAsync(&bad, c->err, 4, cudaMemcpyDeviceToHost, s));
  CK(cudaMemsetAsync(c->err, 0, 4, s));
  CK(cudaStreamSynchronize(s));
  if (bad) return AJ_OK;
  c->sdim = dim;
  c->sN = N;
  *is = true;
  return AJ_OK;
}

static int log2_slice(int C) { return C == 8 ? 3 : C == 16 ? 4 : 5; }

// Times the sweep with at most `ctas` CTAs per SM (0: the kernel's occupancy).
static aj_status time_grid(aj_ctx* c, int ctas, double* ms) {
  c->ctas_cap = ctas;
  return time_sweeps(c, ms);
}

static aj_status choose_format(aj_ctx* c, const aj_params* p) {
  const int sig = p->sell_sigma > 0 ? p->sell_sigma : 256;
  const int lmx = p->sell_lmax > 0 ? p->sell_lmax : 64;
  c->ctas_cap = 0;
  c->tuned = 0;
  if (p->format == AJ_FMT_SELL) return build_sell(c, sig, lmx, log2_slice(p->sell_c));
  c->sws.release();
  c->fmt = 0;
  c->fill = 1.0;
  if (p->format == AJ_FMT_CSR) return AJ_OK;
  // AUTO leaves FP64 with several right-hand sides, or in the lazy form, on
  // CSR: measured slower there in the stencil format (a 1024^2 grid, 4 RHS:
  // 0.91x in the difference form, 0.80x lazy); every other precision and form
  // gains (FP32 values on 256^3: 1.43x per sweep)
  const bool stencil_pays = !(c->pol == AJ_FP64 && (c->nrhs > 1 || c->qx == 0));
  if (p->format == AJ_FMT_STENCIL || (p->format == AJ_FMT_AUTO && stencil_pays)) {
    bool is = false;
    aj_status e = detect_stencil(c, &is);
    if (e != AJ_OK) return e;
    if (is) {
      c->fmt = 2;
      c->fill = 0.0;
      return AJ_OK;
    }
    if (p->format == AJ_FMT_STENCIL) return AJ_EINVAL;
  }
  // a block-diagonal J needs each block's rows in adjacent lanes: CSR order
  if (c->jblk > 1) return AJ_OK;
  const int n = (int)c->n;
  // few rows of many entries (a dense or nearly dense Q): CSR runs one CTA per
  // tile of rows, too few to fill the GPU; SELL's long-row bucket cuts such
  // rows into tiles of at most kLongTileEntries entries
  {
    const long long rpt = kThreads >> lanes_log2(c->nrhs);
    const long long ntiles = ((long long)n + rpt - 1) / rpt;
    if (c->maxlen > kResidLong && ntiles < c->sm_count && c->nnz >= (long long)c->sm_count * kLongTileEntries / 8)
      return build_sell(c, sig, lmx);
  }
  // AUTO: CSR unless the rows are long-tailed and the system is large
  if (n < 65536) return AJ_OK;
  if (c->maxlen <= 2.0 * ((double)c->nnz / n) + 8.0) return AJ_OK;  // near-uniform rows
  std::vector<int> rp((size_t)n + 1);
  CK(cudaMemcpyAsync(rp.data(), c->rp, rp.size() * 4, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  int64_t sumsq = 0, maxlen = 0;
  for (int i = 0; i < n; i++) {
    const int64_t l = rp[i + 1] - rp[i];
    sumsq += l * l;
    maxlen = std::max(maxlen, l);
  }
  const double mean = (double)c->nnz / n;
  if (maxlen <= 2.0 * mean + 8.0) return AJ_OK;
  // the autotuner (long-tailed rows): format and SELL's sorting window sigma
  // and long-row threshold, then SELL's slice height C in {32, 16, 8} (rows
  // per warp step; 32 / C lanes share a row), then the CTAs per SM; every
  // candidate timed over 8 sweeps, the choice cached per matrix shape
  const TuneKey key{c->n, c->nnz, sumsq, maxlen, c->pol, c->nrhs, c->qx, c->ordered};
  auto apply = [&](const TuneVal& v) -> aj_status {
    aj_status e = AJ_OK;
    if (v.fmt == 1) {
      e = build_sell(c, v.sigma, v.lmax, v.cl);
    } else {
      c->sws.release();
      c->fmt = 0;
      c->fill = 1.0;
    }
    c->ctas_cap = v.ctas;
    c->tuned = 1;
    return e;
  };
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      const TuneVal v = it->second;
      g_tune_hits.fetch_add(1);
      return apply(v);
    }
  }
  g_tune_misses.fetch_add(1);
  const TuneVal cand[] = {{0, 0, 0, 5, 0}, {1, 256, 64, 5, 0}, {1, 4096, 64, 5, 0}, {1, 256, 256, 5, 0}};
  TuneVal best = cand[0];
  double best_ms = 1e300;
  auto consider = [&](const TuneVal& v) -> aj_status {
    aj_status e = apply(v);
    if (e == AJ_ENOMEM) return AJ_OK;  // a candidate that does not fit is skipped
    if (e != AJ_OK) return e;
    double ms = 0.0;
    e = time_grid(c, v.ctas, &ms);
    if (e != AJ_OK) return e;
    if (ms < best_ms) { best_ms = ms; best = v; }
    return AJ_OK;
  };
  for (const auto& v : cand) {
    aj_status e = consider(v);
    if (e != AJ_OK) return e;
  }
  if (best.fmt == 1 && c->nrhs == 1) {
    for (int cl : {4, 3}) {
      TuneVal v = best;
      v.cl = cl;
      aj_status e = consider(v);
      if (e != AJ_OK) return e;
    }
  }
#ifndef AJ_TUNE_CTAS
#define AJ_TUNE_CTAS 1
#endif
  if (AJ_TUNE_CTAS) {
    // CTAs per SM below the kernel's occupancy (fewer CTAs, less imbalance at
    // each grid barrier, more L1 per CTA)
    const int fm = best.fmt == 1 ? (best.cl < 5 ? 4 : AJ_SELL_FM) : 0;
    const int occ = std::max(1, persistent_blocks_per_sm(kernel_pol(c->pol), c->nrhs, c->qx, fm));
    for (int k = occ - 1; k >= std::max(2, occ - 2); k--) {
      TuneVal v = best;
      v.ctas = k;
      aj_status e = consider(v);
      if (e != AJ_OK) return e;
    }
  }
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = best;
  }
  return apply(best);
}

extern "C" aj_status aj_get_tuning(aj_ctx* c, aj_tuning* out) {
  if (!c || !out || !c->have_prm) return AJ_EINVAL;
  std::memset(out, 0, sizeof(*out));
  out->format = c->fmt == 1 ? AJ_FMT_SELL : c->fmt == 2 ? AJ_FMT_STENCIL : AJ_FMT_CSR;
  const bool sell = c->fmt == 1;
  const int lg = lanes_log2(c->nrhs);
  out->sell_c = sell ? 1 << c->sell_cl : 0;
  out->sell_sigma = sell ? c->sell_sigma : 0;
  out->sell_lmax = sell ? c->sell_lmax : 0;
  out->lanes_per_row = sell && c->sell_cl < 5 ? 32 >> c->sell_cl : 1 << lg;
  out->rows_per_cta = sell && c->sell_cl < 5 ? kWarps << c->sell_cl : kThreads >> lg;
  out->threads_per_cta = kThreads;
  out->grid = c->grid;
  out->ctas_per_sm = (c->grid + c->sm_count - 1) / std::max(1, c->sm_count);
  out->sweep_form = c->qx == 0 ? AJ_SWEEP_LAZY : c->qx == 1 ? AJ_SWEEP_STORED : c->qx == 2 ? AJ_SWEEP_DELTA
                                                                                         : AJ_SWEEP_Y;
  out->tuned = c->tuned;
  out->fill_ratio = c->fill;
  return AJ_OK;
}

extern "C" aj_status aj_get_format(aj_ctx* c, int* format, int* sigma, int* lmax, double* fill_ratio) {
  if (!c) return AJ_EINVAL;
  if (format) *format = c->fmt == 1 ? AJ_FMT_SELL : c->fmt == 2 ? AJ_FMT_STENCIL : AJ_FMT_CSR;
  if (sigma) *sigma = c->fmt == 1 ? c->sell_sigma : 0;
  if (lmax) *lmax = c->fmt == 1 ? c->sell_lmax : 0;
  if (fill_ratio) *fill_ratio = c->fill;
  return AJ_OK;
}

// ---------------------------------------------------------------- batched launches
// One system of a batched launch: its context, its state (host copy, in/out)
// and the arguments of its run.
struct BatchItem {
  aj_ctx* c;
  std::vector<RhsState>* st;
  const void* bvec;
  long long maxit;
  int stop;
  double tol, fstar, fscale;
  long long max_sweeps;  // sweeps this launch may run (maxit + 2: to the end)
};

// Tiles of a context's sweep (rows per tile 256 >> lgr).
static long long ctx_tiles(const aj_ctx* c) {
  const long long rpt = kThreads >> lanes_log2(c->nrhs);
  return std::max<long long>(1, (c->n + rpt - 1) / rpt);
}

// Units a system gets in a lockstep launch (V_s).  A context's own grid_ctas
// fixes it; a system's arithmetic depends only on this count, so such a
// batch member computes exactly what aj_solve computes with the same
// grid_ctas.  Otherwise it follows the launch's load: about 16 units per CTA
// over all active systems (active_tiles in total), a system's share in
// proportion to its tiles -- coarse units while many systems run, fine ones
// when a few large systems remain -- at most one per tile and at most the
// CTA count its partial-sum buffer holds.  The reduction grouping then
// changes between launches, which moves the FP64 sums by rounding only.
static int batch_units(const aj_ctx* c, long long active_tiles, int grid) {
  const int cap = std::max(1, c->part_cap);
  if (c->prm.grid_ctas > 0) return std::max(1, std::min(c->prm.grid_ctas, cap));
  const long long nt = ctx_tiles(c);
  const double want = (double)nt * 16.0 * grid / (double)std::max<long long>(active_tiles, 1);
  const long long v = (long long)std::ceil(want);
  return (int)std::max<long long>(1, std::min<long long>({v, nt, (long long)cap}));
}

// 1: every lockstep launch prints its systems, units, grid, sweeps and device
// time to stderr (a diagnostic build)
#ifndef AJ_TRACE_LOCKSTEP
#define AJ_TRACE_LOCKSTEP 0
#endif

// Device buffers of lockstep launches, kept between launches and grown on
// demand (a server keeps one for its lifetime).
struct LockWs {
  Workspace mem;
  cudaStream_t stream = nullptr;  // stream of the launches (allocations follow it)
  size_t cap_m = 0, cap_nu = 0;
  void* d_sys = nullptr;
  int *d_unit = nullptr, *d_u0 = nullptr, *d_nu = nullptr, *d_cta = nullptr, *d_err = nullptr;
  RhsState *d_st2 = nullptr, *d_out = nullptr;
  unsigned long long* d_bar = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  LockWs() { mem.stream = &stream; }
  LockWs(const LockWs&) = delete;
  LockWs& operator=(const LockWs&) = delete;
  ~LockWs() {
    mem.release();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  }
  size_t cap_g = 0;
  bool reserve(size_t m, size_t nu, size_t g, size_t abytes) {
    if (d_sys && m <= cap_m && nu <= cap_nu && g <= cap_g) return true;
    mem.release();
    cap_m = std::max(m, 2 * cap_m);
    cap_nu = std::max(nu, 2 * cap_nu);
    cap_g = std::max(g, cap_g);
    d_sys = mem.alloc(cap_m * abytes);
    d_cta = (int*)mem.alloc((cap_g + 1) * 4);
    d_u0 = (int*)mem.alloc(cap_m * 4);
    d_nu = (int*)mem.alloc(cap_m * 4);
    d_unit = (int*)mem.alloc(cap_nu * 4);
    d_st2 = (RhsState*)mem.alloc(cap_m * 2 * kMaxRhs * sizeof(RhsState));
    d_out = (RhsState*)mem.alloc(cap_m * kMaxRhs * sizeof(RhsState));
    d_bar = (unsigned long long*)mem.alloc(64);
    d_err = (int*)mem.alloc(64);
    if (!e0 && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) return false;
    return d_sys && d_u0 && d_nu && d_cta && d_unit && d_st2 && d_out && d_bar && d_err;
  }
};

// Solves every item (one precision and sweep form, any right-hand-side
// counts) with lockstep launches.  Each launch runs a chunk of sweeps over
// the systems still running (at most what each item has left of its
// max_sweeps) and drops those that stopped; the chunk starts at chunk0 and
// doubles while a launch takes under 5 ms of device time, so small systems
// retire early and the large ones run long launches.  Each item's state
// (host copy, in/out) is carried from launch to launch.
static aj_status run_batched(std::vector<BatchItem>& items, bool log_restarts, double* kernel_ms,
                             LockWs* wsp = nullptr, long long chunk0 = 16) {
  if (items.empty()) return AJ_OK;
  aj_ctx* c0 = items[0].c;
  cudaStream_t s = c0->stream;
  const int pol = c0->pol, qx = c0->qx;
  LockWs local;
  local.stream = s;
  LockWs& ws = wsp ? *wsp : local;
  const size_t abytes = iter_args_bytes();
  const int bps = lockstep_blocks_per_sm(pol, qx);
  if (bps < 1) return AJ_ECUDA;
  const int gmax = bps * c0->sm_count;
  const int m_all = (int)items.size();
  std::vector<int> V(m_all, 1);
  std::vector<long long> left(m_all);
  std::vector<IterLaunch> Ls(m_all);
  for (int i = 0; i < m_all; i++) {
    const BatchItem& it = items[i];
    left[i] = it.max_sweeps;
    Ls[i] = make_launch(it.c, it.bvec, it.maxit, it.stop, it.tol, it.fstar, it.fscale);
    if (log_restarts) CK(cudaMemsetAsync(it.c->rlog, 0xff, (size_t)kMaxRhs * it.c->rlog_cap * 8, s));
  }
  auto running = [&](int i) {
    if (left[i] <= 0) return false;
    for (int r = 0; r < items[i].c->nrhs; r++)
      if (!(*items[i].st)[r].done) return true;
    return false;
  };
  long long chunk = std::max<long long>(1, chunk0);
  std::vector<int> act, u0, nu, unit, cta;
  std::vector<double> ucost;
  std::vector<unsigned char> sysh;
  std::vector<RhsState> st2, out;
  for (;;) {
    act.clear();
    for (int i = 0; i < m_all; i++)
      if (running(i)) act.push_back(i);
    if (act.empty()) break;
    // the launch runs as many sweeps as the item with the most left may use
    // (at most the chunk); each item runs at most what it has left
    long long most = 0;
    for (int i : act) most = std::max(most, left[i]);
    const long long sweeps = std::min(chunk, most);
    const int m = (int)act.size();
    long long active_tiles = 0;
    for (int i : act) active_tiles += ctx_tiles(items[i].c);
    for (int i : act) V[i] = batch_units(items[i].c, active_tiles, gmax);
    u0.assign(m, 0);
    nu.assign(m, 0);
    unit.clear();
    ucost.clear();
    sysh.resize((size_t)m * abytes);
    st2.assign((size_t)m * 2 * kMaxRhs, RhsState());
    for (int j = 0; j < m; j++) {
      const int i = act[j];
      u0[j] = (int)unit.size();
      nu[j] = V[i];
      // estimated work of unit v: its tiles x row-RHS pairs per tile x
      // (entries per row + the per-row update), plus a fixed cost of about
      // one tile for the unit's own reductions; a stencil row loads no
      // column or value, only its x gathers, about 0.4 of a CSR entry's cost
      const aj_ctx* c = items[i].c;
      const long long rpt = kThreads >> lanes_log2(c->nrhs);
      const long long ntiles = ctx_tiles(c);
      const double epr = (double)c->nnz / std::max<int64_t>(c->n, 1) * (c->fmt == 2 ? 0.4 : 1.0);
      const double per_tile = (double)rpt * c->nrhs * (epr + 9.0);
      const long long mine = std::min(left[i], sweeps);  // sweeps this item runs in the launch
      for (int v = 0; v < V[i]; v++) {
        unit.push_back(j);
        const long long tv = v < ntiles ? (ntiles - 1 - v) / V[i] + 1 : 0;
        ucost.push_back(per_tile * (double)(tv + 1) * (double)mine / (double)sweeps);
      }
      Ls[i].max_sweeps = mine;
      pack_iter_args(pol, Ls[i], sysh.data() + (size_t)j * abytes);
      for (int r = 0; r < items[i].c->nrhs; r++) st2[(size_t)j * 2 * kMaxRhs + r] = (*items[i].st)[r];
    }
    // contiguous unit ranges of about equal estimated work, one per CTA
    const int grid = std::max(1, std::min(gmax, (int)unit.size()));
    double total = 0.0;
    for (double w : ucost) total += w;
    cta.assign((size_t)grid + 1, (int)unit.size());
    cta[0] = 0;
    {
      double acc = 0.0;
      int c = 1;
      for (size_t u = 0; u < unit.size() && c < grid; u++) {
        // unit u starts at acc; it opens CTA c's range once acc reaches c/grid of the total
        while (c < grid && acc >= total * c / grid) cta[c++] = (int)u;
        acc += ucost[u];
      }
    }
    if (!ws.reserve(m, unit.size(), grid, abytes)) return AJ_ENOMEM;
    CK(cudaMemcpyAsync(ws.d_cta, cta.data(), cta.size() * 4, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ws.d_sys, sysh.data(), sysh.size(), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ws.d_unit, unit.data(), unit.size() * 4, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ws.d_u0, u0.data(), (size_t)m * 4, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ws.d_nu, nu.data(), (size_t)m * 4, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ws.d_st2, st2.data(), st2.size() * sizeof(RhsState), cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(ws.d_bar, 0, 64, s));
    CK(cudaMemsetAsync(ws.d_err, 0, 64, s));
    LockLaunch B;
    B.sys = ws.d_sys;
    B.unit_sys = ws.d_unit;
    B.sys_u0 = ws.d_u0;
    B.sys_nu = ws.d_nu;
    B.cta_u0 = ws.d_cta;
    B.st2 = ws.d_st2;
    B.st_out = ws.d_out;
    B.nu = (int)unit.size();
    B.sweeps = sweeps;
    B.bar = ws.d_bar;
    B.err = ws.d_err;
    CK(cudaEventRecord(ws.e0, s));
    CK(launch_lockstep(pol, qx, B, grid, s));
    counted();
    CK(cudaEventRecord(ws.e1, s));
    out.resize((size_t)m * kMaxRhs);
    int err = 0;
    CK(cudaMemcpyAsync(out.data(), ws.d_out, out.size() * sizeof(RhsState), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&err, ws.d_err, 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    float kms = 0.f;
    cudaEventElapsedTime(&kms, ws.e0, ws.e1);
    if (kernel_ms) *kernel_ms += kms;
#if AJ_TRACE_LOCKSTEP
    {
      long long rows = 0, nnz = 0;
      for (int i : act) {
        rows += items[i].c->n * items[i].c->nrhs;
        nnz += items[i].c->nnz * items[i].c->nrhs;
      }
      fprintf(stderr, "lockstep systems %d units %zu grid %d sweeps %lld ms %.3f rowrhs %lld nnzrhs %lld\n", m,
              unit.size(), grid, sweeps, kms, rows, nnz);
    }
#endif
    if (err != 0) return err == kETimeout ? AJ_ETIMEOUT : AJ_ECUDA;
    for (int j = 0; j < m; j++) {
      const int i = act[j];
      for (int r = 0; r < items[i].c->nrhs; r++) (*items[i].st)[r] = out[(size_t)j * kMaxRhs + r];
      left[i] -= std::min(left[i], sweeps);
    }
    if (kms < 5.0f && chunk < 4096) chunk *= 2;
  }
  return AJ_OK;
}

static aj_status fetch_rlog(aj_ctx* c, const std::vector<RhsState>& st, bool append) {
  std::vector<long long> h((size_t)kMaxRhs * c->rlog_cap);
  CK(cudaMemcpyAsync(h.data(), c->rlog, h.size() * 8, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (!append) c->rlog_h.assign(c->nrhs, {});
  c->rlog_h.resize(c->nrhs);
  for (int r = 0; r < c->nrhs; r++)
    for (int k = 0; k < c->rlog_cap; k++) {
      long long v = h[(size_t)r * c->rlog_cap + k];
      if (v >= 0) c->rlog_h[r].push_back(v);
    }
  (void)st;
  return AJ_OK;
}

// FP64 residual of an interleaved FP64 iterate: relres and objgap per RHS.
// The rows longer than kResidLong in the run's order, for the residual's
// warp-per-row pass: built on first use and again after a change of order.
static aj_status resid_long_rows(aj_ctx* c) {
  if (c->maxlen <= kResidLong) {
    c->n_resid_long = 0;
    return AJ_OK;
  }
  if (c->resid_long_order == c->ordered) return AJ_OK;
  const int n = (int)c->n;
  std::vector<int> rp((size_t)n + 1), rows;
  CK(cudaMemcpyAsync(rp.data(), c->rp, rp.size() * 4, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  for (int i = 0; i < n; i++)
    if (rp[i + 1] - rp[i] > kResidLong) rows.push_back(i);
  c->rws.release();
  c->n_resid_long = (int)rows.size();
  const int nb = (c->n_resid_long + kSetupThreads / 32 - 1) / (kSetupThreads / 32);
  c->d_resid_long = (int*)c->rws.alloc((rows.size() + 1) * 4);
  c->part_long = (double*)c->rws.alloc((size_t)std::max(nb, 1) * kMaxRhs * 3 * 8);
  if (!c->d_resid_long || !c->part_long) return AJ_ENOMEM;
  if (!rows.empty())
    CK(cudaMemcpyAsync(c->d_resid_long, rows.data(), rows.size() * 4, cudaMemcpyHostToDevice, c->stream));
  c->resid_long_order = c->ordered;
  return AJ_OK;
}

static aj_status fp64_report(aj_ctx* c, const double* x_il, double* relres, double* objgap,
                             double* r_out) {
  const int n = (int)c->n;
  const int nrhs = c->nrhs;
  const int blocks = std::max(1, (int)grid1d(n));
  aj_status st = resid_long_rows(c);
  if (st != AJ_OK) return st;
  const int nl = c->n_resid_long;
  const int lblocks = (nl + kSetupThreads / 32 - 1) / (kSetupThreads / 32);
  if (n > 0) {
    k_residual<<<blocks, kSetupThreads, 0, c->stream>>>(n, nrhs, c->rp, c->ci, c->val64, c->b64,
                                                        x_il, r_out, c->part_small, nl > 0 ? kResidLong : -1);
    counted();
    if (nl > 0) {
      k_residual_long<<<lblocks, kSetupThreads, 0, c->stream>>>(nl, c->d_resid_long, nrhs, c->rp, c->ci,
                                                                c->val64, c->b64, x_il, r_out, c->part_long);
      counted();
    }
  } else
    CK(cudaMemsetAsync(c->part_small, 0, (size_t)nrhs * 3 * 8, c->stream));
  CK(cudaGetLastError());
  double sums[kMaxRhs * 3];
  st = host_sum_parts(c, c->part_small, n > 0 ? blocks : 1, nrhs * 3, sums);
  if (st != AJ_OK) return st;
  if (n > 0 && nl > 0) {
    double more[kMaxRhs * 3];
    st = host_sum_parts(c, c->part_long, lblocks, nrhs * 3, more);
    if (st != AJ_OK) return st;
    for (int k = 0; k < nrhs * 3; k++) sums[k] += more[k];
  }
  for (int r = 0; r < nrhs; r++) {
    const double rn = std::sqrt(sums[r * 3 + 0]);
    const double bn = std::sqrt(c->bnorm2[r]);
    relres[r] = bn > 0.0 ? rn / bn : rn;
    const double f = 0.5 * sums[r * 3 + 1] - sums[r * 3 + 2];
    objgap[r] = std::fabs(f - c->prm.fstar) / (1.0 + std::fabs(c->prm.fstar));
  }
  return AJ_OK;
}

static aj_status status_of(int s) {
  switch (s) {
    case kOk: return AJ_OK;
    case kEMaxit: return AJ_EMAXIT;
    case kEDiverged: return AJ_EDIVERGED;
    case kENonfinite: return AJ_ENONFINITE;
    case kETimeout: return AJ_ETIMEOUT;
  }
  return AJ_ECUDA;
}

// Initial point x^0 (interleaved FP64) into tmp64.
static aj_status load_x0(aj_ctx* c) {
  const int n = (int)c->n;
  const long long m = (long long)n * c->nrhs;
  cudaStream_t s = c->stream;
  if (m == 0) return AJ_OK;
  if (!c->prm.x0) {
    CK(cudaMemsetAsync(c->tmp64, 0, (size_t)m * 8, s));
    return AJ_OK;
  }
  // x0 is column-major: interleave it on the host
  std::vector<double> h((size_t)m), il((size_t)m);
  CK(cudaMemcpyAsync(h.data(), c->prm.x0, (size_t)m * 8,
                     c->prm.x0_on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost, s));
  CK(cudaStreamSynchronize(s));
  // (row i of the run's order is the caller's row perm[i] when renumbered)
  for (int r = 0; r < c->nrhs; r++)
    for (int i = 0; i < n; i++)
      il[(size_t)i * c->nrhs + r] = h[(size_t)r * n + (c->ordered ? c->perm_h[i] : i)];
  CK(cudaMemcpyAsync(c->tmp64, il.data(), (size_t)m * 8, cudaMemcpyHostToDevice, s));
  CK(cudaStreamSynchronize(s));
  return AJ_OK;
}

static aj_status write_output(aj_ctx* c, const double* x_il, double* x_out, int x_on_device) {
  const int n = (int)c->n;
  const long long m = (long long)n * c->nrhs;
  cudaStream_t s = c->stream;
  if (m == 0) return AJ_OK;
  if (c->ordered) {
    // back to the caller's rows and column-major layout in one gather
    double* cm = x_il == c->tmp64 ? c->r64 : c->tmp64;
    if (!cm || cm == x_il) return AJ_EINVAL;
    k_unpermute_deinterleave<<<grid1d(m), kSetupThreads, 0, s>>>(n, c->nrhs, c->perm, x_il, cm);
    counted();
    CK(cudaMemcpyAsync(x_out, cm, (size_t)m * 8,
                       x_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return AJ_OK;
  }
  if (c->nrhs == 1) {
    CK(cudaMemcpyAsync(x_out, x_il, (size_t)m * 8,
                       x_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return AJ_OK;
  }
  double* cm = x_il == c->tmp64 ? c->r64 : c->tmp64;
  if (!cm || cm == x_il) {
    // fall back to a host-side transpose
    std::vector<double> h((size_t)m), o((size_t)m);
    CK(cudaMemcpyAsync(h.data(), x_il, (size_t)m * 8, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (int r = 0; r < c->nrhs; r++)
      for (int i = 0; i < n; i++) o[(size_t)r * n + i] = h[(size_t)i * c->nrhs + r];
    CK(cudaMemcpyAsync(x_out, o.data(), (size_t)m * 8,
                       x_on_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost, s));
    CK(cudaStreamSynchronize(s));
    return AJ_OK;
  }
  k_deinterleave<<<grid1d(m), kSetupThreads, 0, s>>>(n, c->nrhs, x_il, cm);
  counted();
  CK(cudaMemcpyAsync(x_out, cm, (size_t)m * 8,
                     x_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return AJ_OK;
}

// Direct solve (FP64 or DF64 arithmetic in the persistent kernel), in three
// parts so that a batch can run the middle one for many contexts at once.
struct DirectRun {
  std::vector<RhsState> st;
  double sb[kMaxRhs];
  const void* bvec = nullptr;
  double fscale = 1.0;
};

static aj_status direct_prepare(aj_ctx* c, DirectRun& d) {
  const int nrhs = c->nrhs;
  const double sq = c->sQ;
  double bn2[kMaxRhs];
  for (int r = 0; r < nrhs; r++) {
    d.sb[r] = c->pol == AJ_FP64 ? 1.0 : pow2_near(std::sqrt(c->bnorm2[r] / std::max<int64_t>(c->n, 1)));
    bn2[r] = c->bnorm2[r] * d.sb[r] * d.sb[r];
  }
  d.st.assign(nrhs, RhsState());
  if (c->resume) {
    d.st = c->st_h;
    for (int r = 0; r < nrhs; r++) d.sb[r] = c->sb[r];
    for (int r = 0; r < nrhs; r++)
      if (d.st[r].done && d.st[r].status == kEMaxit) { d.st[r].done = 0; d.st[r].status = 0; }
  } else {
    for (int r = 0; r < nrhs; r++) c->sb[r] = d.sb[r];
    init_state(c, d.st.data(), bn2);
    aj_status e = load_x0(c);
    if (e != AJ_OK) return e;
    double xs[kMaxRhs];
    for (int r = 0; r < nrhs; r++) xs[r] = d.sb[r] / sq;
    to_policy(c, c->tmp64, c->x[0], xs);
  }
  // right-hand side in the iteration precision
  d.bvec = c->b64;
  if (c->pol != AJ_FP64) {
    to_policy(c, c->b64, c->bp, d.sb);
    d.bvec = c->bp;
  }
  CK(cudaGetLastError());
  // f of the scaled problem is (sb^2 / sQ) f of the original one
  d.fscale = sq / (d.sb[0] * d.sb[0]);
  return AJ_OK;
}

static aj_status direct_finish(aj_ctx* c, DirectRun& d, double* x_out, int x_on_device,
                               aj_info* per) {
  const int nrhs = c->nrhs;
  const double sq = c->sQ;
  aj_status e = fetch_rlog(c, d.st, false);
  if (e != AJ_OK) return e;
  int cur[kMaxRhs];
  double osc[kMaxRhs];
  for (int r = 0; r < nrhs; r++) {
    cur[r] = d.st[r].cur;
    osc[r] = sq / d.sb[r];
  }
  double* xil = c->pol == AJ_FP64 ? c->tmp64 : c->x64;
  e = from_policy(c, cur, osc, xil);
  if (e != AJ_OK) return e;
  double rel[kMaxRhs], og[kMaxRhs];
  e = fp64_report(c, xil, rel, og, nullptr);
  if (e != AJ_OK) return e;
  e = write_output(c, xil, x_out, x_on_device);
  if (e != AJ_OK) return e;
  c->st_h = d.st;
  for (int r = 0; r < nrhs; r++) {
    per[r].iters = d.st[r].t_final;
    per[r].restarts = d.st[r].ell;
    per[r].sweeps = d.st[r].t_final + 1;
    per[r].outer = 0;
    per[r].relres = rel[r];
    per[r].objgap = og[r];
    per[r].L_used = c->L_used;
    per[r].status = status_of(d.st[r].status);
  }
  return AJ_OK;
}

static aj_status solve_direct(aj_ctx* c, double* x_out, int x_on_device, aj_info* per) {
  DirectRun d;
  aj_status e = direct_prepare(c, d);
  if (e != AJ_OK) return e;
  e = run_persistent(c, d.st, d.bvec, c->prm.maxit, c->prm.stop, c->prm.tol, c->prm.fstar,
                     d.fscale, true);
  if (e != AJ_OK) return e;
  return direct_finish(c, d, x_out, x_on_device, per);
}

// FP64 iterative refinement around the low-precision persistent solver, for
// one or many contexts: each outer step computes the FP64 residual of every
// unfinished context, solves Q d = r in the iteration precision (one
// persistent launch per context, or one batched launch for all of them) and
// adds d to the FP64 iterate.  The steps are separate functions so that the
// server can drive one context through them between its rounds.
struct IrRun {
  long long iters[kMaxRhs] = {0, 0, 0, 0}, rest[kMaxRhs] = {0, 0, 0, 0};
  int status[kMaxRhs] = {kEMaxit, kEMaxit, kEMaxit, kEMaxit};
  bool done[kMaxRhs] = {false, false, false, false};
  double rel[kMaxRhs] = {0, 0, 0, 0}, og[kMaxRhs] = {0, 0, 0, 0}, sr[kMaxRhs] = {1, 1, 1, 1};
  long long outer = 0;
  bool finished = false;
  std::vector<RhsState> st;
};

// x64 = x^0.
static aj_status ir_begin(aj_ctx* c, IrRun& q) {
  aj_status e = load_x0(c);
  if (e != AJ_OK) return e;
  const long long m = (long long)c->n * c->nrhs;
  if (m > 0) CK(cudaMemcpyAsync(c->x64, c->tmp64, (size_t)m * 8, cudaMemcpyDeviceToDevice, c->stream));
  c->rlog_h.assign(c->nrhs, {});
  (void)q;
  return AJ_OK;
}

// FP64 residual of x64 and the outer stop test; sets q.finished.
static aj_status ir_check(aj_ctx* c, IrRun& q) {
  aj_status e = AJ_OK;
  if (q.outer == 0 && !c->prm.x0) {
    // x^0 = 0: the residual is b itself (relative residual 1, f = 0)
    const long long m = (long long)c->n * c->nrhs;
    if (m > 0) CK(cudaMemcpyAsync(c->r64, c->b64, (size_t)m * 8, cudaMemcpyDeviceToDevice, c->stream));
    for (int r = 0; r < c->nrhs; r++) {
      q.rel[r] = c->bnorm2[r] > 0.0 ? 1.0 : 0.0;
      q.og[r] = std::fabs(c->prm.fstar) / (1.0 + std::fabs(c->prm.fstar));
    }
  } else {
    e = fp64_report(c, c->x64, q.rel, q.og, c->r64);
  }
  if (e != AJ_OK) return e;
  bool all = true;
  for (int r = 0; r < c->nrhs; r++) {
    if (q.done[r]) continue;
    bool ok = false;
    if (c->prm.stop == AJ_STOP_RELRES) ok = q.rel[r] <= c->prm.tol;
    else if (c->prm.stop == AJ_STOP_OBJGAP) ok = q.og[r] <= c->prm.tol;
    if (ok) { q.done[r] = true; q.status[r] = kOk; }
    else if (!std::isfinite(q.rel[r])) { q.done[r] = true; q.status[r] = kENonfinite; }
    all = all && q.done[r];
  }
  long long used = 0;
  for (int r = 0; r < c->nrhs; r++) used = std::max(used, q.iters[r]);
  if (all || q.outer >= c->prm.max_outer || used >= c->prm.maxit) q.finished = true;
  return AJ_OK;
}

// Inner right-hand side (the residual scaled by a power of two per RHS), the
// inner state and x = 0; returns the inner run as a batch item.
static BatchItem ir_inner_setup(aj_ctx* c, IrRun& q) {
  const int n = (int)c->n;
  const long long m = (long long)n * c->nrhs;
  q.outer++;
  double bn2[kMaxRhs];
  for (int r = 0; r < c->nrhs; r++) {
    const double rn = q.rel[r] * std::sqrt(c->bnorm2[r] > 0 ? c->bnorm2[r] : 1.0);
    q.sr[r] = pow2_near(rn / std::sqrt((double)std::max(n, 1)));
    bn2[r] = rn * rn * q.sr[r] * q.sr[r];
  }
  to_policy(c, c->r64, c->bp, q.sr);
  q.st.assign(c->nrhs, RhsState());
  init_state(c, q.st.data(), bn2);
  for (int r = 0; r < c->nrhs; r++)
    if (q.done[r]) { q.st[r].done = 1; q.st[r].status = kOk; }
  if (m > 0) cudaMemsetAsync(c->x[0], 0, (size_t)m * xelem_bytes(c->pol), c->stream);
  long long used = 0;
  for (int r = 0; r < c->nrhs; r++) used = std::max(used, q.iters[r]);
  const long long budget = std::max<long long>(1, c->prm.maxit - used);
  return BatchItem{c, &q.st, c->bp, budget, AJ_STOP_RELRES, c->prm.inner_tol, 0.0, 1.0, budget + 2};
}

// x64 += (sQ / sr) d for the right-hand sides that were still running.
static aj_status ir_inner_finish(aj_ctx* c, IrRun& q) {
  const long long m = (long long)c->n * c->nrhs;
  aj_status e = fetch_rlog(c, q.st, true);
  if (e != AJ_OK) return e;
  int cur[kMaxRhs];
  double osc[kMaxRhs];
  for (int r = 0; r < c->nrhs; r++) {
    cur[r] = q.st[r].cur;
    osc[r] = c->sQ / q.sr[r];
  }
  e = from_policy(c, cur, osc, c->tmp64);
  if (e != AJ_OK) return e;
  unsigned mask = 0;
  for (int r = 0; r < c->nrhs; r++)
    if (!q.done[r]) {
      mask |= 1u << r;
      q.iters[r] += q.st[r].t_final;
      q.rest[r] += q.st[r].ell;
      if (q.st[r].status == kENonfinite || q.st[r].status == kEDiverged) {
        q.done[r] = true;
        q.status[r] = q.st[r].status;
      }
    }
  if (m > 0) {
    k_axpy_masked<<<grid1d(m), kSetupThreads, 0, c->stream>>>(m, c->nrhs, mask, c->tmp64, 1.0, c->x64);
    counted();
  }
  CK(cudaGetLastError());
  return AJ_OK;
}

static aj_status ir_end(aj_ctx* c, IrRun& q, double* x_out, int x_on_device, aj_info* per) {
  aj_status e = write_output(c, c->x64, x_out, x_on_device);
  if (e != AJ_OK) return e;
  for (int r = 0; r < c->nrhs; r++) {
    aj_info& o = per[r];
    o.iters = q.iters[r];
    o.restarts = q.rest[r];
    o.sweeps = q.iters[r] + q.outer;
    o.outer = q.outer;
    o.relres = q.rel[r];
    o.objgap = q.og[r];
    o.L_used = c->L_used;
    o.status = q.done[r] ? status_of(q.status[r]) : AJ_EMAXIT;
  }
  return AJ_OK;
}

static aj_status ir_solve(aj_ctx* const* cs, int count, double* const* x_out, int x_on_device,
                          aj_info* const* per, bool batched, double* batch_kms) {
  std::vector<IrRun> R(count);
  for (int i = 0; i < count; i++) {
    aj_status e = ir_begin(cs[i], R[i]);
    if (e != AJ_OK) return e;
  }
  for (;;) {
    std::vector<int> act;
    for (int i = 0; i < count; i++) {
      if (R[i].finished) continue;
      aj_status e = ir_check(cs[i], R[i]);
      if (e != AJ_OK) return e;
      if (!R[i].finished) act.push_back(i);
    }
    if (act.empty()) break;
    std::vector<BatchItem> items;
    for (int i : act) items.push_back(ir_inner_setup(cs[i], R[i]));
    CK(cudaGetLastError());
    if (batched) {
      aj_status e = run_batched(items, true, batch_kms);
      if (e != AJ_OK) return e;
    } else {
      for (auto& it : items) {
        aj_status e = run_persistent(it.c, *it.st, it.bvec, it.maxit, it.stop, it.tol, it.fstar,
                                     it.fscale, true);
        if (e != AJ_OK) return e;
      }
    }
    for (int i : act) {
      aj_status e = ir_inner_finish(cs[i], R[i]);
      if (e != AJ_OK) return e;
    }
  }
  for (int i = 0; i < count; i++) {
    aj_status e = ir_end(cs[i], R[i], x_out[i], x_on_device, per[i]);
    if (e != AJ_OK) return e;
  }
  return AJ_OK;
}

static aj_status solve_ir(aj_ctx* c, double* x_out, int x_on_device, aj_info* per) {
  aj_ctx* cs[1] = {c};
  double* xo[1] = {x_out};
  aj_info* pp[1] = {per};
  return ir_solve(cs, 1, xo, x_on_device, pp, false, nullptr);
}

// The report of the right-hand side with the worst residual, with the largest
// iteration and restart counts over all right-hand sides.
static void summarize(const aj_info* per, int nrhs, aj_info* out) {
  int w = 0;
  for (int r = 1; r < nrhs; r++)
    if (per[r].status != AJ_OK || per[r].relres > per[w].relres) w = r;
  *out = per[w];
  long long it = 0, rs = 0;
  for (int r = 0; r < nrhs; r++) {
    it = std::max<long long>(it, per[r].iters);
    rs = std::max<long long>(rs, per[r].restarts);
  }
  out->iters = it;
  out->restarts = rs;
}

extern "C" aj_status aj_solve_rhs(aj_ctx* c, double* x_out, int x_on_device, aj_info* per_rhs) {
  if (!c || (!x_out && c->n > 0)) return AJ_EINVAL;
  if (!c->have_prm) {
    aj_params p;
    aj_params_default(&p);
    aj_status st = aj_set(c, &p);
    if (st != AJ_OK) return st;
  }
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != c->dev) cudaSetDevice(c->dev);
  aj_info per[kMaxRhs];
  std::memset(per, 0, sizeof(per));
  c->kernel_ms = 0.0;
  t_launches = 0;
  CK(cudaEventRecord(c->ev0, c->stream));
  aj_status st;
  if (c->pol == AJ_FP64 || c->pol == AJ_DF64) st = solve_direct(c, x_out, x_on_device, per);
  else st = solve_ir(c, x_out, x_on_device, per);
  CK(cudaEventRecord(c->ev1, c->stream));
  CK(cudaEventSynchronize(c->ev1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, c->ev0, c->ev1);
  c->resume = false;
  if (cur != c->dev) cudaSetDevice(cur);
  if (st != AJ_OK) return st;
  aj_status worst = AJ_OK;
  for (int r = 0; r < c->nrhs; r++) {
    per[r].ms = ms;
    per[r].kernel_ms = c->kernel_ms;
    per[r].launches = t_launches;
    if (per[r].status != AJ_OK && worst == AJ_OK) worst = per[r].status;
  }
  if (per_rhs)
    for (int r = 0; r < c->nrhs; r++) per_rhs[r] = per[r];
  return worst;
}

extern "C" aj_status aj_solve(aj_ctx* c, double* x_out, int x_on_device, aj_info* info) {
  if (!c) return AJ_EINVAL;
  aj_info per[kMaxRhs];
  std::memset(per, 0, sizeof(per));
  aj_status st = aj_solve_rhs(c, x_out, x_on_device, per);
  if (info && (st == AJ_OK || st == AJ_EMAXIT || st == AJ_EDIVERGED || st == AJ_ENONFINITE)) {
    summarize(per, c->nrhs, info);
  } else if (info) {
    std::memset(info, 0, sizeof(*info));
    info->status = st;
  }
  return st;
}

// ---------------------------------------------------------------- PCG comparator
// Conjugate gradients with M = diag(Q) (Sec. 4.2's comparator) on the
// context's matrix and its one right-hand side, FP64, CSR rows in the
// context's current order; tol, maxit and x0 from aj_set.
extern "C" aj_status aj_pcg_solve(aj_ctx* c, double* x_out, int x_on_device, aj_info* info) {
  if (!c || (!x_out && c->n > 0) || c->nrhs != 1) return AJ_EINVAL;
  if (!c->have_prm) {
    aj_params p;
    aj_params_default(&p);
    aj_status st = aj_set(c, &p);
    if (st != AJ_OK) return st;
  }
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != c->dev) cudaSetDevice(c->dev);
  struct Restore {
    int dev, cur;
    ~Restore() { if (cur != dev) cudaSetDevice(cur); }
  } restore{c->dev, cur};
  const int n = (int)c->n;
  cudaStream_t s = c->stream;
  t_launches = 0;
  Workspace w;
  w.stream = &c->stream;
  struct Release {
    Workspace& w;
    ~Release() { w.release(); }
  } release{w};
  CK(cudaEventRecord(c->ev0, s));
  const size_t vb = ((size_t)n + 1) * 8;
  PcgArgs a;
  std::memset(&a, 0, sizeof(a));
  a.n = n;
  a.rp = c->rp;
  a.ci = c->ci;
  a.val = c->val64;
  a.b = c->b64;
  a.x = (double*)w.alloc(vb);
  a.r = (double*)w.alloc(vb);
  a.z = (double*)w.alloc(vb);
  a.p[0] = (double*)w.alloc(vb);
  a.p[1] = (double*)w.alloc(vb);
  a.q = (double*)w.alloc(2 * vb);
  int bps = 0;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, aj_pcg_kernel, kThreads, 0));
  const long long ntiles = std::max<long long>(1, ((long long)n + kThreads - 1) / kThreads);
  long long g = std::min<long long>((long long)std::max(1, bps) * c->sm_count, ntiles);
  if (c->prm.grid_ctas > 0) g = std::min<long long>(c->prm.grid_ctas, (long long)std::max(1, bps) * c->sm_count);
  const int grid = (int)std::max<long long>(1, g);
  a.part = (double*)w.alloc((size_t)2 * grid * 2 * 8);
  a.bar = (unsigned long long*)w.alloc(64);
  a.out_iters = (long long*)w.alloc(16);
  a.out_rn = (double*)w.alloc(16);
  if (!a.x || !a.r || !a.z || !a.p[0] || !a.p[1] || !a.q || !a.part || !a.bar || !a.out_iters || !a.out_rn)
    return AJ_ENOMEM;
  a.err = c->err;
  a.maxit = c->prm.maxit;
  a.tol = c->prm.tol;
  a.bnorm = std::sqrt(c->bnorm2[0]);
  aj_status e = load_x0(c);
  if (e != AJ_OK) return e;
  if (n > 0) CK(cudaMemcpyAsync(a.x, c->tmp64, (size_t)n * 8, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemsetAsync(a.bar, 0, 64, s));
  CK(cudaMemsetAsync(c->err, 0, 4, s));
  CK(cudaMemsetAsync(a.out_iters, 0, 16, s));
  CK(cudaMemsetAsync(a.out_rn, 0, 16, s));
  CK(cudaEventRecord(c->kev0, s));
  if (n > 0) {
    void* args[] = {&a};
    CK(cudaLaunchCooperativeKernel((const void*)aj_pcg_kernel, dim3(grid), dim3(kThreads), args, 0, s));
    counted();
  }
  CK(cudaEventRecord(c->kev1, s));
  long long iters = 0;
  double rn = 0.0;
  int err = 0;
  CK(cudaMemcpyAsync(&iters, a.out_iters, 8, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&rn, a.out_rn, 8, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&err, c->err, 4, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (err != 0) return err == kETimeout ? AJ_ETIMEOUT : AJ_ECUDA;
  double relres = 0.0, objgap = 0.0;
  e = fp64_report(c, a.x, &relres, &objgap, nullptr);
  if (e != AJ_OK) return e;
  e = write_output(c, a.x, x_out, x_on_device);
  if (e != AJ_OK) return e;
  CK(cudaEventRecord(c->ev1, s));
  CK(cudaEventSynchronize(c->ev1));
  float ms = 0.f, kms = 0.f;
  cudaEventElapsedTime(&ms, c->ev0, c->ev1);
  cudaEventElapsedTime(&kms, c->kev0, c->kev1);
  aj_status st = !std::isfinite(rn) ? AJ_ENONFINITE
                 : (rn <= c->prm.tol * a.bnorm) ? AJ_OK : AJ_EMAXIT;
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->iters = iters;
    info->sweeps = 2 * iters + 1;
    info->relres = relres;
    info->objgap = objgap;
    info->ms = ms;
    info->kernel_ms = kms;
    info->launches = t_launches;
    info->status = st;
  }
  return st;
}

extern "C" aj_status aj_restart_log(aj_ctx* c, int rhs, int64_t* iters, int64_t cap, int64_t* count) {
  if (!c || rhs < 0 || rhs >= c->nrhs || !count || cap < 0 || (cap > 0 && !iters)) return AJ_EINVAL;
  if ((int)c->rlog_h.size() <= rhs) { *count = 0; return AJ_OK; }
  const auto& v = c->rlog_h[rhs];
  *count = (int64_t)v.size();
  for (int64_t k = 0; k < cap && k < (int64_t)v.size(); k++) iters[k] = v[k];
  return AJ_OK;
}

// ---------------------------------------------------------------- state
struct StateHeader {
  uint64_t magic;
  int64_t n;
  int32_t nrhs, pol;
  int32_t state_bytes, pad;  // pad: sweep form of the saved run | row order (bit 8)
  double sb[kMaxRhs];
};
static const uint64_t kStateMagic = 0x414a535441544531ull;  // "AJSTATE1"

extern "C" aj_status aj_get_state(aj_ctx* c, void* buf, size_t* size) {
  if (!c || !size) return AJ_EINVAL;
  if (c->pol != AJ_FP64 && c->pol != AJ_DF64) return AJ_EINVAL;
  if ((int)c->st_h.size() != c->nrhs) return AJ_EINVAL;  // no finished solve yet
  const size_t vb = (size_t)c->n * c->nrhs * xelem_bytes(c->pol);
  const size_t need = sizeof(StateHeader) + sizeof(RhsState) * c->nrhs + 6 * vb;
  if (!buf) { *size = need; return AJ_OK; }
  if (*size < need) { *size = need; return AJ_EINVAL; }
  char* p = (char*)buf;
  StateHeader h;
  std::memset(&h, 0, sizeof(h));
  h.magic = kStateMagic;
  h.n = c->n;
  h.nrhs = c->nrhs;
  h.pol = c->pol;
  h.state_bytes = (int)sizeof(RhsState);
  h.pad = c->qx | (c->ordered << 8);
  for (int r = 0; r < kMaxRhs; r++) h.sb[r] = c->sb[r];
  std::memcpy(p, &h, sizeof(h));
  p += sizeof(h);
  std::memcpy(p, c->st_h.data(), sizeof(RhsState) * c->nrhs);
  p += sizeof(RhsState) * c->nrhs;
  for (int k = 0; k < 6; k++) {
    void* src = k < 3 ? c->x[k] : k < 5 ? c->u[k - 3] : c->dl;
    if (vb) CK(cudaMemcpyAsync(p, src, vb, cudaMemcpyDeviceToHost, c->stream));
    p += vb;
  }
  CK(cudaStreamSynchronize(c->stream));
  *size = need;
  return AJ_OK;
}

extern "C" aj_status aj_set_state(aj_ctx* c, const void* buf, size_t size) {
  if (!c || !buf || !c->have_prm) return AJ_EINVAL;
  if (c->pol != AJ_FP64 && c->pol != AJ_DF64) return AJ_EINVAL;
  if (size < sizeof(StateHeader)) return AJ_EINVAL;
  StateHeader h;
  std::memcpy(&h, buf, sizeof(h));
  const size_t vb = (size_t)c->n * c->nrhs * xelem_bytes(c->pol);
  const size_t need = sizeof(StateHeader) + sizeof(RhsState) * c->nrhs + 6 * vb;
  if (h.magic != kStateMagic || h.n != c->n || h.nrhs != c->nrhs || h.pol != c->pol ||
      h.state_bytes != (int)sizeof(RhsState) || h.pad != (c->qx | (c->ordered << 8)) || size < need)
    return AJ_EINVAL;
  const char* p = (const char*)buf + sizeof(h);
  c->st_h.resize(c->nrhs);
  std::memcpy(c->st_h.data(), p, sizeof(RhsState) * c->nrhs);
  p += sizeof(RhsState) * c->nrhs;
  for (int k = 0; k < 6; k++) {
    void* dst = k < 3 ? c->x[k] : k < 5 ? c->u[k - 3] : c->dl;
    if (vb) CK(cudaMemcpyAsync(dst, p, vb, cudaMemcpyHostToDevice, c->stream));
    p += vb;
  }
  CK(cudaStreamSynchronize(c->stream));
  for (int r = 0; r < kMaxRhs; r++) c->sb[r] = h.sb[r];
  c->resume = true;
  return AJ_OK;
}

// ---------------------------------------------------------------- batch
extern "C" aj_status aj_solve_batch(aj_ctx* const* ctx, int count, double* const* x_out,
                                    int x_on_device, aj_info* info) {
  if (count < 0 || (count > 0 && (!ctx || !x_out))) return AJ_EINVAL;
  if (count == 0) return AJ_OK;
  for (int i = 0; i < count; i++) {
    if (!ctx[i] || (!x_out[i] && ctx[i]->n > 0)) return AJ_EINVAL;
    for (int j = 0; j < i; j++)
      if (ctx[j] == ctx[i]) return AJ_EINVAL;  // a context appears once
  }
  for (int i = 0; i < count; i++)
    if (!ctx[i]->have_prm) {
      aj_params p;
      aj_params_default(&p);
      aj_status st = aj_set(ctx[i], &p);
      if (st != AJ_OK) return st;
    }
  aj_ctx* c0 = ctx[0];
  bool mixed = false;
  for (int i = 1; i < count; i++) {
    if (ctx[i]->dev != c0->dev || ctx[i]->pol != c0->pol) return AJ_EINVAL;
    mixed = mixed || ctx[i]->qx != c0->qx;
  }
  if (mixed) {
    // one lockstep batch per sweep form (AUTO gives SELL matrices the stored
    // form and CSR ones the lazy form; the kernel runs one form), in turn
    aj_status worst = AJ_OK;
    double ms_all = 0.0, kms_all = 0.0;
    int64_t launches_all = 0;
    for (int q = 0; q < 4; q++) {
      std::vector<aj_ctx*> cs;
      std::vector<double*> xs;
      std::vector<int> idx;
      for (int i = 0; i < count; i++)
        if (ctx[i]->qx == q) {
          cs.push_back(ctx[i]);
          xs.push_back(x_out[i]);
          idx.push_back(i);
        }
      if (cs.empty()) continue;
      std::vector<aj_info> inf(cs.size());
      const aj_status s = aj_solve_batch(cs.data(), (int)cs.size(), xs.data(), x_on_device, inf.data());
      if (s != AJ_OK && s != AJ_EMAXIT && s != AJ_EDIVERGED && s != AJ_ENONFINITE) return s;
      for (size_t k = 0; k < cs.size(); k++)
        if (info) info[idx[k]] = inf[k];
      // the launches of one form run one after another: the call's totals are their sums
      ms_all += inf[0].ms;
      kms_all += inf[0].kernel_ms;
      launches_all += inf[0].launches;
      if (s != AJ_OK && worst == AJ_OK) worst = s;
    }
    if (info)
      for (int i = 0; i < count; i++) {
        info[i].ms = ms_all;
        info[i].kernel_ms = kms_all;
        info[i].launches = launches_all;
      }
    return worst;
  }
  int dev_prev = 0;
  cudaGetDevice(&dev_prev);
  if (dev_prev != c0->dev) cudaSetDevice(c0->dev);
  // every context's GPU work runs on the first context's stream for the batch
  std::vector<cudaStream_t> saved(count);
  for (int i = 0; i < count; i++) {
    saved[i] = ctx[i]->stream;
    ctx[i]->stream = c0->stream;
    ctx[i]->kernel_ms = 0.0;
  }
  t_launches = 0;
  std::vector<aj_info> per((size_t)count * kMaxRhs);
  std::memset(per.data(), 0, per.size() * sizeof(aj_info));
  double kms = 0.0;
  aj_status st = AJ_OK;
  cudaEventRecord(c0->ev0, c0->stream);
  if (c0->pol == AJ_FP64 || c0->pol == AJ_DF64) {
    std::vector<DirectRun> d(count);
    std::vector<BatchItem> items;
    for (int i = 0; i < count && st == AJ_OK; i++) {
      st = direct_prepare(ctx[i], d[i]);
      items.push_back({ctx[i], &d[i].st, d[i].bvec, ctx[i]->prm.maxit, ctx[i]->prm.stop,
                       ctx[i]->prm.tol, ctx[i]->prm.fstar, d[i].fscale, ctx[i]->prm.maxit + 2});
    }
    if (st == AJ_OK) st = run_batched(items, true, &kms);
    for (int i = 0; i < count && st == AJ_OK; i++)
      st = direct_finish(ctx[i], d[i], x_out[i], x_on_device, per.data() + (size_t)i * kMaxRhs);
  } else {
    std::vector<aj_info*> pp(count);
    for (int i = 0; i < count; i++) pp[i] = per.data() + (size_t)i * kMaxRhs;
    st = ir_solve(ctx, count, x_out, x_on_device, pp.data(), true, &kms);
  }
  cudaEventRecord(c0->ev1, c0->stream);
  cudaEventSynchronize(c0->ev1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, c0->ev0, c0->ev1);
  for (int i = 0; i < count; i++) {
    ctx[i]->stream = saved[i];
    ctx[i]->resume = false;
  }
  if (dev_prev != c0->dev) cudaSetDevice(dev_prev);
  if (st != AJ_OK) return st;
  aj_status worst = AJ_OK;
  for (int i = 0; i < count; i++) {
    aj_info* pr = per.data() + (size_t)i * kMaxRhs;
    for (int r = 0; r < ctx[i]->nrhs; r++) {
      pr[r].ms = ms;
      pr[r].kernel_ms = kms;
      pr[r].launches = t_launches;
    }
    aj_info sum;
    summarize(pr, ctx[i]->nrhs, &sum);
    if (info) info[i] = sum;
    if (sum.status != AJ_OK && worst == AJ_OK) worst = sum.status;
  }
  return worst;
}

// ---------------------------------------------------------------- server
// Continuous batching.  A host thread runs rounds: one batched launch over
// every admitted request, each running at most `round_sweeps` sweeps from its
// resident state.  After a round, finished requests are retired (their device
// memory freed when the server created it) and queued requests are admitted,
// first fit, while the device-memory budget and the slot count allow.  The
// sweep sequence of a request does not depend on where rounds cut it, so its
// result equals a solo run with the same gang size.
struct ServerReq {
  uint64_t ticket = 0;
  aj_ctx* c = nullptr;
  bool owned = false;  // created by the server from a host copy (aj_submit_csr)
  int64_t n = 0, nnz = 0;
  int nrhs = 1;
  std::vector<int32_t> rp, ci;
  std::vector<double> val, b, x0;
  aj_params prm;
  size_t bytes = 0;
  cudaStream_t user_stream = nullptr;
  std::chrono::steady_clock::time_point t_submit;
  bool ir = false;
  DirectRun d;
  IrRun q;
  BatchItem item;
};

// A finished request's result: x is allocated when the request finishes,
// uninitialised (the device copy fills it), and handed over by aj_poll.
struct ServerDone {
  aj_status st = AJ_OK;
  aj_info info;
  std::unique_ptr<double[]> x;
  size_t m = 0;
};

struct aj_server {
  size_t budget = 0;
  int max_slots = 1;
  int dev = 0;
  cudaStream_t stream = nullptr;      // rounds
  cudaStream_t adm_stream = nullptr;  // admission: context creation and set-up
  std::thread adm_th;
  std::deque<ServerReq*> ready;       // started by the admission thread, waiting for a round
  int preparing = 0;                  // being started by the admission thread
  long long round_sweeps = 32;
  LockWs lws;  // lockstep launch buffers, kept for the server's lifetime
  std::mutex mu;
  std::condition_variable cv;
  std::deque<ServerReq*> queue;
  std::vector<ServerReq*> active;
  std::map<uint64_t, ServerDone> done;
  std::map<uint64_t, int> pending;  // tickets submitted and not yet finished
  size_t in_use = 0;
  uint64_t next = 1;
  bool stop = false;
  std::thread th;
  aj_server_stats stats;
};

static size_t ctx_bytes(const aj_ctx* c) { return c->base.bytes + c->pws.bytes + c->sws.bytes + c->ows.bytes; }

// Device bytes a context of this shape allocates (aj_create + aj_set).
static size_t estimate_bytes(int64_t n, int64_t nnz, int nrhs, int precision) {
  const size_t m = (size_t)n * nrhs + 1;
  const size_t xe = xelem_bytes(precision);
  size_t v = (size_t)(n + 17) * 4 + (size_t)(nnz + 16) * 12 + (size_t)(n + 1) * 16 + m * 16;
  v += (size_t)(n / kSetupThreads + 2) * kMaxRhs * 3 * 8;
  if (precision != AJ_FP64) v += (size_t)(nnz + 16) * velem_bytes(precision) + m * xe + (size_t)(n + 1) * xe;
  v += 5 * m * xe + 2 * m * 8;
  v += (size_t)2 * 2048 * kMaxRhs * kNRed * 8 + 4096;
  return v;
}

static void server_complete(aj_server* s, ServerReq* r, aj_status st, const aj_info* per,
                            std::unique_ptr<double[]>&& x, size_t m) {
  ServerDone dn;
  dn.st = st;
  std::memset(&dn.info, 0, sizeof(dn.info));
  if (per && r->c) summarize(per, r->c->nrhs, &dn.info);
  dn.info.status = st == AJ_OK ? dn.info.status : st;
  dn.info.ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() -
                                                         r->t_submit).count();
  dn.x = std::move(x);
  dn.m = dn.x ? m : 0;
  if (r->c) {
    if (r->owned) aj_destroy(r->c);
    else aj_set_stream(r->c, r->user_stream);
  }
  std::lock_guard<std::mutex> lk(s->mu);
  s->in_use -= std::min(s->in_use, r->bytes);
  s->pending.erase(r->ticket);
  s->stats.completed++;
  s->done[r->ticket] = std::move(dn);
  delete r;
  s->cv.notify_all();
}

// Admission, on the admission thread: create the context if the server owns
// it and start its run, all on stream st; the round thread takes it over.
static aj_status server_start(aj_server* s, ServerReq* r, cudaStream_t st) {
  if (r->owned) {
    aj_csr Q;
    Q.n = r->n;
    Q.nnz = r->nnz;
    Q.row_ptr = r->rp.data();
    Q.col = r->ci.data();
    Q.val = r->val.data();
    Q.on_device = 0;
    aj_status e = aj_create(&Q, r->b.data(), r->nrhs, &r->c);
    if (e != AJ_OK) return e;
    e = aj_set_stream(r->c, st);
    if (e != AJ_OK) return e;
    aj_params p = r->prm;
    p.x0 = r->x0.empty() ? nullptr : r->x0.data();
    p.x0_on_device = 0;
    e = aj_set(r->c, &p);
    if (e != AJ_OK) return e;
    const size_t actual = ctx_bytes(r->c);
    std::lock_guard<std::mutex> lk(s->mu);
    s->in_use = s->in_use - std::min(s->in_use, r->bytes) + actual;
    r->bytes = actual;
  } else {
    r->user_stream = r->c->stream;
    aj_status e = aj_set_stream(r->c, st);
    if (e != AJ_OK) return e;
    if (!r->c->have_prm) {
      aj_params p;
      aj_params_default(&p);
      aj_status e = aj_set(r->c, &p);
      if (e != AJ_OK) return e;
    }
  }
  aj_ctx* c = r->c;
  c->resume = false;
  c->kernel_ms = 0.0;
  CK(cudaMemsetAsync(c->rlog, 0xff, (size_t)kMaxRhs * c->rlog_cap * 8, st));
  r->ir = !(c->pol == AJ_FP64 || c->pol == AJ_DF64);
  if (!r->ir) {
    aj_status e = direct_prepare(c, r->d);
    if (e != AJ_OK) return e;
    r->item = {c, &r->d.st, r->d.bvec, c->prm.maxit, c->prm.stop, c->prm.tol, c->prm.fstar,
               r->d.fscale, s->round_sweeps};
  } else {
    aj_status e = ir_begin(c, r->q);
    if (e == AJ_OK) e = ir_check(c, r->q);
    if (e != AJ_OK) return e;
    if (!r->q.finished) r->item = ir_inner_setup(c, r->q);
  }
  CK(cudaGetLastError());
  // hand the context to the round stream (waits for the set-up above)
  return aj_set_stream(c, s->stream);
}

// After a round: retire what finished, start the next inner solve of the
// refinement requests.  Returns true when r is finished (completed).
static bool server_advance(aj_server* s, ServerReq* r) {
  aj_ctx* c = r->c;
  aj_info per[kMaxRhs];
  std::memset(per, 0, sizeof(per));
  const size_t m = (size_t)c->n * c->nrhs;
  std::unique_ptr<double[]> x;
  aj_status e = AJ_OK;
  if (!r->ir) {
    for (int k = 0; k < c->nrhs; k++)
      if (!r->d.st[k].done) return false;
    x.reset(new double[std::max<size_t>(m, 1)]);
    e = direct_finish(c, r->d, x.get(), 0, per);
  } else {
    if (!r->q.finished) {
      for (int k = 0; k < c->nrhs; k++)
        if (!r->q.st[k].done) return false;
      e = ir_inner_finish(c, r->q);
      if (e == AJ_OK) e = ir_check(c, r->q);
      if (e == AJ_OK && !r->q.finished) {
        cudaMemsetAsync(c->rlog, 0xff, (size_t)kMaxRhs * c->rlog_cap * 8, s->stream);
        r->item = ir_inner_setup(c, r->q);
        return false;
      }
    }
    if (e == AJ_OK) {
      x.reset(new double[std::max<size_t>(m, 1)]);
      e = ir_end(c, r->q, x.get(), 0, per);
    }
  }
  aj_status st = e;
  if (st == AJ_OK)
    for (int k = 0; k < c->nrhs; k++)
      if (per[k].status != AJ_OK && st == AJ_OK) st = per[k].status;
  if (e != AJ_OK) x.reset();
  server_complete(s, r, st, e == AJ_OK ? per : nullptr, std::move(x), m);
  return true;
}

// The admission thread: takes queued requests first fit, in submission
// order, while the device memory of admitted requests stays within the
// budget and the slots allow, creates and starts them on its own stream
// (host-to-device copies, set-up kernels, format and order choice), and
// hands them to the round thread.  That work overlaps the rounds.
static void server_admit_main(aj_server* s) {
  cudaSetDevice(s->dev);
  for (;;) {
    ServerReq* r = nullptr;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      auto pick = [&]() -> std::deque<ServerReq*>::iterator {
        const int used = (int)(s->active.size() + s->ready.size()) + s->preparing;
        if (used >= s->max_slots) return s->queue.end();
        for (auto it = s->queue.begin(); it != s->queue.end(); ++it)
          if (s->in_use + (*it)->bytes <= s->budget) return it;
        return s->queue.end();
      };
      s->cv.wait(lk, [&] { return s->stop || pick() != s->queue.end(); });
      if (s->stop) break;
      auto it = pick();
      r = *it;
      s->queue.erase(it);
      s->in_use += r->bytes;
      s->stats.admitted++;
      s->stats.peak_bytes = std::max<uint64_t>(s->stats.peak_bytes, s->in_use);
      s->preparing++;
    }
    const aj_status e = server_start(s, r, s->adm_stream);
    if (e != AJ_OK) {
      {
        std::lock_guard<std::mutex> lk(s->mu);
        s->preparing--;
      }
      server_complete(s, r, e, nullptr, nullptr, 0);
      continue;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    s->preparing--;
    s->ready.push_back(r);
    s->cv.notify_all();
  }
}

// The round thread: takes the started requests and runs rounds over them.
static void server_main(aj_server* s) {
  cudaSetDevice(s->dev);
  for (;;) {
    std::vector<ServerReq*> admit;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      if (s->active.empty())
        s->cv.wait(lk, [&] { return s->stop || !s->ready.empty(); });
      if (s->stop) break;
      admit.assign(s->ready.begin(), s->ready.end());
      s->ready.clear();
    }
    for (ServerReq* r : admit) {
      if (r->ir && r->q.finished) server_advance(s, r);
      else s->active.push_back(r);
    }
    if (s->active.empty()) continue;
    // one round: a batched launch per (precision, sweep form) over every admitted request
    std::map<std::pair<int, int>, std::vector<BatchItem>> groups;
    for (ServerReq* r : s->active) {
      r->item.max_sweeps = s->round_sweeps;
      groups[{r->c->pol, r->c->qx}].push_back(r->item);
    }
    double kms = 0.0;
    aj_status e = AJ_OK;
    for (auto& g : groups) {
      e = run_batched(g.second, false, &kms, &s->lws, s->round_sweeps);
      if (e != AJ_OK) break;
    }
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->stats.rounds++;
      s->stats.peak_active = std::max<int64_t>(s->stats.peak_active, (int64_t)s->active.size());
      s->stats.kernel_ms += kms;
    }
    // keep a round between about 1 and 4 ms of device time
    if (kms < 1.0 && s->round_sweeps < 1024) s->round_sweeps *= 2;
    else if (kms > 4.0 && s->round_sweeps > 4) s->round_sweeps /= 2;
    std::vector<ServerReq*> still;
    for (ServerReq* r : s->active) {
      if (e != AJ_OK) server_complete(s, r, e, nullptr, nullptr, 0);
      else if (!server_advance(s, r)) still.push_back(r);
    }
    s->active.swap(still);
  }
  for (ServerReq* r : s->active) server_complete(s, r, AJ_ECUDA, nullptr, nullptr, 0);
  s->active.clear();
}

extern "C" aj_status aj_server_create(size_t hbm_budget_bytes, int max_slots, aj_server** out) {
  if (!out || max_slots < 1 || hbm_budget_bytes == 0) return AJ_EINVAL;
  *out = nullptr;
  aj_server* s = new aj_server();
  s->budget = hbm_budget_bytes;
  s->max_slots = max_slots;
  std::memset(&s->stats, 0, sizeof(s->stats));
  cudaGetDevice(&s->dev);
  if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    s->stream = nullptr;
    delete s;
    return AJ_ECUDA;
  }
  if (cudaStreamCreateWithFlags(&s->adm_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    s->adm_stream = nullptr;
    cudaStreamDestroy(s->stream);
    s->stream = nullptr;
    delete s;
    return AJ_ECUDA;
  }
  s->lws.stream = s->stream;
  s->th = std::thread(server_main, s);
  s->adm_th = std::thread(server_admit_main, s);
  *out = s;
  return AJ_OK;
}

static aj_status server_enqueue(aj_server* s, ServerReq* r, uint64_t* ticket) {
  std::lock_guard<std::mutex> lk(s->mu);
  r->ticket = s->next++;
  r->t_submit = std::chrono::steady_clock::now();
  s->pending[r->ticket] = 1;
  s->queue.push_back(r);
  *ticket = r->ticket;
  s->cv.notify_all();
  return AJ_OK;
}

extern "C" aj_status aj_submit(aj_server* s, aj_ctx* c, uint64_t* ticket) {
  if (!s || !c || !ticket) return AJ_EINVAL;
  if (c->dev != s->dev) return AJ_EINVAL;
  const size_t bytes = ctx_bytes(c);
  if (bytes > s->budget) return AJ_EBUSY;
  ServerReq* r = new ServerReq();
  r->c = c;
  r->bytes = bytes;
  return server_enqueue(s, r, ticket);
}

extern "C" aj_status aj_submit_csr(aj_server* s, const aj_csr* Q, const double* b, int nrhs,
                                   const aj_params* p, uint64_t* ticket) {
  if (!s || !Q || !ticket || nrhs < 1 || nrhs > kMaxRhs || Q->n < 0 || Q->nnz < 0) return AJ_EINVAL;
  if (Q->n >= (1ll << 31) - 1 || Q->nnz >= (1ll << 31) - 1) return AJ_EINVAL;
  if (Q->n > 0 && (!Q->row_ptr || !b)) return AJ_EINVAL;
  if (Q->nnz > 0 && (!Q->col || !Q->val)) return AJ_EINVAL;
  aj_params prm;
  if (p) prm = *p;
  else aj_params_default(&prm);
  if (prm.precision < AJ_FP64 || prm.precision > AJ_BF16_IR) return AJ_EINVAL;
  const size_t est = estimate_bytes(Q->n, Q->nnz, nrhs, prm.precision);
  if (est > s->budget) return AJ_EBUSY;
  ServerReq* r = new ServerReq();
  r->owned = true;
  r->n = Q->n;
  r->nnz = Q->nnz;
  r->nrhs = nrhs;
  r->prm = prm;
  r->bytes = est;
  const size_t m = (size_t)Q->n * nrhs;
  r->rp.resize((size_t)Q->n + 1);
  r->ci.resize((size_t)Q->nnz);
  r->val.resize((size_t)Q->nnz);
  r->b.resize(m);
  const cudaMemcpyKind k = Q->on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost;
  bool ok = cudaMemcpy(r->rp.data(), Q->row_ptr, r->rp.size() * 4, k) == cudaSuccess &&
            (Q->nnz == 0 || (cudaMemcpy(r->ci.data(), Q->col, r->ci.size() * 4, k) == cudaSuccess &&
                             cudaMemcpy(r->val.data(), Q->val, r->val.size() * 8, k) == cudaSuccess)) &&
            (m == 0 || cudaMemcpy(r->b.data(), b, m * 8, k) == cudaSuccess);
  if (ok && prm.x0) {
    r->x0.resize(m);
    ok = m == 0 || cudaMemcpy(r->x0.data(), prm.x0, m * 8,
                              prm.x0_on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost) ==
                       cudaSuccess;
  }
  if (!ok) {
    cudaGetLastError();
    delete r;
    return AJ_ECUDA;
  }
  r->prm.x0 = nullptr;
  return server_enqueue(s, r, ticket);
}

extern "C" aj_status aj_poll(aj_server* s, uint64_t ticket, double* x_out, aj_info* info) {
  if (!s) return AJ_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->done.find(ticket);
  if (it == s->done.end()) return s->pending.count(ticket) ? AJ_PENDING : AJ_EINVAL;
  if (x_out && it->second.x) std::memcpy(x_out, it->second.x.get(), it->second.m * 8);
  if (info) *info = it->second.info;
  const aj_status st = it->second.st;
  s->done.erase(it);
  return st;
}

extern "C" aj_status aj_server_wait(aj_server* s, uint64_t ticket, double timeout_ms) {
  if (!s) return AJ_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto ready = [&] { return s->done.count(ticket) || !s->pending.count(ticket); };
  if (timeout_ms < 0) s->cv.wait(lk, ready);
  else s->cv.wait_for(lk, std::chrono::duration<double, std::milli>(timeout_ms), ready);
  if (s->done.count(ticket)) return AJ_OK;
  return s->pending.count(ticket) ? AJ_PENDING : AJ_EINVAL;
}

extern "C" aj_status aj_server_get_stats(aj_server* s, aj_server_stats* out) {
  if (!s || !out) return AJ_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->stats;
  out->in_use_bytes = s->in_use;
  out->queued = (int64_t)s->queue.size();
  return AJ_OK;
}

extern "C" void aj_server_destroy(aj_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv.notify_all();
  }
  if (s->th.joinable()) s->th.join();
  if (s->adm_th.joinable()) s->adm_th.join();
  // started but never run: drop them (owned contexts destroyed, others get their stream back)
  std::vector<ServerReq*> left(s->ready.begin(), s->ready.end());
  s->ready.clear();
  for (ServerReq* r : left) server_complete(s, r, AJ_ECUDA, nullptr, nullptr, 0);
  for (ServerReq* r : s->queue) delete r;
  s->queue.clear();
  if (s->stream) {
    s->lws.mem.release();
    cudaStreamSynchronize(s->stream);
    cudaStreamDestroy(s->stream);
  }
  if (s->adm_stream) {
    cudaStreamSynchronize(s->adm_stream);
    cudaStreamDestroy(s->adm_stream);
  }
  delete s;
}

extern "C" uint64_t aj_kernel_launches(void) { return g_launches.load(); }

extern "C" void aj_cache_stats(uint64_t* order_hits, uint64_t* order_misses, uint64_t* tune_hits,
                               uint64_t* tune_misses) {
  if (order_hits) *order_hits = g_order_hits.load();
  if (order_misses) *order_misses = g_order_misses.load();
  if (tune_hits) *tune_hits = g_tune_hits.load();
  if (tune_misses) *tune_misses = g_tune_misses.load();
}

extern "C" aj_status aj_test_barrier_stall(int cta, double timeout_ms) {
  if (cta < -1 || !(timeout_ms > 0.0) || timeout_ms > 4000.0) return AJ_EINVAL;
  g_stall_timeout_ns.store((long long)(timeout_ms * 1e6));
  g_stall_cta.store(cta);
  return AJ_OK;
}

extern "C" aj_status aj_test_alloc_fail(int64_t after) {
  if (after < -1) return AJ_EINVAL;
  g_alloc_fail_after.store(after);
  return AJ_OK;
}
