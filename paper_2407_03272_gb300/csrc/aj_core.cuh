// aj_core.cuh -- device side of the fused accelerated-Jacobi (AJ) iteration.
//
// One persistent, grid-synchronised kernel runs Algorithm alg-jacobi of
// Liang, Pang, Toh and Yang (arXiv 2407.03272, Section 3) with the restart
// rule of Algorithm alg-apg-re (Section 2.2).  Each sweep s streams the matrix
// once and, per owned row i and right-hand side r, forms x^s from
// y^s = x^{s-1} + beta (x^{s-1} - x^{s-2}) without ever storing y:
//
//   (Q y^s)_i = sx_i + beta (sx_i - sp_i),  sx = Q x^{s-1},  sp = Q x^{s-2}
//   g_i = (Q y^s)_i - b_i,   x^s_i = y^s_i - J^{-1}_ii g_i              (x^t = y^t + J^-1(b - Q y^t))
//   d  += g_i (x^s_i - x^{s-1}_i)                                      (restart test <Q y^t - b, x^t - x^{t-1}>)
//   rr += (b_i - sx_i)^2                                               (exact residual of x^{s-1})
//
// Two sweep forms give sp:
//   lazy  (QX = false): sp is a second row sum over the gathered x^{s-2};
//         two multiply-adds per stored entry, four n-vectors of traffic.
//   stored (QX = true): u = Q x is written every sweep (u^{s-1} = sx) and
//         u^{s-2} is read back for own rows only; one multiply-add per stored
//         entry, two more n-vectors of traffic.  On GB300 FP64 issue is the
//         binding resource of the FP64 policy, so it uses this form.
// After a grid barrier every CTA sums the per-CTA partials in one fixed order
// (identical bits in every CTA), checks the stop test for x^{s-1}, then takes
// the restart/momentum branch for iteration s.  Buffers rotate by index.
//
// Precision policies (template parameter P):
//   PolF64  IEEE FP64 everywhere (FMA row sums).
//   PolDF64 double-float: values/vectors are (hi, lo) FP32 pairs; row sums use
//           TwoProd/TwoSum error-free transforms (Ogita, Rump and Oishi,
//           "Accurate sum and dot product", SIAM J. Sci. Comput. 26, 2005) and
//           the row update uses the double-word algorithms of Joldes, Muller
//           and Popescu ("Tight and rigorous error bounds for basic building
//           blocks of double-word arithmetic", ACM TOMS 44, 2017).  Runs on the
//           FP32 pipes, which on GB300 issue ~70x more operations than FP64.
//   PolF32  FP32 values, vectors and row arithmetic.
//   PolB16  BF16 values, FP32 vectors and row arithmetic.
// The restart/stop reductions are FP64 in every policy: per-thread
// compensated double-float accumulators (F32/BF16/DF64) or FP64 (F64),
// combined in FP64 across threads, CTAs and the grid.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

// SELL sweeps: the instantiation (3: SELL alone, 1: the any-format one) and
// the tile order (0: sliced tiles, then long-row tiles, then huge rows;
// 1: huge rows and long-row tiles first -- measured slower on the 8.4M-vertex
// Chung-Lu graph, 0.87 against 0.79 ms per FP32 sweep)
#ifndef AJ_SELL_FM
#define AJ_SELL_FM 3
#endif
#ifndef AJ_SELL_HEAVY_FIRST
#define AJ_SELL_HEAVY_FIRST 0
#endif
// SELL: 1 rotates the slices of a tile over the warps from tile to tile
// (0: warp w always takes slice w; 1.04 against 0.87 ms per FP32 sweep of that graph)
#ifndef AJ_SELL_ROTATE
#define AJ_SELL_ROTATE 1
#endif

namespace aj {

constexpr int kThreads = 256;  // threads per CTA = rows per tile (one row per thread)
constexpr int kWarps = kThreads / 32;
constexpr int kMaxRhs = 4;
constexpr int kNRed = 5;       // per right-hand side: d, gg, rr, xqx, bx
constexpr int kLongRow = 32;   // rows longer than this are summed by the whole warp
constexpr unsigned long long kBarrierTimeoutNs = 4000000000ull;  // 4 s per barrier wait
constexpr long long kBarrierMaxSpins = 1ll << 27;

// status codes shared with aj.h (kept numerically identical)
constexpr int kOk = 0, kEMaxit = -4, kEDiverged = -5, kENonfinite = -6, kETimeout = -7;

enum StopKind { kStopRelres = 0, kStopObjgap = 1, kStopNone = 2 };

// Per right-hand-side solver state.  Every CTA keeps an identical copy in
// shared memory; CTA 0 writes it back to global memory at exit.
struct RhsState {
  double alpha;       // alpha_t of the next iteration t = cur_t + 1
  double beta;        // y^{t+1} = x^t + beta (x^t - x^{t-1}) for the next sweep
  double bnorm2;      // ||b||^2 (FP64)
  double rr0;         // squared residual of x^0 (divergence guard)
  double relres;      // relative residual of the last checked iterate
  double fval;        // f(x) of the last checked iterate (objective stop only)
  long long t;        // index of the iterate in buffer `cur`
  long long ell;      // restarts so far
  long long K;        // K_ell
  long long Kre;      // K_re
  long long t_final;  // index of the returned iterate
  int cur, prev, nxt; // buffer indices of x^t, x^{t-1} (may equal cur), spare
  int done;           // 1 once this right-hand side has stopped
  int status;         // kOk / kEMaxit / kEDiverged / kENonfinite
  int uw;             // stored form: u buffer written this sweep (Q x^t); 1 - uw holds Q x^{t-1}
  // explicit-y form (SF = 3) only:
  int yb;             // u buffer holding y^{t+1} for the next sweep (unless cur == prev:
                      // then y^{t+1} = x^t is the buffer cur itself)
  int chk;            // the next sweep also sums Q x^t for the exact stop test
  int near;           // the monitor is within kNearFactor of the stop: sum it every sweep
  int pad_;
  double beta_next;   // beta_{t+2} = (alpha_{t+1} - 1) / alpha_{t+2}: the next sweep writes
                      // y^{t+2} = x^{t+1} + beta_next (x^{t+1} - x^t), the point iteration
                      // t+2 uses unless iteration t+1 restarts
  double gmon;        // the last ||Q y - b||^2 summed (the monitor of the check schedule)
  double gcal;        // the largest ||b - Q x||^2 / monitor seen on check sweeps (>= 1 used)
};

// ----------------------------------------------------------------------------
// Memory helpers.  Iterate buffers are rewritten by other CTAs between sweeps,
// so they are read at L2 (ld.global.cg), never through the incoherent L1/tex
// paths.  The matrix, b and J^{-1} never change during a launch.
template <class T>
__device__ __forceinline__ T ld_l2(const T* p) { return __ldcg(p); }
template <class T>
__device__ __forceinline__ T ld_ro(const T* p) { return __ldg(p); }
// Gathers of the iterate x^{s-1} (and x^{s-2} in the lazy form) may be
// cached in L1 (AJ_GATHER_L1, default on): within a sweep those buffers are
// read only, and the writes of the previous sweep are ordered before these
// loads by the grid barrier (release/acquire at GPU scope by thread 0, then
// the CTA barrier), which the PTX memory model makes visible to them.  The
// parity tests include systems whose whole iterate fits in one SM's L1 for
// hundreds of sweeps.  Measured gain: 12 % per sweep on a power-law graph in
// SELL (hub columns are gathered by many rows), 1-2 % on stencils.
#ifndef AJ_GATHER_L1
#define AJ_GATHER_L1 1
#endif
template <class T>
__device__ __forceinline__ T ld_gather(const T* p) {
#if AJ_GATHER_L1
  return __ldca(p);
#else
  return __ldcg(p);
#endif
}
template <class T>
__device__ __forceinline__ void st_l2(T* p, T v) { __stcg(p, v); }

// Asynchronous 16-byte copies global -> shared (cp.async, read at L2 like
// ld_l2), src_bytes <= 16 of them read and the rest of the 16 zero-filled;
// both addresses 16-byte aligned.  A thread's copies form groups
// (commit); wait<N> returns when all but the newest N of its groups have
// landed.  The waits are the hardware's own: no spin in this code.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int src_bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_add_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier for a cooperative (co-resident) launch.  `target` is the
// arrival count that completes this barrier (k * gridDim.x for the k-th).
// Every wait is bounded: after timeout_ns (or kBarrierMaxSpins polls) the CTA
// records kETimeout in *err and returns false; a CTA that sees *err != 0 also
// returns false.  `withhold` keeps this CTA's arrival back (failure-detection
// tests: the other CTAs' waits then run out and the launch ends with
// kETimeout; the withholding CTA waits, bounded, like the others).
__device__ __forceinline__ bool grid_sync(unsigned long long* bar, unsigned long long target,
                                          int* err, unsigned int nctas,
                                          unsigned long long timeout_ns = kBarrierTimeoutNs,
                                          bool withhold = false) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    if (nctas > 1) {
      __threadfence();
      if (!withhold) red_release_add_u64(bar, 1ull);
      unsigned long long t0 = global_ns();
      long long spins = 0;
      while (ld_acquire_u64(bar) < target) {
        ++spins;
        if ((spins & 63) == 0) {
          if (*(volatile int*)err != 0) { ok = 0; break; }
          if (global_ns() - t0 > timeout_ns || spins > kBarrierMaxSpins) {
            atomicCAS(err, 0, kETimeout);
            ok = 0;
            break;
          }
        }
        __nanosleep(40);
      }
      __threadfence();
    }
    if (*(volatile int*)err != 0) ok = 0;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// ----------------------------------------------------------------------------
// Double-word (FP32 pair) building blocks: Knuth's TwoSum, Dekker's
// Fast2Sum (|a| >= |b|), FMA-based TwoProd.
struct dw {
  float hi, lo;
};
__device__ __forceinline__ dw two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ dw fast_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float e = __fsub_rn(b, __fsub_rn(s, a));
  return {s, e};
}
__device__ __forceinline__ dw two_prod(float a, float b) {
  float p = __fmul_rn(a, b);
  float e = __fmaf_rn(a, b, -p);
  return {p, e};
}
// Accurate double-word + double-word (Joldes-Muller-Popescu Alg. 6, error <= 3u^2).
__device__ __forceinline__ dw dw_add(dw x, dw y) {
  dw s = two_sum(x.hi, y.hi);
  dw t = two_sum(x.lo, y.lo);
  float c = __fadd_rn(s.lo, t.hi);
  dw v = fast_two_sum(s.hi, c);
  float w = __fadd_rn(t.lo, v.lo);
  return fast_two_sum(v.hi, w);
}
__device__ __forceinline__ dw dw_neg(dw x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ dw dw_sub(dw x, dw y) { return dw_add(x, dw_neg(y)); }
// Double-word x double-word with FMA (Joldes-Muller-Popescu Alg. 12, error <= 4u^2).
__device__ __forceinline__ dw dw_mul(dw x, dw y) {
  dw c = two_prod(x.hi, y.hi);
  float tl0 = __fmul_rn(x.lo, y.lo);
  float tl1 = __fmaf_rn(x.hi, y.lo, tl0);
  float cl2 = __fmaf_rn(x.lo, y.hi, tl1);
  float cl3 = __fadd_rn(c.lo, cl2);
  return fast_two_sum(c.hi, cl3);
}
__device__ __forceinline__ dw dw_from_double(double v) {
  float h = __double2float_rn(v);
  float l = __double2float_rn(v - (double)h);
  return {h, l};
}
__device__ __forceinline__ double dw_to_double(dw x) { return (double)x.hi + (double)x.lo; }

// Compensated running sum (double-word accumulator) fed with exact products.
struct acc_dw {
  float hi, lo;
};
__device__ __forceinline__ void acc_zero(acc_dw& a) { a.hi = 0.f; a.lo = 0.f; }
__device__ __forceinline__ void acc_add_term(acc_dw& a, float ph, float pl) {
  dw s = two_sum(a.hi, ph);
  a.hi = s.hi;
  a.lo = __fadd_rn(a.lo, __fadd_rn(s.lo, pl));
}
__device__ __forceinline__ double acc_value(const acc_dw& a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ void acc_zero(double& a) { a = 0.0; }
__device__ __forceinline__ double acc_value(double a) { return a; }

// ----------------------------------------------------------------------------
// Precision policies.  kMinBlocks / kMinBlocksMulti: co-resident CTAs per SM
// the register allocation must allow for one right-hand side and for the
// lanes-per-row form of several (measured on GB300, fixed-iteration sweeps of
// the 256^3 Poisson system and of a 1024^2 grid with 4 RHS):
//   FP64   4 / 4  (FP64-issue bound; 3 CTAs/SM is 18 % slower)
//   DF64   4 / 4  (5 CTAs/SM is 7 % slower)
//   FP32   6 / 4  (one RHS: 6 CTAs/SM 23 % faster than 4 in the lazy form;
//                  4 RHS: 4 CTAs/SM 20 % faster than 6)
//   BF16   8 / 4  (one RHS: 8 CTAs/SM 30 % faster than 4 in the lazy form)
#ifndef AJ_MINB_F64
#define AJ_MINB_F64 4
#endif
#ifndef AJ_MINB_DF64
#define AJ_MINB_DF64 4
#endif
#ifndef AJ_MINB_F32
#define AJ_MINB_F32 6
#endif
#ifndef AJ_MINB_B16
#define AJ_MINB_B16 8
#endif
#ifndef AJ_MINB_MULTI
#define AJ_MINB_MULTI 4
#endif
struct PolF64 {
  using V = double;  // stored matrix value
  using X = double;  // stored vector element
  using S = double;  // row arithmetic
  using A = double;  // per-thread reduction accumulator
  static constexpr int kId = 0;
  static constexpr int kMinBlocks = AJ_MINB_F64;
  static constexpr int kMinBlocksMulti = AJ_MINB_MULTI;
  __device__ static S zero() { return 0.0; }
  __device__ static S from_x(X v) { return v; }
  __device__ static S ldx(const X* p) { return ld_l2(p); }
  __device__ static S ldg(const X* p) { return ld_gather(p); }
  __device__ static S ldr(const X* p) { return ld_ro(p); }
  __device__ static void stx(X* p, S v) { st_l2(p, v); }
  __device__ static V ldv(const V* p) { return ld_ro(p); }
  __device__ static V vzero() { return 0.0; }
  __device__ static void macv(S& acc, V v, S x) { acc = fma(v, x, acc); }
  __device__ static void mac(S& acc, const V* v, S x) { macv(acc, ldv(v), x); }
  __device__ static S finish(S a) { return a; }
  __device__ static S neg(S a) { return -a; }
  __device__ static S add(S a, S b) { return a + b; }
  __device__ static S sub(S a, S b) { return a - b; }
  __device__ static S mul(S a, S b) { return a * b; }
  __device__ static S fma_(S a, S b, S c) { return fma(a, b, c); }  // a*b + c
  __device__ static S fnma(S a, S b, S c) { return fma(-a, b, c); }  // c - a*b
  __device__ static S coef(double c) { return c; }
  __device__ static void acc_prod(A& a, S u, S v) { a = fma(u, v, a); }
  __device__ static S shfl_xor(S v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
  __device__ static S shfl(S v, int src) { return __shfl_sync(0xffffffffu, v, src); }
  __device__ static S combine(S a, S b) { return a + b; }
  __device__ static bool finite(S v) { return isfinite(v); }
};

struct PolDF64 {
  using V = float2;
  using X = float2;
  using S = dw;
  using A = acc_dw;
  static constexpr int kId = 1;
  static constexpr int kMinBlocks = AJ_MINB_DF64;
  static constexpr int kMinBlocksMulti = AJ_MINB_MULTI;
  __device__ static S zero() { return {0.f, 0.f}; }
  __device__ static S from_x(X v) { return {v.x, v.y}; }
  __device__ static S ldx(const X* p) { float2 v = ld_l2(p); return {v.x, v.y}; }
  __device__ static S ldg(const X* p) { float2 v = ld_gather(p); return {v.x, v.y}; }
  __device__ static S ldr(const X* p) { float2 v = ld_ro(p); return {v.x, v.y}; }
  __device__ static void stx(X* p, S v) { st_l2(p, make_float2(v.hi, v.lo)); }
  __device__ static V ldv(const V* p) { return ld_ro(p); }
  __device__ static V vzero() { return make_float2(0.f, 0.f); }
  __device__ static void mac(S& acc, const V* vp, S x) { macv(acc, ldv(vp), x); }
  // acc += v * x with the product split exactly (TwoProd) and cross terms folded
  // into the low word; the sum of high words is kept by TwoSum (Dot2 pattern).
  __device__ static void macv(S& acc, V v, S x) {
    dw p = two_prod(v.x, x.hi);
    float pl = __fmaf_rn(v.x, x.lo, p.lo);
    pl = __fmaf_rn(v.y, x.hi, pl);
    dw s = two_sum(acc.hi, p.hi);
    acc.hi = s.hi;
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(s.lo, pl));
  }
  __device__ static S finish(S a) { return fast_two_sum_ordered(a); }
  __device__ static S fast_two_sum_ordered(S a) { return two_sum(a.hi, a.lo); }
  __device__ static S neg(S a) { return dw_neg(a); }
  __device__ static S add(S a, S b) { return dw_add(a, b); }
  __device__ static S sub(S a, S b) { return dw_sub(a, b); }
  __device__ static S mul(S a, S b) { return dw_mul(a, b); }
  __device__ static S fma_(S a, S b, S c) { return dw_add(dw_mul(a, b), c); }
  __device__ static S fnma(S a, S b, S c) { return dw_sub(c, dw_mul(a, b)); }
  __device__ static S coef(double c) { return dw_from_double(c); }
  __device__ static void acc_prod(A& a, S u, S v) {
    dw p = two_prod(u.hi, v.hi);
    float pl = __fmaf_rn(u.hi, v.lo, p.lo);
    pl = __fmaf_rn(u.lo, v.hi, pl);
    acc_add_term(a, p.hi, pl);
  }
  __device__ static S shfl_xor(S v, int m) {
    return {__shfl_xor_sync(0xffffffffu, v.hi, m), __shfl_xor_sync(0xffffffffu, v.lo, m)};
  }
  __device__ static S shfl(S v, int src) {
    return {__shfl_sync(0xffffffffu, v.hi, src), __shfl_sync(0xffffffffu, v.lo, src)};
  }
  __device__ static S combine(S a, S b) { return dw_add(a, b); }
  __device__ static bool finite(S v) { return isfinite(v.hi) && isfinite(v.lo); }
};

struct PolF32 {
  using V = float;
  using X = float;
  using S = float;
  using A = acc_dw;
  static constexpr int kId = 2;
  static constexpr int kMinBlocks = AJ_MINB_F32;
  static constexpr int kMinBlocksMulti = AJ_MINB_MULTI;
  __device__ static S zero() { return 0.f; }
  __device__ static S from_x(X v) { return v; }
  __device__ static S ldx(const X* p) { return ld_l2(p); }
  __device__ static S ldg(const X* p) { return ld_gather(p); }
  __device__ static S ldr(const X* p) { return ld_ro(p); }
  __device__ static void stx(X* p, S v) { st_l2(p, v); }
  __device__ static V ldv(const V* p) { return ld_ro(p); }
  __device__ static V vzero() { return 0.f; }
  __device__ static void macv(S& acc, V v, S x) { acc = __fmaf_rn(v, x, acc); }
  __device__ static void mac(S& acc, const V* v, S x) { macv(acc, ldv(v), x); }
  __device__ static S finish(S a) { return a; }
  __device__ static S neg(S a) { return -a; }
  __device__ static S add(S a, S b) { return __fadd_rn(a, b); }
  __device__ static S sub(S a, S b) { return __fsub_rn(a, b); }
  __device__ static S mul(S a, S b) { return __fmul_rn(a, b); }
  __device__ static S fma_(S a, S b, S c) { return __fmaf_rn(a, b, c); }
  __device__ static S fnma(S a, S b, S c) { return __fmaf_rn(-a, b, c); }
  __device__ static S coef(double c) { return __double2float_rn(c); }
  __device__ static void acc_prod(A& a, S u, S v) {
    dw p = two_prod(u, v);
    acc_add_term(a, p.hi, p.lo);
  }
  __device__ static S shfl_xor(S v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
  __device__ static S shfl(S v, int src) { return __shfl_sync(0xffffffffu, v, src); }
  __device__ static S combine(S a, S b) { return __fadd_rn(a, b); }
  __device__ static bool finite(S v) { return isfinite(v); }
};

struct PolB16 : PolF32 {
  using V = __nv_bfloat16;
  static constexpr int kId = 3;
  static constexpr int kMinBlocks = AJ_MINB_B16;
  __device__ static V ldv(const V* p) { return ld_ro(p); }
  __device__ static V vzero() { return __float2bfloat16_rn(0.f); }
  __device__ static void macv(S& acc, V v, S x) { acc = __fmaf_rn(__bfloat162float(v), x, acc); }
  __device__ static void mac(S& acc, const V* v, S x) { macv(acc, ldv(v), x); }
};

// ----------------------------------------------------------------------------
// Kernel arguments.  Vectors with several right-hand sides are interleaved:
// element (i, r) lives at i * nrhs + r.
//
// Lanes per row.  A system with nrhs right-hand sides gives each matrix row
// 2^lgr adjacent lanes of a warp (lgr = 0, 1, 2 for nrhs = 1, 2, 3-4); lane r
// of a row owns right-hand side r (with nrhs = 3 the fourth lane idles).  The
// lanes of a row read the same matrix entries (one broadcast access) and
// gather x[col * nrhs + r], adjacent words of one sector.  Every lane carries
// the state of one right-hand side only, so a thread needs the registers of a
// one-RHS sweep whatever nrhs is, and a tile holds 256 >> lgr rows.
//
// Matrix formats.  CSR: tile k is rows k*T .. k*T + T-1 (T = 256 >> lgr), one
// row per lane group.  SELL-C-sigma (C = 32): the rows without the long ones
// are sorted by length (longest first) within windows of sigma rows; position
// p of that order holds row perm[p], and slice p / 32 stores its 32 rows
// column-major, entry k of position p at sptr[p / 32] + 32 k + p % 32, so
// consecutive positions read consecutive words.  Entries keep their CSR
// order, so a row sums in the same order in both formats.  Tiles past the SELL
// ones hold the long rows (long_rows, longest first, at most T and a bounded
// number of entries per tile, dealt round-robin over the warps), each summed
// by a whole warp from the CSR arrays; the last tiles hold one huge row each,
// summed by the whole CTA.
template <class P>
struct IterArgs {
  int n;
  int nrhs;                   // right-hand sides, 1..4
  int lgr;                    // log2 of the lanes per row (0, 1 or 2)
  const int* row_ptr;
  const int* col;
  const typename P::V* val;
  int fmt;                    // 0 CSR, 1 SELL, 2 constant-coefficient stencil
  int sdim;                   // stencil: 2 (5-point, N x N) or 3 (7-point, N^3), natural row order
  int sN;                     // stencil: grid side N
  int sdiag_at, soff_at;      // stencil: entries of val holding the diagonal and the off-diagonal value
  unsigned long long smag;    // stencil: q / N = (q * smag) >> sshift for 0 <= q < 2^31
  int sshift;
  int short_rows;             // 1: no row has more than kLongRow entries
  int jblk;                   // rows per block of J (1: diagonal J; 2, 4, 8: eq. J-blkdiag,
                              // jinv then holds row k of each block's inverse at jinv[k * jblk])
  int nsell;                  // SELL: rows in the sliced part
  int sell_cl;                // SELL: log2 of the slice height C (5: 32 rows; 4, 3: 16, 8 rows,
                              // one right-hand side only, 32 / C lanes per row)
  int ntiles_sell;            // SELL: tiles of the sliced part
  int nltiles;                // SELL: tiles of long rows
  const int* perm;            // SELL: [nsell] row at each position
  const int* rlen;            // SELL: [nsell] entries of the row at each position
  const int* sptr;            // SELL: [nsell / 32 + 1] slice offsets (entries)
  const int* scol;            // SELL: sliced column indices
  const typename P::V* sval;  // SELL: sliced values
  const int* long_rows;       // SELL: rows summed by a whole warp
  const int* ltp;             // SELL: [nltiles + 1] long tile k = long_rows[ltp[k] .. ltp[k+1])
  int nhuge;                  // SELL: rows summed by a whole CTA, one per tile
  const int* huge_rows;       // SELL: [nhuge]
  const typename P::X* b;     // [n * nrhs]
  const typename P::X* jinv;  // [n]
  typename P::X* x[3];        // three iterate buffers, [n * nrhs] each
  typename P::X* u[2];        // stored form: Q x^t and Q x^{t-1}, [n * nrhs] each
  typename P::X* dl;          // difference form: x^t - x^{t-1}, [n * nrhs], own rows only
  double* partials;           // [2][gridDim][nrhs][kNRed]
  unsigned long long* bar;    // barrier arrival counter, zero at launch
  int* err;                   // device error word, zero at launch
  RhsState* state;            // [nrhs], in/out
  long long* rlog;            // [nrhs][rlog_cap] restart iterations
  int rlog_cap;
  double* trace;              // optional [trace_cap][nrhs][4]: d, ||g||^2, rr, beta per sweep
  long long trace_cap;
  long long maxit;
  int stop;
  int restart;
  int momentum;
  double tol;
  double fstar;
  double fscale;              // f(x) = fscale * (1/2 <x~, Q~ x~> - <b~, x~>) for scaled data
  long long max_sweeps;       // sweeps allowed in this launch (chunked runs), >= 1
  unsigned long long bar_timeout_ns;  // limit of each grid-barrier wait
  int bar_withhold_cta;       // failure-detection tests: this CTA withholds its first
                              // barrier arrival (-1: none)
};

// log2 of the lanes per row for nrhs right-hand sides.
__host__ __device__ constexpr int lanes_log2(int nrhs) { return nrhs <= 1 ? 0 : nrhs == 2 ? 1 : 2; }

// Iterate buffer k (0..2) and stored-product buffer k (0..1), chosen by
// selects so that no argument array is indexed at run time.
template <class P>
__device__ __forceinline__ typename P::X* xbuf(const IterArgs<P>& a, int k) {
  return k == 0 ? a.x[0] : k == 1 ? a.x[1] : a.x[2];
}
template <class P>
__device__ __forceinline__ typename P::X* ubuf(const IterArgs<P>& a, int k) {
  return k == 0 ? a.u[0] : a.u[1];
}

// Partial row sums over entries q0, q0 + step, ... < re (CSR arrays) for
// right-hand side r of an nr-RHS system, U entries loaded before their
// multiply-adds, which run in entry order.  lx sums against x^{s-1} (buffer
// xc); lp against x^{s-2} (buffer xp) when `two` (lazy form, the two differ).
template <class P, bool QX>
__device__ __forceinline__ void row_sums_strided(const IterArgs<P>& a, int nr, int r,
                                                 const typename P::X* xc, const typename P::X* xp,
                                                 bool two, int q0, int re, int step,
                                                 typename P::S& lx, typename P::S& lp) {
  using S = typename P::S;
  using V = typename P::V;
  constexpr int U = 4;
  for (int q = q0; q < re; q += U * step) {
    int cc[U];
    V vv[U];
#pragma unroll
    for (int k = 0; k < U; k++) {
      const bool in = q + k * step < re;
      cc[k] = in ? ld_ro(a.col + q + k * step) : 0;
      vv[k] = in ? P::ldv(a.val + q + k * step) : P::vzero();
    }
    S xv[U], pv[U];
#pragma unroll
    for (int k = 0; k < U; k++) {
      xv[k] = P::zero();
      pv[k] = P::zero();
      if (q + k * step < re) {
        xv[k] = P::ldg(xc + (size_t)cc[k] * nr + r);
        if (two) pv[k] = P::ldg(xp + (size_t)cc[k] * nr + r);
      }
    }
#pragma unroll
    for (int k = 0; k < U; k++) {
      if (q + k * step >= re) break;
      P::macv(lx, vv[k], xv[k]);
      if (two) P::macv(lp, vv[k], pv[k]);
    }
  }
}

// Warp-cooperative row sums of one long row for right-hand side r (lanes
// stride over the entries, then a fixed xor tree).  Returns the sums in every
// lane; sp equals sx when the stored form or x^{s-1} = x^{s-2} needs no
// second sum.  Every lane of the warp must call it.
template <class P, bool QX>
__device__ __forceinline__ void long_row_sums(const IterArgs<P>& a, const RhsState& q, int nr, int r,
                                              int rs, int re, typename P::S& sx, typename P::S& sp) {
  using S = typename P::S;
  const int lane = threadIdx.x & 31;
  const bool two = !QX && q.cur != q.prev;
  S lx = P::zero(), lp = P::zero();
  if (!q.done)
    row_sums_strided<P, QX>(a, nr, r, xbuf(a, q.cur), xbuf(a, q.prev), two, rs + lane, re, 32, lx, lp);
  lx = P::finish(lx);
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) lx = P::combine(lx, P::shfl_xor(lx, m));
  sx = lx;
  sp = lx;
  if (two) {
    lp = P::finish(lp);
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) lp = P::combine(lp, P::shfl_xor(lp, m));
    sp = lp;
  }
}

// CTA-cooperative row sums of one huge row for right-hand side r: threads
// stride over the entries, then a fixed xor tree per warp and the warps in
// order.  Results valid in every thread.  Every thread of the CTA must call it.
template <class P, bool QX>
__device__ __forceinline__ void cta_row_sums(const IterArgs<P>& a, const RhsState& q, int nr, int r,
                                             int rs, int re, typename P::S& sx, typename P::S& sp) {
  using S = typename P::S;
  __shared__ S red[2][kWarps];
  const bool two = !QX && q.cur != q.prev;
  S lx = P::zero(), lp = P::zero();
  if (!q.done)
    row_sums_strided<P, QX>(a, nr, r, xbuf(a, q.cur), xbuf(a, q.prev), two, rs + threadIdx.x, re,
                            kThreads, lx, lp);
  const int w = threadIdx.x >> 5;
  lx = P::finish(lx);
  lp = P::finish(lp);
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) {
    lx = P::combine(lx, P::shfl_xor(lx, m));
    if (two) lp = P::combine(lp, P::shfl_xor(lp, m));
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][w] = lx;
    red[1][w] = lp;
  }
  __syncthreads();
  S tx = red[0][0], tp = red[1][0];
  for (int k = 1; k < kWarps; k++) {
    tx = P::combine(tx, red[0][k]);
    if (two) tp = P::combine(tp, red[1][k]);
  }
  sx = tx;
  sp = two ? tp : tx;
  __syncthreads();
}

// The explicit-y form (SF 3) gathers from its own sources: y^s (the
// buffer x^{s-1} itself on the first sweep and after a restart, where
// y^s = x^{s-1}), and x^{s-1} again in a second pass on a check sweep, where
// the exact stop test needs Q x^{s-1}.  Sources for right-hand side state q:
template <class P>
__device__ __forceinline__ const typename P::X* y_source(const IterArgs<P>& a, const RhsState& q) {
  return q.cur == q.prev ? xbuf(a, q.cur) : ubuf(a, q.yb);
}
template <class P>
__device__ __forceinline__ bool y_check(const RhsState& q) {
  return q.chk && q.cur != q.prev;
}

// Fixed xor tree of a warp's partial sums; the total in every lane.
template <class P>
__device__ __forceinline__ typename P::S warp_total(typename P::S v) {
  v = P::finish(v);
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) v = P::combine(v, P::shfl_xor(v, m));
  return v;
}

// long_row_sums of the explicit-y form: sx over y^s; sp over x^{s-1} on a
// check sweep, in a second pass (else sp = sx).  Every lane must call it.
template <class P>
__device__ __forceinline__ void long_row_sums_y(const IterArgs<P>& a, const RhsState& q, int nr, int r,
                                                int rs, int re, typename P::S& sx, typename P::S& sp) {
  using S = typename P::S;
  const int lane = threadIdx.x & 31;
  S lx = P::zero(), unused = P::zero();
  if (!q.done)
    row_sums_strided<P, true>(a, nr, r, y_source(a, q), nullptr, false, rs + lane, re, 32, lx, unused);
  sx = warp_total<P>(lx);
  sp = sx;
  if (y_check<P>(q)) {
    S l2 = P::zero();
    if (!q.done)
      row_sums_strided<P, true>(a, nr, r, xbuf(a, q.cur), nullptr, false, rs + lane, re, 32, l2, unused);
    sp = warp_total<P>(l2);
  }
}

// cta_row_sums of the explicit-y form (same sources as long_row_sums_y).
// Every thread of the CTA must call it.
template <class P>
__device__ __forceinline__ typename P::S cta_total(typename P::S v, typename P::S* red) {
  using S = typename P::S;
  v = warp_total<P>(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  S t = red[0];
  for (int k = 1; k < kWarps; k++) t = P::combine(t, red[k]);
  __syncthreads();
  return t;
}
template <class P>
__device__ __forceinline__ void cta_row_sums_y(const IterArgs<P>& a, const RhsState& q, int nr, int r,
                                               int rs, int re, typename P::S& sx, typename P::S& sp) {
  using S = typename P::S;
  __shared__ S red[kWarps];
  S lx = P::zero(), unused = P::zero();
  if (!q.done)
    row_sums_strided<P, true>(a, nr, r, y_source(a, q), nullptr, false, rs + threadIdx.x, re, kThreads,
                              lx, unused);
  sx = cta_total<P>(lx, red);
  sp = sx;
  if (y_check<P>(q)) {
    S l2 = P::zero();
    if (!q.done)
      row_sums_strided<P, true>(a, nr, r, xbuf(a, q.cur), nullptr, false, rs + threadIdx.x, re, kThreads,
                                l2, unused);
    sp = cta_total<P>(l2, red);
  }
}

// Loop-invariant values of the explicit-y form's row update (nothing for the
// other forms, whose registers they would otherwise take).
template <class P, bool YS>
struct YConst {
  __device__ explicit YConst(const RhsState&) {}
};
template <class P>
struct YConst<P, true> {
  typename P::S bnext;  // beta of the candidate y^{s+1}
  __device__ explicit YConst(const RhsState& q) : bnext(P::coef(q.beta_next)) {}
};

// One row's sum against src over entries colp[k * stride], valp[k * stride],
// k < cnt, added to acc in chunks of U loads issued before their
// multiply-adds (entry order), for the second pass of an explicit-y check
// sweep.
template <class P, int U>
__device__ __forceinline__ typename P::S row_pass(const int* colp, const typename P::V* valp, int cnt,
                                                  int stride, const typename P::X* src, int nr, int r,
                                                  typename P::S acc) {
  using S = typename P::S;
  using V = typename P::V;
  for (int q0 = 0; q0 < cnt; q0 += U) {
    int cc[U];
    V vv[U];
#pragma unroll
    for (int k = 0; k < U; k++) {
      const bool in = q0 + k < cnt;
      cc[k] = in ? ld_ro(colp + (q0 + k) * stride) : 0;
      vv[k] = in ? P::ldv(valp + (q0 + k) * stride) : P::vzero();
    }
    S xv[U];
#pragma unroll
    for (int k = 0; k < U; k++) xv[k] = q0 + k < cnt ? P::ldg(src + (size_t)cc[k] * nr + r) : P::zero();
#pragma unroll
    for (int k = 0; k < U; k++) {
      if (q0 + k >= cnt) break;
      P::macv(acc, vv[k], xv[k]);
    }
  }
  return P::finish(acc);
}

// The same for stencil row i (a 5- or 7-point constant-coefficient
// Dirichlet Laplacian in natural order; bit k of inm: neighbour k of
// -N^2, -N, -1, 0, +1, +N, +N^2 lies in the grid).
template <class P, int U>
__device__ __forceinline__ typename P::S stencil_pass(int i, unsigned inm, int N, int NN, typename P::V s_diag,
                                                      typename P::V s_off, const typename P::X* src, int nr,
                                                      int r, typename P::S acc) {
  using S = typename P::S;
#pragma unroll
  for (int k0 = 0; k0 < 7; k0 += U) {
    S xv[U];
#pragma unroll
    for (int j = 0; j < U; j++) {
      const int k = k0 + j;
      const int off = k == 0 ? -NN : k == 1 ? -N : k == 2 ? -1 : k == 3 ? 0 : k == 4 ? 1 : k == 5 ? N : NN;
      xv[j] = (k < 7 && (inm >> k & 1u)) ? P::ldg(src + (size_t)(i + off) * nr + r) : P::zero();
    }
#pragma unroll
    for (int j = 0; j < U; j++) {
      const int k = k0 + j;
      if (k >= 7 || !(inm >> k & 1u)) continue;
      P::macv(acc, k == 3 ? s_diag : s_off, xv[j]);
    }
  }
  return P::finish(acc);
}

// Reduction slots a sweep fills: d and rr always, ||Q y - b||^2 in the
// explicit-y form (want_gg), the objective terms only for the objective-gap
// stop.
__device__ __forceinline__ bool slot_used(int k, bool want_obj, bool want_gg) {
  return k == 0 || k == 2 || (want_gg && k == 1) || (want_obj && k >= 3);
}

// Block reduction of per-thread FP64 values in a fixed order; result valid in
// thread 0.  `sm` holds kWarps doubles.
__device__ __forceinline__ double block_sum(double v, double* sm) {
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) sm[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < kWarps; i++) s += sm[i];
  __syncthreads();
  return s;
}

// Per right-hand side r < nr, the CTA's sum of v over the lanes that own r:
// a xor tree over the lanes of equal r within each warp, then the warps in
// order.  Result valid in thread r.  `sm` holds kWarps * kMaxRhs doubles.
// With one lane per row (lg = 0) this is block_sum.
__device__ __forceinline__ double block_sum_rhs(double v, double* sm, int lg, int nr) {
  for (int m = 16; m >= (1 << lg); m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane < (1 << lg)) sm[w * kMaxRhs + lane] = v;
  __syncthreads();
  double s = 0.0;
  if ((int)threadIdx.x < nr)
    for (int i = 0; i < kWarps; i++) s += sm[i * kMaxRhs + threadIdx.x];
  __syncthreads();
  return s;
}

// Entries per unrolled chunk of a short row: as many gathers in flight as the
// register budget allows for the sweep form.
#ifndef AJ_ROW_UNROLL
#define AJ_ROW_UNROLL 8
#endif
__host__ __device__ constexpr int row_unroll(bool qx) {
  return (qx ? 1 : 2) * 8 / AJ_ROW_UNROLL >= 2 ? 4 : 8;
}

// The FP64 explicit-y sweep on CSR rows (one RHS) runs 5 CTAs per SM with
// chunks of 4 entries: at 48 registers its gathers stay in flight and the FP64
// pipe busy (256^3 Poisson: 0.480 against 0.522 ms per sweep at 4 CTAs and
// chunks of 8).  Its stencil-only twin keeps 4 CTAs and chunks of 8 (0.427
// against 0.468 ms).  Every other kernel: the policy's CTAs per SM.
#ifndef AJ_Y_CSR_MINB
#define AJ_Y_CSR_MINB 5
#endif
template <class P, int SF, int FM, bool MULTI>
__host__ __device__ constexpr bool y_csr_f64() {
  return std::is_same<P, PolF64>::value && SF == 3 && FM == 0 && !MULTI;
}
// CTAs per SM of the one-RHS SELL-only kernels of the FP32 and BF16 policies
// (0: the policy's own); see AJ_SELL_PIPE
#ifndef AJ_SELL_MINB
#define AJ_SELL_MINB 4
#endif
// AJ_Y_CSR_TWO: the FP64 explicit-y CSR sweep keeps two rows per thread in
// flight (tiles t and t + ncta), at AJ_Y_CSR_TWO_MINB CTAs/SM with chunks of
// AJ_Y_CSR_TWO_U entries (256^3 Poisson: 0.464 ms per sweep at 4 CTAs/SM and
// chunks of 4, against 0.486 ms with one row per thread at 5 CTAs/SM)
#ifndef AJ_Y_CSR_TWO
#define AJ_Y_CSR_TWO 1
#endif
#ifndef AJ_Y_CSR_TWO_MINB
#define AJ_Y_CSR_TWO_MINB 4
#endif
#ifndef AJ_Y_CSR_TWO_U
#define AJ_Y_CSR_TWO_U 4
#endif
// AJ_Y_CSR_TWO_EARLY: 0 loads J^-1_i and x^{t-1}_i after the row sums; 1 loads
// them before the chunk loop; 2 prefetches their lines into L2 before it.
// Measured per 256^3 sweep: 0.457 ms, 0.515 ms (spills), 0.464 ms.
#ifndef AJ_Y_CSR_TWO_EARLY
#define AJ_Y_CSR_TWO_EARLY 0
#endif
template <class P, int SF, int FM, bool MULTI>
__host__ __device__ constexpr int kernel_min_blocks() {
  return y_csr_f64<P, SF, FM, MULTI>() ? (AJ_Y_CSR_TWO ? AJ_Y_CSR_TWO_MINB : AJ_Y_CSR_MINB)
         : (FM >= 3 && !MULTI && P::kId >= 2 && AJ_SELL_MINB > 0) ? AJ_SELL_MINB
         : MULTI ? P::kMinBlocksMulti : P::kMinBlocks;
}
// The SELL-only kernels (FM 3, 4).  FP32 and BF16 values: chunks of
// AJ_SELL_UNROLL entries, and (AJ_SELL_PIPE) chunk q + 1's columns and values
// loaded while chunk q's gathers are in flight, at AJ_SELL_MINB CTAs per SM.
// FP64 and double-float values: chunks of AJ_SELL_UNROLL_F64, no pipeline.
// Chung-Lu graph, n = 8.4M, per sweep: FP32 0.80 -> 0.71 ms (pipelined
// chunks of 8 at 4 CTAs/SM; at the 40-register cap of 6 CTAs/SM the pipeline
// spilled, 1.03 ms), FP64 1.13 -> 1.10 ms (chunks of 4).
#ifndef AJ_SELL_UNROLL
#define AJ_SELL_UNROLL 8
#endif
#ifndef AJ_SELL_UNROLL_F64
#define AJ_SELL_UNROLL_F64 4
#endif
#ifndef AJ_SELL_PIPE
#define AJ_SELL_PIPE 1
#endif
template <class P>
__host__ __device__ constexpr bool sell_pipe() {
  return P::kId >= 2 && AJ_SELL_PIPE;
}
template <class P, int SF, int FM, bool MULTI>
__host__ __device__ constexpr int kernel_row_unroll() {
  return y_csr_f64<P, SF, FM, MULTI>() ? 4
         : FM >= 3 ? (P::kId >= 2 ? AJ_SELL_UNROLL : AJ_SELL_UNROLL_F64)
                   : row_unroll(SF != 0);
}

// One sweep over the CTA's tiles: the fused SpMV at y, x update and reduction
// terms.  `compute_x` is false on a residual-only sweep (no x^s is formed).
// Reduction slots (per lane, for the lane's right-hand side): 0 d, 1
// ||Q y - b||^2 (explicit-y form), 2 rr, 3 <x, Qx> and 4 <b, x> (objective
// stop only).
// FM: the formats the instantiation reads -- 0 CSR only, which keeps the
// other formats' code and registers out of the CSR kernel; 1 any (runtime
// a.fmt: CSR, SELL or stencil; needed by the block-diagonal J on CSR and by
// the batched kernel); 2 the stencil rows alone; 3 SELL alone with slices
// of 32 rows (the graph sweeps, without the CSR, stencil and block-J code);
// 4 SELL alone with slices of 8 or 16 rows (split rows).  MULTI:
// nrhs and the lanes per row come from the arguments; otherwise one.
// SF: sweep form -- 0 lazy, 1 stored, 2 stored with the difference
// delta = x^{s-1} - x^{s-2} kept in a.dl (y = x + beta delta costs one
// instruction instead of two; delta is the same rounded difference the
// update computes anyway for the restart test), 3 explicit y: the sweep
// gathers y^s itself, written by the previous sweep as the candidate
// y^s = x^{s-1} + beta_s (x^{s-1} - x^{s-2}) (beta_s needs only alpha_{s-1},
// known before the restart test), and writes the candidate y^{s+1} in u; a
// restart drops the candidate, and y^{s+1} = x^{s-1} is read from that
// iterate's buffer.  One row sum and no Q x vectors, but no exact residual
// on the way: the stop test's Q x^{s-1} is summed in a second pass on check
// sweeps only (RhsState::chk), which ||Q y^s - b||^2 (slot 1) schedules.
// (The explicit-y code sits in `if constexpr` blocks of its own: at the
// register caps of the FP32 and BF16 policies even values the other forms
// never use changed their register allocation, and their speed.)
// ----------------------------------------------------------------------------
// The stencil sweep of the explicit-y form with one right-hand side, its
// gathers staged in shared memory.  A tile of 256 rows i0 .. i0 + 255 gathers
// y only from five contiguous segments -- rows i0 + off .. i0 + 255 + off for
// off = -N^2, -N, +N, +N^2, and i0 - 1 .. i0 + 256 for the row itself and its
// +-1 neighbours -- and reads its own rows of x^{s-1}, b and J^{-1}.  Those
// eight pieces are copied to shared memory by cp.async, STAGES - 1 tiles
// ahead of the tile being summed, so the sweep waits on memory once per
// launch instead of once per tile.  Every row sums the same neighbours in the
// same order with the same operations as the unstaged stencil rows (and so
// as CSR rows), and the reduction terms accumulate in the same tile order:
// the iterates are the unstaged sweep's bit for bit.
// AJ_STENCIL_STAGE: the policies that stage, bit P::kId (1 FP64, 2
// double-float, 4 FP32, 8 BF16); AJ_STAGE_ST64 / AJ_STAGE_ST32: the stages
// of the 8-byte and 4-byte vector policies.  Measured per 256^3 sweep,
// staged against unstaged: FP64 0.418 / 0.426 ms, BF16 values 0.179 / 0.194
// (4 stages; 2 and 3: 0.190, 0.188), FP32 values 0.204 / 0.181 and
// double-float 0.333 / 0.275 -- so FP64 and BF16 stage, the other two do not.
// The staged sweep issues fewer loads but more index arithmetic and a CTA
// barrier per tile, which the FP32 and double-float sweeps, already issue
// bound, pay for.
#ifndef AJ_STENCIL_STAGE
#define AJ_STENCIL_STAGE 9
#endif
#ifndef AJ_STAGE_ST64
#define AJ_STAGE_ST64 2
#endif
#ifndef AJ_STAGE_ST32
#define AJ_STAGE_ST32 4
#endif
// The row tiles (CSR and stencil) a CTA sweeps, cta of ncta: round-robin
// (tiles cta, cta + ncta, ...) or, with AJ_TILE_CONTIG, one contiguous block
// (a 3-D grid's +-N neighbours of a 256-row tile are then the CTA's previous
// and next tiles).  first, step and end of the CTA's tile sequence.  Measured
// on the 256^3 Poisson system, contiguous against round-robin: FP64
// explicit y 0.514 / 0.486 ms per sweep, FP32 lazy 0.356 / 0.317, FP32
// stencil 0.195 / 0.181 -- round-robin keeps the whole grid's gather window
// (and its +-N^2 planes) in L2, which outweighs the L1 hits.
#ifndef AJ_TILE_CONTIG
#define AJ_TILE_CONTIG 0
#endif
struct TileRange {
  int first, step, end;
  __device__ TileRange(int ntiles, int cta, int ncta, bool contig) {
    if (contig) {
      const int per = ntiles / ncta, rem = ntiles - per * ncta;
      first = cta * per + (cta < rem ? cta : rem);
      end = first + per + (cta < rem ? 1 : 0);
      step = 1;
    } else {
      first = cta;
      end = ntiles;
      step = ncta;
    }
  }
};

template <class P>
struct StencilStage {
  using X = typename P::X;
  static constexpr int kE = 16 / (int)sizeof(X);        // elements per 16-byte copy
  static constexpr int kL = kThreads + 2 * kE;           // elements of a y segment
  static constexpr int kStages = P::kId >= 2 ? AJ_STAGE_ST32 : AJ_STAGE_ST64;  // tiles in flight + 1
  static constexpr int kCH = kL / kE;                    // copies per y segment
  static constexpr int kCO = kThreads / kE;              // copies per own-row piece
  static constexpr int kCopies = 5 * kCH + 3 * kCO;      // copies per tile
  static constexpr int kPer = (kCopies + kThreads - 1) / kThreads;  // per thread
  __align__(16) X seg[kStages][5][kL];                   // y^s around the tile
  __align__(16) X own[kStages][3][kThreads];             // x^{s-1}, b, J^{-1} of its rows
};

// The stage buffers: one block of shared memory per kernel, whichever
// monitor variant of the sweep uses it.
template <class P>
__device__ __forceinline__ StencilStage<P>& stencil_stage_smem() {
  __shared__ StencilStage<P> sg;
  return sg;
}

// First element of y segment j (0..4: -N^2, -N, the row and its +-1, +N,
// +N^2) of the tile at row i0, rounded down to a whole 16-byte copy (a
// multiple of E elements; for a negative start too, by the two's-complement
// mask).
template <class P>
__device__ __forceinline__ int stage_seg_start(int i0, int j, int N, int NN) {
  constexpr int E = StencilStage<P>::kE;
  const int base = i0 + (j == 0 ? -NN : j == 1 ? -N : j == 2 ? -1 : j == 3 ? N : NN);
  return base & ~(E - 1);
}

template <class P, bool MON>
__device__ __forceinline__ void sweep_stencil_y_staged(const IterArgs<P>& a, const RhsState& me,
                                                       bool compute_x, typename P::A (&acc)[kNRed],
                                                       int cta, int ncta) {
  using S = typename P::S;
  using V = typename P::V;
  using X = typename P::X;
  using SG = StencilStage<P>;
  constexpr int ST = SG::kStages;
  constexpr int E = SG::kE;
  constexpr int U = kernel_row_unroll<P, 3, 2, false>();
  SG& sg = stencil_stage_smem<P>();
  const X* yc = y_source(a, me);
  const X* xp = xbuf(a, me.cur);
  X* xn = xbuf(a, me.nxt);
  X* yn = ubuf(a, 1 - me.yb);
  const bool same = me.cur == me.prev;
  const bool active = me.done == 0;
  const bool check = y_check<P>(me);
  const YConst<P, true> yk(me);
  const V s_diag = P::ldv(a.val + a.sdiag_at);
  const V s_off = P::ldv(a.val + a.soff_at);
  const int n = a.n;
  const int N = a.sN, NN = a.sdim == 3 ? N * N : 0;
  const int ntiles = (n + kThreads - 1) / kThreads;
  const TileRange tr(ntiles, cta, ncta, AJ_TILE_CONTIG);
  // the copies of tile t into stage slot k, the parts inside the vectors:
  // copy c = threadIdx.x + p * 256 is chunk q of piece j (y segments 0..4,
  // then x^{s-1}, b, J^{-1})
  auto issue = [&](int t, int k) {
    const int i0 = t * kThreads;
#pragma unroll
    for (int p = 0; p < SG::kPer; p++) {
      const int c = (int)threadIdx.x + p * kThreads;
      if (c >= SG::kCopies) continue;
      const X* src;
      X* dst;
      int g;
      if (c < 5 * SG::kCH) {
        const int j = c / SG::kCH, q = c - j * SG::kCH;
        if ((j == 0 || j == 4) && NN == 0) continue;  // 2-D grid: no +-N^2 neighbours
        g = stage_seg_start<P>(i0, j, N, NN) + q * E;
        src = yc;
        dst = &sg.seg[k][j][q * E];
      } else {
        const int j = (c - 5 * SG::kCH) / SG::kCO, q = c - 5 * SG::kCH - j * SG::kCO;
        if (j == 0 && same) continue;  // x^{s-1} = y^s: not read
        g = i0 + q * E;
        src = j == 0 ? xp : j == 1 ? a.b : a.jinv;
        dst = &sg.own[k][j][q * E];
      }
      if (g < 0 || g >= n) continue;
      const int left = n - g;
      cp_async16(dst, src + g, (left < E ? left : E) * (int)sizeof(X));
    }
  };
  __syncthreads();  // the previous sweep's reads of the stage slots are done
#pragma unroll
  for (int p = 0; p < ST - 1; p++) {
    const int t = tr.first + p * tr.step;
    if (t < tr.end) issue(t, p);
    cp_async_commit();
  }
  int k = 0;
  for (int tile = tr.first; tile < tr.end; tile += tr.step, k = k + 1 == ST ? 0 : k + 1) {
    // tile's copies have landed (the newest ST - 2 groups may still fly), and
    // every thread is done with the previous tile's slot, refilled next
    cp_async_wait<ST - 2>();
    __syncthreads();
    {
      const int t = tile + (ST - 1) * tr.step;
      if (t < tr.end) issue(t, k == 0 ? ST - 1 : k - 1);
      cp_async_commit();
    }
    const int i0 = tile * kThreads;
    const int i = i0 + (int)threadIdx.x;
    if (i < n && active) {
      const int q = (int)(((unsigned long long)i * a.smag) >> a.sshift);  // i / N
      const int ix = i - q * N;
      const int iy = a.sdim == 3 ? q - (int)(((unsigned long long)q * a.smag) >> a.sshift) * N : q;
      const unsigned inm = (ix > 0 ? 4u : 0u) | 8u | (ix < N - 1 ? 16u : 0u) | (iy > 0 ? 2u : 0u) |
                           (iy < N - 1 ? 32u : 0u) | (i >= NN && NN ? 1u : 0u) |
                           (NN && i < n - NN ? 64u : 0u);
      const S bi = P::from_x(sg.own[k][1][threadIdx.x]);
      S sx = P::neg(bi);
      // neighbour kn at offset off lies in segment j at (i + off) - start_j;
      // the row's own segment (j = 2) holds -1, 0, +1
      const int r2 = i - stage_seg_start<P>(i0, 2, N, NN);  // the row itself in segment 2
#pragma unroll
      for (int kn = 0; kn < 7; kn++) {
        if (!(inm >> kn & 1u)) continue;
        X v;
        if (kn == 0) v = sg.seg[k][0][i - NN - stage_seg_start<P>(i0, 0, N, NN)];
        else if (kn == 1) v = sg.seg[k][1][i - N - stage_seg_start<P>(i0, 1, N, NN)];
        else if (kn <= 4) v = sg.seg[k][2][r2 + kn - 3];
        else if (kn == 5) v = sg.seg[k][3][i + N - stage_seg_start<P>(i0, 3, N, NN)];
        else v = sg.seg[k][4][i + NN - stage_seg_start<P>(i0, 4, N, NN)];
        P::macv(sx, kn == 3 ? s_diag : s_off, P::from_x(v));
      }
      sx = P::finish(sx);
      const S yi = P::from_x(sg.seg[k][2][r2]);
      const S g = sx;  // Q y^s - b
      if (MON) P::acc_prod(acc[1], g, g);
      if (check) {
        const S sp = stencil_pass<P, U>(i, inm, N, NN, s_diag, s_off, xp, 1, 0, P::neg(bi));
        P::acc_prod(acc[2], sp, sp);
      }
      if (compute_x) {
        const S ji = P::from_x(sg.own[k][2][threadIdx.x]);
        const S xi = same ? yi : P::from_x(sg.own[k][0][threadIdx.x]);
        const S xnew = P::fnma(ji, g, yi);
        const S dx = P::sub(xnew, xi);
        P::stx(xn + i, xnew);
        P::stx(yn + i, P::fma_(yk.bnext, dx, xnew));
        P::acc_prod(acc[0], g, dx);
      }
    }
  }
  cp_async_wait<0>();
}

// Whether the staged stencil sweep can run: a diagonal J, and 16-byte aligned
// vectors for the copies (the iterate buffers, b and J^{-1} are separate
// allocations).
template <class P>
__device__ __forceinline__ bool stencil_stage_ok(const IterArgs<P>& a, const RhsState& me) {
  const unsigned long long m = (unsigned long long)y_source(a, me) | (unsigned long long)xbuf(a, me.cur) |
                               (unsigned long long)a.b | (unsigned long long)a.jinv;
  return ((AJ_STENCIL_STAGE >> P::kId) & 1) && a.jblk == 1 && (m & 15ull) == 0;
}

// The FP64 explicit-y CSR sweep with two rows per thread in flight: the
// thread's row of tile t and of tile t + ncta (the next tile it would sweep)
// load their chunks together, then each row sums and updates exactly as in
// the one-row sweep, the first row first, so the iterates and the reduction
// terms are the one-row sweep's bit for bit.  Only for matrices without
// long rows (a.short_rows) and on sweeps without the check pass.
template <class P, bool MON>
__device__ __forceinline__ void sweep_csr_y_two(const IterArgs<P>& a, const RhsState& me, bool compute_x,
                                                typename P::A (&acc)[kNRed], int cta, int ncta) {
  using S = typename P::S;
  using V = typename P::V;
  using X = typename P::X;
  constexpr int U = AJ_Y_CSR_TWO_U;
  const X* yc = y_source(a, me);
  const X* xp = xbuf(a, me.cur);
  X* xn = xbuf(a, me.nxt);
  X* yn = ubuf(a, 1 - me.yb);
  const bool same = me.cur == me.prev;
  const bool active = me.done == 0;
  const YConst<P, true> yk(me);
  const int n = a.n;
  const int ntiles = (n + kThreads - 1) / kThreads;
  for (int t1 = cta; t1 < ntiles; t1 += 2 * ncta) {
    const int t2 = t1 + ncta;
    const int i1 = t1 * kThreads + (int)threadIdx.x;
    const int i2 = t2 * kThreads + (int)threadIdx.x;
    const bool v1 = i1 < n && active;
    const bool v2 = t2 < ntiles && i2 < n && active;
    int rs1 = 0, c1 = 0, rs2 = 0, c2 = 0;
    if (v1) {
      rs1 = ld_ro(a.row_ptr + i1);
      c1 = ld_ro(a.row_ptr + i1 + 1) - rs1;
    }
    if (v2) {
      rs2 = ld_ro(a.row_ptr + i2);
      c2 = ld_ro(a.row_ptr + i2 + 1) - rs2;
    }
    S s1 = v1 ? P::neg(P::ldr(a.b + i1)) : P::zero();
    S s2 = v2 ? P::neg(P::ldr(a.b + i2)) : P::zero();
    S e_j1 = P::zero(), e_j2 = P::zero(), e_x1 = P::zero(), e_x2 = P::zero();
    if constexpr (AJ_Y_CSR_TWO_EARLY == 1) {
      if (v1 && compute_x) {
        e_j1 = P::ldr(a.jinv + i1);
        if (!same) e_x1 = P::ldx(xp + i1);
      }
      if (v2 && compute_x) {
        e_j2 = P::ldr(a.jinv + i2);
        if (!same) e_x2 = P::ldx(xp + i2);
      }
    } else if constexpr (AJ_Y_CSR_TWO_EARLY == 2) {
      if (v1 && compute_x) {
        asm volatile("prefetch.global.L2 [%0];" ::"l"(a.jinv + i1));
        if (!same) asm volatile("prefetch.global.L2 [%0];" ::"l"(xp + i1));
      }
      if (v2 && compute_x) {
        asm volatile("prefetch.global.L2 [%0];" ::"l"(a.jinv + i2));
        if (!same) asm volatile("prefetch.global.L2 [%0];" ::"l"(xp + i2));
      }
    }
    const int cm = c1 > c2 ? c1 : c2;
    for (int q0 = 0; q0 < cm; q0 += U) {
      int ca[U], cb[U];
      V va[U], vb[U];
#pragma unroll
      for (int k = 0; k < U; k++) {
        const bool ia = q0 + k < c1, ib = q0 + k < c2;
        ca[k] = ia ? ld_ro(a.col + rs1 + q0 + k) : 0;
        va[k] = ia ? P::ldv(a.val + rs1 + q0 + k) : P::vzero();
        cb[k] = ib ? ld_ro(a.col + rs2 + q0 + k) : 0;
        vb[k] = ib ? P::ldv(a.val + rs2 + q0 + k) : P::vzero();
      }
      S ya[U], yb[U];
#pragma unroll
      for (int k = 0; k < U; k++) {
        ya[k] = q0 + k < c1 ? P::ldg(yc + ca[k]) : P::zero();
        yb[k] = q0 + k < c2 ? P::ldg(yc + cb[k]) : P::zero();
      }
#pragma unroll
      for (int k = 0; k < U; k++)
        if (q0 + k < c1) P::macv(s1, va[k], ya[k]);
#pragma unroll
      for (int k = 0; k < U; k++)
        if (q0 + k < c2) P::macv(s2, vb[k], yb[k]);
    }
#pragma unroll
    for (int w = 0; w < 2; w++) {
      const bool v = w == 0 ? v1 : v2;
      if (!v) continue;
      const int i = w == 0 ? i1 : i2;
      const S g = P::finish(w == 0 ? s1 : s2);  // Q y^s - b
      const S yi = P::ldg(yc + i);
      if (MON) P::acc_prod(acc[1], g, g);
      if (!compute_x) continue;
      S ji, xi;
      if constexpr (AJ_Y_CSR_TWO_EARLY == 1) {
        ji = w == 0 ? e_j1 : e_j2;
        xi = same ? yi : (w == 0 ? e_x1 : e_x2);
      } else {
        ji = P::ldr(a.jinv + i);
        xi = same ? yi : P::ldx(xp + i);
      }
      const S xnew = P::fnma(ji, g, yi);
      const S dx = P::sub(xnew, xi);
      P::stx(xn + i, xnew);
      P::stx(yn + i, P::fma_(yk.bnext, dx, xnew));
      P::acc_prod(acc[0], g, dx);
    }
  }
}

template <class P, int SF, int FM, bool MULTI, bool MON = true>
__device__ __forceinline__ void sweep(const IterArgs<P>& a, const RhsState* st, bool compute_x,
                                      bool want_obj, typename P::A (&acc)[kNRed], int cta,
                                      int ncta) {
  if constexpr (y_csr_f64<P, SF, FM, MULTI>() && AJ_Y_CSR_TWO) {
    if (a.short_rows && !y_check<P>(st[0])) {
      sweep_csr_y_two<P, MON>(a, st[0], compute_x, acc, cta, ncta);
      return;
    }
  }
  if constexpr (FM == 2 && !MULTI && SF == 3) {
    if (stencil_stage_ok<P>(a, st[0])) {
      sweep_stencil_y_staged<P, MON>(a, st[0], compute_x, acc, cta, ncta);
      return;
    }
  }
  using S = typename P::S;
  using V = typename P::V;
  using X = typename P::X;
  constexpr bool YS = SF == 3;             // explicit y
  constexpr bool QX = SF == 1 || SF == 2;  // Q x^{s-1} stored for the next sweep
  constexpr bool ONE = SF != 0;            // one gathered vector in the main pass
  constexpr bool DL = SF == 2;
  const int nr = MULTI ? a.nrhs : 1;
  const int lg = MULTI ? a.lgr : 0;
  const int r = threadIdx.x & ((1 << lg) - 1);   // this lane's right-hand side
  const int slot = threadIdx.x >> lg;            // this lane group's row slot in a tile
  const int rpt = kThreads >> lg;                // rows per tile
  const bool lane_on = r < nr;
  const RhsState& me = st[lane_on ? r : 0];
  const X* xc = YS ? y_source(a, me) : xbuf(a, me.cur);  // gathered by the main pass
  const X* xp = YS ? xbuf(a, me.cur) : xbuf(a, me.prev);
  X* xn = xbuf(a, me.nxt);
  X* uc = QX ? ubuf(a, me.uw) : nullptr;
  const X* up = QX ? ubuf(a, 1 - me.uw) : nullptr;
  const bool same = me.cur == me.prev;
  const bool active = lane_on && me.done == 0;
  const S beta = P::coef(me.beta);
  const YConst<P, YS> yk(me);
  const int lane = threadIdx.x & 31;
  constexpr bool ANY = FM != 0;
  const bool sell = FM >= 3 || (FM == 1 && a.fmt == 1);
  // stencil: the rows of a constant-coefficient Dirichlet Laplacian in natural
  // order, their entries known without loading them (same values, same
  // ascending column order as in CSR, so the sums are the CSR sums bit for bit)
  const bool stn = FM == 2 || (FM == 1 && a.fmt == 2);
  // (declared without an initial value: even an unused zero conversion of
  // the BF16 policy changed register allocation in the CSR-only kernel)
  V s_diag, s_off;
  if constexpr (FM != 0) {
    if (stn) {
      s_diag = P::ldv(a.val + a.sdiag_at);
      s_off = P::ldv(a.val + a.soff_at);
    }
  }
  const int ntiles = sell ? a.ntiles_sell + a.nltiles + a.nhuge : (a.n + rpt - 1) / rpt;
  // SELL: the rows of a sorting window run longest first, so slice w of a
  // tile is longer than slice w + 1; warp w takes slice (w + kt) mod 8 of the
  // CTA's kt-th tile, so that no warp takes the longest slice of every tile
  // and waits on the others at the grid barrier the least
  int kt = 0;
  const TileRange tr(ntiles, cta, ncta, AJ_TILE_CONTIG && !sell);
  for (int tile = tr.first; tile < tr.end; tile += tr.step, kt++) {
    // this lane group's row i, its entries colp[k * stride], valp[k * stride]
    // (k < cnt) and, for long rows, its CSR range rs .. re
    int i, rs = 0, re = 0, cnt = 0, stride = 1;
    bool valid, is_long, huge = false;
    int sub = 0;         // SELL with C < 32: this lane's share of its row's entries
    bool split = false;  //   (warp-uniform: the whole CTA sweeps the same tile)
    const int* colp = a.col;
    const V* valp = a.val;
    if (!sell) {
      i = tile * rpt + slot;
      valid = i < a.n;
      if (valid && !stn) {
        rs = ld_ro(a.row_ptr + i);
        re = ld_ro(a.row_ptr + i + 1);
      }
      is_long = valid && (re - rs) > kLongRow;
      cnt = re - rs;
      colp += rs;
      valp += rs;
    } else {
      // SELL: the sliced tiles in row order (neighbouring tiles gather from
      // nearby rows), then the tiles of long rows (longest first), then the
      // huge rows (one per tile, longest first); AJ_SELL_HEAVY_FIRST puts the
      // last two kinds first
#if AJ_SELL_HEAVY_FIRST
      const int kind = tile < a.nhuge ? 2 : tile < a.nhuge + a.nltiles ? 1 : 0;
      const int ix = kind == 2 ? tile : kind == 1 ? tile - a.nhuge : tile - a.nhuge - a.nltiles;
#else
      const int kind = tile < a.ntiles_sell ? 0 : tile < a.ntiles_sell + a.nltiles ? 1 : 2;
      const int ix = kind == 0 ? tile : kind == 1 ? tile - a.ntiles_sell : tile - a.ntiles_sell - a.nltiles;
#endif
      if (kind == 0) {
        // slices of C = 2^cl rows, entry k of a slice's row p at
        // sptr[slice] + C k + p.  With C < 32 (one right-hand side) the
        // L = 32 / C lanes of a row take its entries k = sub, sub + L, ... and
        // a warp reads 32 consecutive stored words per load; a tile is then
        // 8 C rows, one slice per warp
        // (the SELL-32-only kernel, FM 3, never meets split slices)
        const int cl = (FM == 4 || FM == 1) ? a.sell_cl : 5;
        const int wv = ((threadIdx.x >> 5) + AJ_SELL_ROTATE * kt) & (kWarps - 1);  // the slice this warp takes
        int pos;
        if ((FM == 4 || FM == 1) && cl < 5) {
          split = true;
          sub = lane >> cl;
          pos = ix * (kWarps << cl) + (wv << cl) + (lane & ((1 << cl) - 1));
        } else {
          pos = ix * rpt + (wv << (5 - lg)) + (lane >> lg);
        }
        valid = pos < a.nsell;
        i = valid ? ld_ro(a.perm + pos) : 0;
        if (valid) {
          const int len = ld_ro(a.rlen + pos);
          const int lsh = 5 - cl;  // log2 L
          cnt = split ? (len > sub ? (len - sub + (1 << lsh) - 1) >> lsh : 0) : len;
          const int base = ld_ro(a.sptr + (pos >> cl)) + (pos & ((1 << cl) - 1)) + (sub << cl);
          colp = a.scol + base;
          valp = a.sval + base;
          stride = 32;
        }
        is_long = false;
      } else if (kind == 1) {
        // long rows dealt round-robin over the warps: row j of the tile goes to
        // warp j % 8, row slot j / 8 of that warp
        const int pos = ld_ro(a.ltp + ix) + (lane >> lg) * kWarps + (threadIdx.x >> 5);
        valid = pos < ld_ro(a.ltp + ix + 1);
        i = valid ? ld_ro(a.long_rows + pos) : 0;
        if (valid) {
          rs = ld_ro(a.row_ptr + i);
          re = ld_ro(a.row_ptr + i + 1);
        }
        is_long = valid;
      } else {
        i = ld_ro(a.huge_rows + ix);
        rs = ld_ro(a.row_ptr + i);
        re = ld_ro(a.row_ptr + i + 1);
        huge = true;
        is_long = false;
        valid = slot == 0;  // the first lane group owns the row's update
      }
    }
    S sx = P::zero(), sp = P::zero();
    if (ANY && huge) {
      for (int k = 0; k < nr; k++) {
        S hx, hp;
        if constexpr (YS) cta_row_sums_y<P>(a, st[k], nr, k, rs, re, hx, hp);
        else cta_row_sums<P, QX>(a, st[k], nr, k, rs, re, hx, hp);
        if (k == r) { sx = hx; sp = hp; }
      }
      if constexpr (YS) {
        if (valid && active) {  // the explicit-y sums carry -b (see below)
          const S bi = P::ldr(a.b + (size_t)i * nr + r);
          sx = P::sub(sx, bi);
          sp = P::sub(sp, bi);
        }
      }
    } else if (ANY && stn && valid && active) {
      // the up to 7 neighbours in ascending column order: -N^2, -N, -1, 0, +1, +N, +N^2
      // (bit k of inm: neighbour k lies in the grid); grid coordinates by
      // multiply-shift division (Granlund and Montgomery, PLDI 1994)
      const int N = a.sN, NN = a.sdim == 3 ? N * N : 0;
      const int q = (int)(((unsigned long long)i * a.smag) >> a.sshift);  // i / N
      const int ix = i - q * N;
      const int iy = a.sdim == 3 ? q - (int)(((unsigned long long)q * a.smag) >> a.sshift) * N : q;
      const unsigned inm = (ix > 0 ? 4u : 0u) | 8u | (ix < N - 1 ? 16u : 0u) | (iy > 0 ? 2u : 0u) |
                           (iy < N - 1 ? 32u : 0u) | (i >= NN && NN ? 1u : 0u) |
                           (NN && i < a.n - NN ? 64u : 0u);
      const bool two = !ONE && !same;
      // chunks of U neighbours, as for CSR rows: loads first, then the
      // multiply-adds in ascending order
      constexpr int U = kernel_row_unroll<P, SF, FM, MULTI>();
      // explicit y: the row sum starts at -b and yields g = Q y - b itself
      if constexpr (YS) sx = P::neg(P::ldr(a.b + (size_t)i * nr + r));
#pragma unroll
      for (int k0 = 0; k0 < 7; k0 += U) {
        S xv[U], pv[U];
#pragma unroll
        for (int j = 0; j < U; j++) {
          const int k = k0 + j;
          const int off = k == 0 ? -NN : k == 1 ? -N : k == 2 ? -1 : k == 3 ? 0 : k == 4 ? 1 : k == 5 ? N : NN;
          xv[j] = P::zero();
          pv[j] = P::zero();
          if (k < 7 && (inm >> k & 1u)) {
            const size_t e = (size_t)(i + off) * nr + r;
            xv[j] = P::ldg(xc + e);
            if (two) pv[j] = P::ldg(xp + e);
          }
        }
#pragma unroll
        for (int j = 0; j < U; j++) {
          const int k = k0 + j;
          if (k >= 7 || !(inm >> k & 1u)) continue;
          const V v = k == 3 ? s_diag : s_off;
          P::macv(sx, v, xv[j]);
          if (two) P::macv(sp, v, pv[j]);
        }
      }
      sx = P::finish(sx);
      if (!ONE) sp = same ? sx : P::finish(sp);
      if constexpr (YS) {
        sp = sx;
        if (y_check<P>(me))
          sp = stencil_pass<P, U>(i, inm, N, NN, s_diag, s_off, xp, nr, r, P::neg(P::ldr(a.b + (size_t)i * nr + r)));
      }
    } else if (valid && !is_long && active) {
      // chunks of U entries: every load of a chunk is issued before its
      // multiply-adds, which then run in ascending entry order
      constexpr int U = kernel_row_unroll<P, SF, FM, MULTI>();
      const bool two = !ONE && !same;
      if constexpr (YS)  // g = Q y - b itself (-b in the row's first lane only)
        sx = sub == 0 ? P::neg(P::ldr(a.b + (size_t)i * nr + r)) : P::zero();
      if constexpr (FM >= 3 && sell_pipe<P>()) {
        // the same chunks and multiply-adds in the same order; the columns
        // and values of the next chunk are loaded before this chunk's gathers
        // are used
        int cc[U];
        V vv[U];
#pragma unroll
        for (int k = 0; k < U; k++) {
          const bool in = k < cnt;
          cc[k] = in ? ld_ro(colp + k * stride) : 0;
          vv[k] = in ? P::ldv(valp + k * stride) : P::vzero();
        }
        for (int q0 = 0; q0 < cnt; q0 += U) {
          S xv[U], pv[U];
#pragma unroll
          for (int k = 0; k < U; k++) {
            xv[k] = P::zero();
            pv[k] = P::zero();
            if (q0 + k < cnt) {
              xv[k] = P::ldg(xc + (size_t)cc[k] * nr + r);
              if (two) pv[k] = P::ldg(xp + (size_t)cc[k] * nr + r);
            }
          }
          int cn[U];
          V vn[U];
#pragma unroll
          for (int k = 0; k < U; k++) {
            const bool in = q0 + U + k < cnt;
            cn[k] = in ? ld_ro(colp + (q0 + U + k) * stride) : 0;
            vn[k] = in ? P::ldv(valp + (q0 + U + k) * stride) : P::vzero();
          }
#pragma unroll
          for (int k = 0; k < U; k++) {
            if (q0 + k >= cnt) break;
            P::macv(sx, vv[k], xv[k]);
            if (two) P::macv(sp, vv[k], pv[k]);
          }
#pragma unroll
          for (int k = 0; k < U; k++) {
            cc[k] = cn[k];
            vv[k] = vn[k];
          }
        }
      } else {
        for (int q0 = 0; q0 < cnt; q0 += U) {
          int cc[U];
          V vv[U];
#pragma unroll
          for (int k = 0; k < U; k++) {
            const bool in = q0 + k < cnt;
            cc[k] = in ? ld_ro(colp + (q0 + k) * stride) : 0;
            vv[k] = in ? P::ldv(valp + (q0 + k) * stride) : P::vzero();
          }
          S xv[U], pv[U];
#pragma unroll
          for (int k = 0; k < U; k++) {
            xv[k] = P::zero();
            pv[k] = P::zero();
            if (q0 + k < cnt) {
              xv[k] = P::ldg(xc + (size_t)cc[k] * nr + r);
              if (two) pv[k] = P::ldg(xp + (size_t)cc[k] * nr + r);
            }
          }
#pragma unroll
          for (int k = 0; k < U; k++) {
            if (q0 + k >= cnt) break;
            P::macv(sx, vv[k], xv[k]);
            if (two) P::macv(sp, vv[k], pv[k]);
          }
        }
      }
      sx = P::finish(sx);
      if (!ONE) sp = same ? sx : P::finish(sp);
      if constexpr (YS) {
        sp = sx;
        if (y_check<P>(me))
          sp = row_pass<P, U>(colp, valp, cnt, stride, xp, nr, r,
                              sub == 0 ? P::neg(P::ldr(a.b + (size_t)i * nr + r)) : P::zero());
      }
    }
    if constexpr (FM == 4 || FM == 1) {
      if (split) {
        // the lanes of a row add their shares (xor over the lane bits above
        // log2 C, all within the row's lanes); its first lane updates it
        for (int m = 1 << a.sell_cl; m < 32; m <<= 1) {
          sx = P::combine(sx, P::shfl_xor(sx, m));
          sp = P::combine(sp, P::shfl_xor(sp, m));
        }
        valid = valid && sub == 0;
      }
    }
    // long rows: the whole warp sums each one for every right-hand side; the
    // lane of right-hand side k of the row's group takes sum k
    unsigned lm = FM == 2 ? 0u : __ballot_sync(0xffffffffu, is_long && r == 0);
    while (lm) {
      const int src = __ffs(lm) - 1;
      lm &= lm - 1;
      const int lrs = __shfl_sync(0xffffffffu, rs, src);
      const int lre = __shfl_sync(0xffffffffu, re, src);
      for (int k = 0; k < nr; k++) {
        S tx, tp;
        if constexpr (YS) long_row_sums_y<P>(a, st[k], nr, k, lrs, lre, tx, tp);
        else long_row_sums<P, QX>(a, st[k], nr, k, lrs, lre, tx, tp);
        if (lane == src + k) {
          sx = tx;
          sp = tp;
          if constexpr (YS) {  // -b, as the other explicit-y row sums carry it
            const S bi = P::ldr(a.b + (size_t)i * nr + r);
            sx = P::sub(sx, bi);
            sp = P::sub(sp, bi);
          }
        }
      }
    }
    if ((FM == 1 || FM == 2) && a.jblk > 1) {  // (the SELL-only kernels never meet a block J)
      // eq. J-blkdiag: x^t_i = y^t_i - sum_m (J^{bb})^{-1}_{im} g_m over the rows m
      // of i's block, which sit in lanes of this warp (blocks align with tiles
      // and jblk << lg <= 32); every lane takes part in the exchange
      const int jb = a.jblk;
      const bool upd = valid && active;
      const size_t e = (size_t)i * nr + r;
      S g = P::zero(), yi = P::zero(), xi = P::zero();
      if (YS && upd) {
        yi = P::ldg(xc + e);
        xi = same ? yi : P::ldx(xp + e);
        g = sx;  // Q y - b: the explicit-y row sums carry -b
        if (MON) P::acc_prod(acc[1], g, g);
        if (y_check<P>(me)) P::acc_prod(acc[2], sp, sp);
      } else if (upd) {
        xi = P::ldg(xc + e);
        const S bi = P::ldr(a.b + e);
        const S g0 = P::sub(sx, bi);
        P::acc_prod(acc[2], g0, g0);
        if (want_obj) {
          P::acc_prod(acc[3], xi, sx);
          P::acc_prod(acc[4], bi, xi);
        }
        if (QX) P::stx(uc + e, sx);
        if (same) {
          g = g0;
          yi = xi;
        } else {
          const S spi = QX ? P::ldx(up + e) : sp;
          g = P::fma_(beta, P::sub(sx, spi), g0);
          yi = DL ? P::fma_(beta, P::ldx(a.dl + e), xi) : P::fma_(beta, P::sub(xi, P::ldx(xp + e)), xi);
        }
      }
      if (!compute_x) continue;
      const int src0 = ((((int)threadIdx.x >> lg) & ~(jb - 1)) << lg | r) & 31;
      const X* jr = a.jinv + (size_t)i * jb;
      S corr = P::zero();
#pragma unroll
      for (int m = 0; m < 8; m++) {
        if (m >= jb) break;
        const S gm = P::shfl(g, src0 + (m << lg));
        if (upd) corr = P::fma_(P::ldr(jr + m), gm, corr);
      }
      if (upd) {
        const S xnew = P::sub(yi, corr);
        const S dx = P::sub(xnew, xi);
        P::stx(xn + e, xnew);
        if (DL) P::stx(a.dl + e, dx);
        if constexpr (YS) P::stx(ubuf(a, 1 - me.yb) + e, P::fma_(yk.bnext, dx, xnew));
        P::acc_prod(acc[0], g, dx);
      }
      continue;
    }
    if (!valid || !active) continue;
    const S ji = P::ldr(a.jinv + i);
    const size_t e = (size_t)i * nr + r;
    if constexpr (YS) {
      const S yi = P::ldg(xc + e);
      // g = Q y^s - b (the row sums start at -b): its norm schedules the
      // checks, and it is minus the exact residual of x^{s-1} where
      // y^s = x^{s-1}; sp = Q x^{s-1} - b on a check sweep
      const S g = sx;
      if (MON) P::acc_prod(acc[1], g, g);
      if (y_check<P>(me)) P::acc_prod(acc[2], sp, sp);
      if (!compute_x) continue;
      const S xi = same ? yi : P::ldx(xp + e);
      const S xnew = P::fnma(ji, g, yi);
      const S dx = P::sub(xnew, xi);
      P::stx(xn + e, xnew);
      P::stx(ubuf(a, 1 - me.yb) + e, P::fma_(yk.bnext, dx, xnew));
      P::acc_prod(acc[0], g, dx);
      continue;
    }
    const S xi = P::ldg(xc + e);
    const S bi = P::ldr(a.b + e);
    // g0 = Q x^{s-1} - b: minus the exact residual of x^{s-1}
    const S g0 = P::sub(sx, bi);
    P::acc_prod(acc[2], g0, g0);
    if (want_obj) {
      P::acc_prod(acc[3], xi, sx);
      P::acc_prod(acc[4], bi, xi);
    }
    if (QX) P::stx(uc + e, sx);
    if (!compute_x) continue;
    S g, yi;
    if (same) {
      g = g0;
      yi = xi;
    } else {
      const S spi = QX ? P::ldx(up + e) : sp;
      g = P::fma_(beta, P::sub(sx, spi), g0);
      if (DL) {
        yi = P::fma_(beta, P::ldx(a.dl + e), xi);
      } else {
        const S xpi = P::ldx(xp + e);
        yi = P::fma_(beta, P::sub(xi, xpi), xi);
      }
    }
    const S xnew = P::fnma(ji, g, yi);
    const S dx = P::sub(xnew, xi);
    P::stx(xn + e, xnew);
    if (DL) P::stx(a.dl + e, dx);
    P::acc_prod(acc[0], g, dx);
  }
}

// Explicit-y form: the next sweep also sums Q x^t (a check sweep) once
// ||Q y^t - b|| <= kChkFactor * tol * ||b|| / sqrt(gcal) (y^t extrapolates
// towards x^t, so this norm tracks the residual of x^t: measured ratios
// 0.6-2.3 at the stop on grid and graph Laplacians; gcal, the largest
// squared ratio of residual to monitor the check sweeps have seen, widens
// the trigger where it runs high), and in any case every kChkEvery
// iterations, so that a solve stops at most that many iterations after its
// first iterate within tol.
#ifndef AJ_CHK_FACTOR
#define AJ_CHK_FACTOR 1.5
#endif
#ifndef AJ_CHK_EVERY
#define AJ_CHK_EVERY 32
#endif
#ifndef AJ_MON_EVERY
#define AJ_MON_EVERY 4
#endif
constexpr double kChkFactor = AJ_CHK_FACTOR;
constexpr long long kChkEvery = AJ_CHK_EVERY;
// ||Q y - b||^2 is summed on every kMonEvery-th sweep only (one FP64
// instruction per row the other sweeps save), on every sweep once it is
// within kNearFactor of the stop (so that the checks start on a fresh
// value), and on the sweeps where y^s = x^{s-1}, whose exact residual it
// then is.
constexpr long long kMonEvery = AJ_MON_EVERY;
constexpr double kNearFactor = 10.0;
__device__ __forceinline__ bool monitor_sweep(const RhsState& q) {
  return q.cur == q.prev || q.near || q.t % kMonEvery == 0;
}

// alpha_{t+1} = (1 + sqrt(1 + 4 alpha_t^2)) / 2 (Algorithm alg-apg-re).
__device__ __forceinline__ double next_alpha(double a) { return 0.5 * (1.0 + sqrt(1.0 + 4.0 * a * a)); }

// Scalar step after the grid barrier, run by one thread per CTA with the
// grid totals tot[r][k].  Identical inputs give identical decisions in every
// CTA.  Returns true when every right-hand side is done.  ysf: the sweep ran
// in the explicit-y form (see sweep).
template <bool ysf>
__device__ __forceinline__ bool scalar_step(RhsState* st, const double (*tot)[kNRed], int nr, long long s,
                                            long long maxit, int stop, int restart, int momentum,
                                            double tol, double fstar, double fscale, long long* rlog,
                                            int rlog_cap, bool log_it) {
  bool all_done = true;
  for (int r = 0; r < nr; r++) {
    RhsState& q = st[r];
    if (q.done) continue;
    // explicit y: whether this right-hand side's own schedule summed the
    // monitor in the sweep (the sweep sums it for all when one needs it, but
    // each uses it on its own schedule, as it would alone)
    const bool mon = !ysf || monitor_sweep(q);
    const double d = tot[r][0];
    const double gg = tot[r][1];  // explicit y: valid where mon
    const double gmon_before = q.gmon;
    if (ysf && mon) q.gmon = gg;
    // the exact squared residual of x^{s-1}: summed by every sweep of the
    // lazy and stored forms; in the explicit-y form by check sweeps, and equal
    // to ||Q y^s - b||^2 where y^s = x^{s-1} (first sweep, after a restart)
    const bool same = q.cur == q.prev;
    const bool have_rr = !ysf || q.chk || same;
    const double rr = (ysf && same) ? gg : tot[r][2];
    // --- stop test for x^{s-1} (the iterate in buffer cur)
    if (have_rr) {
      const double rnorm = sqrt(rr);
      const double bn = sqrt(q.bnorm2);
      q.relres = bn > 0.0 ? rnorm / bn : rnorm;
      q.fval = fscale * (0.5 * tot[r][3] - tot[r][4]);
    }
    if (s == 1) q.rr0 = rr;
    if (ysf && q.chk && !same && gmon_before > 0.0) q.gcal = fmax(q.gcal, rr / gmon_before);
    bool stop_now = false;
    if (have_rr) {
      if (stop == kStopRelres) stop_now = q.relres <= tol;
      else if (stop == kStopObjgap) stop_now = fabs(q.fval - fstar) / (1.0 + fabs(fstar)) <= tol;
    }
    // divergence guard: the residual (at y^s in the explicit-y form, on its
    // monitor sweeps) against that of x^0
    const double grow = ysf ? (mon ? gg : 0.0) : rr;
    if (!isfinite(grow) || !isfinite(rr) || !isfinite(d)) {
      q.done = 1; q.status = kENonfinite; q.t_final = q.t;
      continue;
    }
    if (stop_now) {
      q.done = 1; q.status = kOk; q.t_final = q.t;
      continue;
    }
    if (q.t >= maxit) {
      q.done = 1; q.status = kEMaxit; q.t_final = q.t;
      continue;
    }
    if (s > 1 && q.rr0 > 0.0 && grow > 1e16 * q.rr0) {
      q.done = 1; q.status = kEDiverged; q.t_final = q.t;
      continue;
    }
    // --- iteration t = s: restart rule of Algorithm alg-apg-re
    const long long t = q.t + 1;
    const bool do_restart = restart && (t > q.Kre + q.K) && (d >= 0.0);
    if (do_restart) {
      if (log_it && q.ell < rlog_cap) rlog[(size_t)r * rlog_cap + q.ell] = t;
      q.Kre = t;
      q.K = 2 * q.K;
      q.ell += 1;
      q.alpha = 1.0;  // alpha_{t+1} = 1 (alpha_t = 0 is never read again)
      q.beta = 0.0;
      // x^t = x^{t-1}: the buffer cur already holds x^{t-1}; prev := cur
      q.prev = q.cur;
      q.nxt = (q.cur == 0) ? 1 : 0;
    } else {
      double an = 1.0, be = 0.0;
      if (momentum) {
        an = next_alpha(q.alpha);
        be = (q.alpha - 1.0) / an;
      }
      q.alpha = an;
      q.beta = be;
      const int oldprev = q.prev, oldcur = q.cur, oldnew = q.nxt;
      q.prev = oldcur;
      q.cur = oldnew;
      q.nxt = (oldprev != oldcur && oldprev != oldnew) ? oldprev : (3 - oldcur - oldnew);
      if (ysf) q.yb = 1 - q.yb;  // explicit y: the candidate this sweep wrote is y^{t+1}
    }
    q.uw = 1 - q.uw;
    q.t = t;
    if (ysf) {
      q.beta_next = momentum ? (q.alpha - 1.0) / next_alpha(q.alpha) : 0.0;
      const double bn2 = q.bnorm2 > 0.0 ? q.bnorm2 : 1.0;
      const double est = q.gmon * fmax(1.0, q.gcal);  // the residual it stands for, squared
      q.chk = stop == kStopRelres &&
              (est <= kChkFactor * kChkFactor * tol * tol * bn2 || t % kChkEvery == 0 || t >= maxit);
      q.near = stop == kStopRelres && est <= kNearFactor * kNearFactor * tol * tol * bn2;
    }
    all_done = false;
  }
  return all_done;
}

// Co-resident CTAs per SM (P::kMinBlocks, P::kMinBlocksMulti) the register
// allocation must allow.  The sweep is latency bound (gathers from L2, the
// matrix stream from DRAM), so warps in flight matter more than registers:
// on the 256^3 Poisson system 4 CTAs/SM beat the compiler's own choice of
// 2-3 by 1.3-1.7x in FP64, and the FP32/BF16 policies gain again from 6-8.

// Shared memory of one solve: per-RHS state, grid totals, reduction scratch.
struct SolveSmem {
  RhsState st[kMaxRhs];
  double tot[kMaxRhs][kNRed];
  double red[kWarps * kMaxRhs * kNRed];
  int done;
};

// Grid totals tot[r][k] of the per-CTA partials part[c][r][k] (c < ncta) for
// every right-hand side r < nr and used slot k, in one pass.  Each total is
// summed in a fixed order that does not depend on nr or on which CTA runs
// this: thread t adds the partials of CTAs t, t + 256, ... in ascending
// order, then a xor tree over the lanes and the warps in order.  Every
// thread must call it; the totals are valid in sm.tot after it returns.
__device__ __forceinline__ void grid_totals(const double* part, int ncta, int nr, bool want_obj,
                                            bool want_gg, SolveSmem& sm) {
  constexpr int NV = kMaxRhs * kNRed;
  double v[NV];
#pragma unroll
  for (int q = 0; q < NV; q++) v[q] = 0.0;
  const int nslot = want_obj ? kNRed : 3;
  for (int c = threadIdx.x; c < ncta; c += kThreads) {
    const double* pc = part + (size_t)c * nr * kNRed;
#pragma unroll
    for (int r = 0; r < kMaxRhs; r++)
#pragma unroll
      for (int k = 0; k < kNRed; k++)
        if (r < nr && k < nslot && slot_used(k, want_obj, want_gg)) v[r * kNRed + k] += __ldcg(pc + r * kNRed + k);
  }
  const int w = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NV; q++) {
    if (q / kNRed >= nr || !slot_used(q % kNRed, want_obj, want_gg)) continue;
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], m);
    if ((threadIdx.x & 31) == 0) sm.red[w * NV + q] = v[q];
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    const int q = threadIdx.x;
    double t = 0.0;
    if (q / kNRed < nr && slot_used(q % kNRed, want_obj, want_gg))
      for (int i = 0; i < kWarps; i++) t += sm.red[i * NV + q];
    sm.tot[q / kNRed][q % kNRed] = t;
  }
  __syncthreads();
}

// Runs sweeps of one system on `ncta` co-resident CTAs (this one is `cta`)
// until every right-hand side is done or a.max_sweeps sweeps have run.  The
// state is in sm.st (identical in every CTA).  `target` is the barrier's
// arrival count so far and `sw` the sweep counter that parity-buffers the
// partials; both carry over between systems that reuse the same barrier.
// Returns false when a barrier gave up (error already recorded in *a.err).
template <class P, int SF, int FM, bool MULTI>
__device__ __forceinline__ bool run_solve(const IterArgs<P>& a, SolveSmem& sm, int cta, int ncta,
                                          unsigned long long& target, long long& sw) {
  using A = typename P::A;
  const bool want_obj = a.stop == kStopObjgap;
  const int nr = MULTI ? a.nrhs : 1;
  const int lg = MULTI ? a.lgr : 0;
  for (long long s0 = 0; s0 < a.max_sweeps; s0++, sw++) {
    // sweep number in the run's own numbering: x^{s-1} is checked, x^s formed
    long long s_run = 0;
    bool compute_x = false;
    bool mon = SF != 3;  // explicit y: is ||Q y - b||^2 summed this sweep?
    for (int r = 0; r < nr; r++) {
      if (!sm.st[r].done) {
        s_run = sm.st[r].t + 1;
        compute_x = compute_x || (sm.st[r].t < a.maxit);
        mon = mon || monitor_sweep(sm.st[r]);
      }
    }
    A acc[kNRed];
#pragma unroll
    for (int k = 0; k < kNRed; k++) acc_zero(acc[k]);
    if constexpr (SF == 3) {
      if (mon) sweep<P, SF, FM, MULTI, true>(a, sm.st, compute_x, want_obj, acc, cta, ncta);
      else sweep<P, SF, FM, MULTI, false>(a, sm.st, compute_x, want_obj, acc, cta, ncta);
    } else {
      sweep<P, SF, FM, MULTI>(a, sm.st, compute_x, want_obj, acc, cta, ncta);
    }
    // CTA partials -> global (parity-buffered by sweep)
    double* part = a.partials + (size_t)(sw & 1) * ncta * nr * kNRed;
#pragma unroll
    for (int k = 0; k < kNRed; k++) {
      if (!slot_used(k, want_obj, SF == 3)) continue;
      const double v = block_sum_rhs(acc_value(acc[k]), sm.red, lg, nr);
      if ((int)threadIdx.x < nr) __stcg(part + ((size_t)cta * nr + threadIdx.x) * kNRed + k, v);
    }
    target += (unsigned long long)ncta;
    if (!grid_sync(a.bar, target, a.err, (unsigned)ncta, a.bar_timeout_ns,
                   s0 == 0 && cta == a.bar_withhold_cta))
      return false;
    // every CTA sums the partials in the same fixed order
    grid_totals(part, ncta, nr, want_obj, SF == 3, sm);
    if (threadIdx.x == 0) {
      if (a.trace && cta == 0 && s_run >= 1 && s_run <= a.trace_cap) {
        for (int r = 0; r < nr; r++) {
          double* tr = a.trace + ((size_t)(s_run - 1) * nr + r) * 4;
          tr[0] = sm.tot[r][0];
          tr[1] = sm.tot[r][1];
          tr[2] = sm.tot[r][2];
          tr[3] = sm.st[r].beta;
        }
      }
      sm.done = scalar_step<SF == 3>(sm.st, sm.tot, nr, s_run, a.maxit, a.stop, a.restart, a.momentum,
                                     a.tol, a.fstar, a.fscale, a.rlog, a.rlog_cap, cta == 0)
                    ? 1
                    : 0;
    }
    __syncthreads();
    if (sm.done) {
      sw++;
      break;
    }
  }
  return true;
}

// The persistent fused AJ kernel for one system.  Launch cooperatively with
// kThreads threads per CTA; every CTA of the grid works on the system.  FM
// selects the formats the instantiation reads (see sweep), MULTI the one for
// several right-hand sides.
template <class P, int SF, int FM, bool MULTI>
__global__ void __launch_bounds__(kThreads, (kernel_min_blocks<P, SF, FM, MULTI>())) aj_persistent_kernel(IterArgs<P> a) {
  __shared__ SolveSmem sm;
  const int nr = MULTI ? a.nrhs : 1;
  if ((int)threadIdx.x < nr) sm.st[threadIdx.x] = a.state[threadIdx.x];
  __syncthreads();
  unsigned long long target = 0;
  long long sw = 0;
  if (!run_solve<P, SF, FM, MULTI>(a, sm, blockIdx.x, gridDim.x, target, sw)) return;
  if (blockIdx.x == 0 && (int)threadIdx.x < nr) a.state[threadIdx.x] = sm.st[threadIdx.x];
}

// ----------------------------------------------------------------------------
// Many independent systems in lockstep.  System s is cut into V_s units: unit
// v holds its tiles v, v + V_s, ... -- exactly the tiles CTA v of a solo run
// with V_s CTAs sweeps, in the same order, with the same per-unit reduction,
// so a system computes bit for bit what aj_solve computes with grid_ctas =
// V_s.  Every sweep each CTA takes a contiguous range of the unit list, the
// ranges cut so that each holds about the same estimated work (the units of
// a system are consecutive, so a CTA meets few systems), then all CTAs meet
// at one grid barrier: a sweep costs the combined work of the active systems
// spread over the whole GPU.
//
// State.  The state a system uses in sweep k of this launch is kept in
// st2[s][k & 1] (st2[s][0] staged by the host).  A CTA that meets system s in
// sweep k >= 1 first turns state k-1 and the partial sums of sweep k-1 into
// state k (identical bits in every CTA); the CTA that holds unit 0 stores it.
// A system whose right-hand sides are all done stops sweeping.  After the
// last sweep the CTA holding unit 0 applies the last transition and writes
// the state to st_out[s], so that a launch takes a state and returns one,
// exactly as a solo run of `sweeps` sweeps would.
template <class P>
struct LockArgs {
  const IterArgs<P>* sys;     // [m] per system; partials [2][V_s][nrhs][kNRed] are its own
  const int* unit_sys;        // [nu] system of each unit (the units of a system are consecutive)
  const int* sys_u0;          // [m] first unit of each system
  const int* sys_nu;          // [m] V_s
  const int* cta_u0;          // [gridDim + 1] CTA c sweeps units cta_u0[c] .. cta_u0[c+1]-1
  RhsState* st2;              // [m][2][kMaxRhs]
  RhsState* st_out;           // [m][kMaxRhs]
  int nu;
  long long sweeps;           // sweeps of this launch, >= 1
  unsigned long long* bar;    // grid barrier counter, zero at launch
  int* err;                   // device error word, zero at launch
};

// RhsState moved word by word through L2 (other CTAs write it between sweeps).
static_assert(sizeof(RhsState) % 8 == 0, "state of whole 64-bit words");
__device__ __forceinline__ RhsState ld_state_l2(const RhsState* p) {
  RhsState v;
  const unsigned long long* src = reinterpret_cast<const unsigned long long*>(p);
  unsigned long long* dst = reinterpret_cast<unsigned long long*>(&v);
#pragma unroll
  for (int k = 0; k < (int)(sizeof(RhsState) / 8); k++) dst[k] = __ldcg(src + k);
  return v;
}
__device__ __forceinline__ void st_state_l2(RhsState* p, const RhsState& v) {
  const unsigned long long* src = reinterpret_cast<const unsigned long long*>(&v);
  unsigned long long* dst = reinterpret_cast<unsigned long long*>(p);
#pragma unroll
  for (int k = 0; k < (int)(sizeof(RhsState) / 8); k++) __stcg(dst + k, src[k]);
}

// Loads system s's arguments into shared memory and brings its state to
// sweep k (applying the transition of sweep k-1 when k >= 1).  A system runs
// kmax = min(launch sweeps, a.max_sweeps) sweeps in this launch: at k = kmax
// its last transition is applied and kept, and from then on it pauses (its
// state stays in st2[kmax & 1]).  Returns, in every thread, whether the
// system skips sweep k (done or paused).  `store` makes this CTA the one that
// keeps the new state in st2; `log_it` the one that records restarts.
template <class P, int SF>
__device__ __forceinline__ bool lock_enter(const LockArgs<P>& b, IterArgs<P>& a, SolveSmem& sm, int s,
                                           long long k, bool store, bool log_it) {
  constexpr int kWords = (int)(sizeof(IterArgs<P>) / 4);
  static_assert(sizeof(IterArgs<P>) % 4 == 0, "argument block of whole words");
  __syncthreads();
  const unsigned* src = reinterpret_cast<const unsigned*>(b.sys + s);
  unsigned* dst = reinterpret_cast<unsigned*>(&a);
  for (int w = threadIdx.x; w < kWords; w += kThreads) dst[w] = __ldg(src + w);
  __syncthreads();
  const int nr = a.nrhs;
  const bool want_obj = a.stop == kStopObjgap;
  const int V = __ldg(b.sys_nu + s);
  const long long kmax = a.max_sweeps < b.sweeps ? a.max_sweeps : b.sweeps;
  const bool paused = k > kmax;
  const long long kk = paused ? kmax : k;
  RhsState* stc = b.st2 + ((size_t)s * 2 + (kk & 1)) * kMaxRhs;
  const RhsState* stp = b.st2 + ((size_t)s * 2 + ((kk - 1) & 1)) * kMaxRhs;
  if ((int)threadIdx.x < nr)
    sm.st[threadIdx.x] = ld_state_l2((paused || k == 0) ? stc + threadIdx.x : stp + threadIdx.x);
  __syncthreads();
  if (threadIdx.x == 0) {
    int d = 1;
    for (int r = 0; r < nr; r++) d = d && sm.st[r].done;
    sm.done = d;
  }
  __syncthreads();
  if (!paused && k > 0 && !sm.done) {
    long long s_run = 0;
    for (int r = 0; r < nr; r++)
      if (!sm.st[r].done) s_run = sm.st[r].t + 1;
    grid_totals(a.partials + (size_t)((k - 1) & 1) * V * nr * kNRed, V, nr, want_obj, SF == 3, sm);
    if (threadIdx.x == 0)
      sm.done = scalar_step<SF == 3>(sm.st, sm.tot, nr, s_run, a.maxit, a.stop, a.restart, a.momentum,
                                     a.tol, a.fstar, a.fscale, a.rlog, a.rlog_cap, log_it)
                    ? 1
                    : 0;
    __syncthreads();
  }
  if (!paused && store && k > 0 && (int)threadIdx.x < nr) st_state_l2(stc + threadIdx.x, sm.st[threadIdx.x]);
  return sm.done != 0 || k >= kmax;
}

// One unit's sweep in the instantiation of its system's format (as a solo
// run of the same system launches it): the stencil rows alone, SELL alone
// (slices of 32 rows, or of 8 or 16 with split rows), CSR alone, or any
// format for the block-diagonal J.
#ifndef AJ_LOCK_BY_FORMAT
#define AJ_LOCK_BY_FORMAT 1
#endif
// CTAs per SM of the lockstep kernel: 5 for FP32 and BF16 values (256
// systems of the batched mix in FP32-IR: 7.03 s, against 8.0 s at 4, 8.2 s
// at 6 where it spills and 9.5 s at 3), the policy's multi-RHS count for
// FP64 and double-float values; AJ_LOCK_MINB > 0 overrides both
#ifndef AJ_LOCK_MINB
#define AJ_LOCK_MINB 0
#endif
template <class P>
__host__ __device__ constexpr int lock_min_blocks() {
  return AJ_LOCK_MINB > 0 ? AJ_LOCK_MINB : P::kId >= 2 ? 5 : P::kMinBlocksMulti;
}
template <class P, int SF, bool MON>
__device__ __forceinline__ void lock_sweep(const IterArgs<P>& a, const RhsState* st, bool compute_x,
                                           bool want_obj, typename P::A (&acc)[kNRed], int v, int V) {
  if (!AJ_LOCK_BY_FORMAT || a.jblk > 1) sweep<P, SF, 1, true, MON>(a, st, compute_x, want_obj, acc, v, V);
  else if (a.fmt == 2) sweep<P, SF, 2, true, MON>(a, st, compute_x, want_obj, acc, v, V);
  else if (a.fmt == 1 && a.sell_cl < 5) sweep<P, SF, 4, true, MON>(a, st, compute_x, want_obj, acc, v, V);
  else if (a.fmt == 1) sweep<P, SF, 3, true, MON>(a, st, compute_x, want_obj, acc, v, V);
  else sweep<P, SF, 0, true, MON>(a, st, compute_x, want_obj, acc, v, V);
}

template <class P, int SF>
__global__ void __launch_bounds__(kThreads, lock_min_blocks<P>()) aj_lockstep_kernel(LockArgs<P> b) {
  __shared__ SolveSmem sm;
  __shared__ IterArgs<P> a;
  using A = typename P::A;
  const int u_lo = __ldg(b.cta_u0 + blockIdx.x);
  const int u_hi = __ldg(b.cta_u0 + blockIdx.x + 1);
  unsigned long long target = 0;
  for (long long k = 0; k < b.sweeps; k++) {
    int cur = -1;
    bool done = false;
    for (int u = u_lo; u < u_hi; u++) {
      const int s = __ldg(b.unit_sys + u);
      const int v = u - __ldg(b.sys_u0 + s);
      if (s != cur) {
        done = lock_enter<P, SF>(b, a, sm, s, k, v == 0, v == 0);
        cur = s;
      }
      if (done) continue;
      const int nr = a.nrhs;
      const bool want_obj = a.stop == kStopObjgap;
      const int V = __ldg(b.sys_nu + s);
      bool compute_x = false;
      bool mon = SF != 3;  // the monitor schedule of a solo run, from the same state
      for (int r = 0; r < nr; r++)
        if (!sm.st[r].done) {
          compute_x = compute_x || (sm.st[r].t < a.maxit);
          mon = mon || monitor_sweep(sm.st[r]);
        }
      A acc[kNRed];
#pragma unroll
      for (int q = 0; q < kNRed; q++) acc_zero(acc[q]);
      // (the objective-gap stop never takes the explicit-y form)
      if constexpr (SF == 3) {
        if (mon) lock_sweep<P, SF, true>(a, sm.st, compute_x, false, acc, v, V);
        else lock_sweep<P, SF, false>(a, sm.st, compute_x, false, acc, v, V);
      } else {
        lock_sweep<P, SF, true>(a, sm.st, compute_x, want_obj, acc, v, V);
      }
      double* part = a.partials + (size_t)(k & 1) * V * nr * kNRed;
#pragma unroll
      for (int q = 0; q < kNRed; q++) {
        if (!slot_used(q, want_obj, SF == 3)) continue;
        const double t = block_sum_rhs(acc_value(acc[q]), sm.red, a.lgr, nr);
        if ((int)threadIdx.x < nr) __stcg(part + ((size_t)v * nr + threadIdx.x) * kNRed + q, t);
      }
    }
    target += (unsigned long long)gridDim.x;
    if (!grid_sync(b.bar, target, b.err, gridDim.x)) return;
  }
  // the last transition, by the CTA that holds each system's unit 0
  for (int u = u_lo; u < u_hi; u++) {
    const int s = __ldg(b.unit_sys + u);
    if (u != __ldg(b.sys_u0 + s)) continue;
    lock_enter<P, SF>(b, a, sm, s, b.sweeps, false, true);
    if ((int)threadIdx.x < a.nrhs) b.st_out[(size_t)s * kMaxRhs + threadIdx.x] = sm.st[threadIdx.x];
  }
}

}  // namespace aj
