// aj_pcg.cuh -- the comparator of Sec. 4.2: conjugate gradients with the
// diagonal preconditioner M = diag(Q), FP64, as one persistent cooperative
// kernel over the context's CSR rows (one right-hand side).
//
// The recurrence is Saad's Alg. 9.1 (Iterative Methods for Sparse Linear
// Systems, 2nd ed.).  Each iteration is two grid-synchronised passes:
//   A: p_i = z_i + beta p'_i and q_i = sum_j Q_ij (z_j + beta p'_j), the new
//      direction formed inside the SpMV gather (p' is the previous one), and
//      the partial sums of <p, q>;
//   B: alpha = <r, z> / <p, q>; x += alpha p; r -= alpha q; z = M^{-1} r, and
//      the partial sums of <r, z> and <r, r>.
// After B every CTA sums the partials in the same order, so all take the same
// beta and the same stop decision (||r|| <= tol ||b||, the recursive
// residual, as in the oracle).  Rows longer than 32 entries are summed by the
// whole warp.
#pragma once
#include "aj_core.cuh"

namespace aj {

struct PcgArgs {
  int n;
  const int* rp;
  const int* ci;
  const double* val;
  const double* b;
  double* x;        // x^0 on entry, the result on exit
  double* r;
  double* z;
  double* p[2];     // directions of even and odd iterations
  double* q;
  double* part;     // [2][grid][2] per-CTA partial sums, parity-buffered by pass
  unsigned long long* bar;
  int* err;
  long long maxit;
  double tol;
  double bnorm;
  long long* out_iters;
  double* out_rn;
};

// sum_j Q_ij v_j over entries e = e0, e0 + step, ... < e1, with
// v_j = z_j + beta p'_j (p' = nullptr: v = x)
__device__ __forceinline__ double pcg_dot_row(const PcgArgs& a, const double* v0, const double* pold,
                                              double beta, int e0, int e1, int step) {
  double s = 0.0;
  for (int e = e0; e < e1; e += step) {
    const int c = ld_ro(a.ci + e);
    const double vj = pold ? fma(beta, ld_l2(pold + c), ld_l2(v0 + c)) : ld_l2(v0 + c);
    s = fma(ld_ro(a.val + e), vj, s);
  }
  return s;
}

// Sum of two per-thread values over the grid: block sums to part[parity],
// a barrier, then every CTA adds the grid's partials in CTA order.
__device__ __forceinline__ bool pcg_grid_sum2(const PcgArgs& a, double v0, double v1, int parity,
                                              unsigned long long& target, double& s0, double& s1) {
  __shared__ double sm[kWarps];
  __shared__ double tot[2];
  const double b0 = block_sum(v0, sm);
  const double b1 = block_sum(v1, sm);
  double* part = a.part + (size_t)parity * gridDim.x * 2;
  if (threadIdx.x == 0) {
    st_l2(part + 2 * blockIdx.x, b0);
    st_l2(part + 2 * blockIdx.x + 1, b1);
  }
  target += gridDim.x;
  if (!grid_sync(a.bar, target, a.err, gridDim.x)) return false;
  if (threadIdx.x == 0) {
    double t0 = 0.0, t1 = 0.0;
    for (unsigned k = 0; k < gridDim.x; k++) {
      t0 += ld_l2(part + 2 * k);
      t1 += ld_l2(part + 2 * k + 1);
    }
    tot[0] = t0;
    tot[1] = t1;
  }
  __syncthreads();
  s0 = tot[0];
  s1 = tot[1];
  return true;
}

// One pass of row sums over the CTA's tiles: for row i, q_i = sum_j Q_ij v_j
// (v as in pcg_dot_row); fn(i, q_i) consumes each.
template <class F>
__device__ __forceinline__ void pcg_rows(const PcgArgs& a, const double* v0, const double* pold, double beta,
                                         F fn) {
  const int lane = threadIdx.x & 31;
  const int ntiles = (a.n + kThreads - 1) / kThreads;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int i = tile * kThreads + threadIdx.x;
    const bool valid = i < a.n;
    int rs = 0, re = 0;
    if (valid) {
      rs = ld_ro(a.rp + i);
      re = ld_ro(a.rp + i + 1);
    }
    const bool is_long = valid && re - rs > 32;
    double s = 0.0;
    if (valid && !is_long) s = pcg_dot_row(a, v0, pold, beta, rs, re, 1);
    unsigned lm = __ballot_sync(0xffffffffu, is_long);
    while (lm) {
      const int src = __ffs(lm) - 1;
      lm &= lm - 1;
      const int lrs = __shfl_sync(0xffffffffu, rs, src);
      const int lre = __shfl_sync(0xffffffffu, re, src);
      double t = pcg_dot_row(a, v0, pold, beta, lrs + lane, lre, 32);
#pragma unroll
      for (int m = 16; m >= 1; m >>= 1) t += __shfl_xor_sync(0xffffffffu, t, m);
      if (lane == src) s = t;
    }
    if (valid) fn(i, s);
  }
}

__global__ void __launch_bounds__(kThreads, 4) aj_pcg_kernel(PcgArgs a) {
  unsigned long long target = 0;
  int parity = 0;
  // r^0 = b - Q x^0, z^0 = M^{-1} r^0, p' = 0 so that p^0 = z^0.  M^{-1}
  // goes to the second half of q (the caller gives q room for 2n values);
  // every row's values are written and read by the same thread, as are r, x
  // and q in pass B, while z and p are gathered by all CTAs after a barrier
  double* minv = a.q + a.n;
  double rz = 0.0, rr = 0.0;
  {
    double lz = 0.0, lr = 0.0;
    pcg_rows(a, a.x, nullptr, 0.0, [&](int i, double qx) {
      double d = 0.0;
      for (int e = ld_ro(a.rp + i); e < ld_ro(a.rp + i + 1); e++)
        if (ld_ro(a.ci + e) == i) d += ld_ro(a.val + e);
      const double ri = ld_ro(a.b + i) - qx;
      const double mi = 1.0 / (d == 0.0 ? 1.0 : d);
      const double zi = mi * ri;
      st_l2(a.r + i, ri);
      st_l2(a.z + i, zi);
      st_l2(a.p[1] + i, 0.0);
      st_l2(minv + i, mi);
      lz = fma(ri, zi, lz);
      lr = fma(ri, ri, lr);
    });
    if (!pcg_grid_sum2(a, lz, lr, parity, target, rz, rr)) return;
    parity ^= 1;
  }
  long long t = 0;
  double rn = sqrt(rr);
  double beta = 0.0;
  while (t < a.maxit && !(rn <= a.tol * a.bnorm)) {
    double* pnew = a.p[t & 1];
    const double* pold = a.p[(t & 1) ^ 1];
    // pass A
    double lpq = 0.0;
    pcg_rows(a, a.z, pold, beta, [&](int i, double qi) {
      const double pi = fma(beta, ld_l2(pold + i), ld_l2(a.z + i));
      st_l2(pnew + i, pi);
      st_l2(a.q + i, qi);
      lpq = fma(pi, qi, lpq);
    });
    double pq = 0.0, unused = 0.0;
    if (!pcg_grid_sum2(a, lpq, 0.0, parity, target, pq, unused)) return;
    parity ^= 1;
    // pass B
    const double alpha = rz / pq;
    double lz = 0.0, lr = 0.0;
    for (int tile = blockIdx.x; tile * kThreads < a.n; tile += gridDim.x) {
      const int i = tile * kThreads + threadIdx.x;
      if (i < a.n) {
        const double pi = ld_l2(pnew + i);
        const double xi = fma(alpha, pi, ld_l2(a.x + i));
        const double ri = fma(-alpha, ld_l2(a.q + i), ld_l2(a.r + i));
        const double zi = ld_l2(minv + i) * ri;
        st_l2(a.x + i, xi);
        st_l2(a.r + i, ri);
        st_l2(a.z + i, zi);
        lz = fma(ri, zi, lz);
        lr = fma(ri, ri, lr);
      }
    }
    double rz_new = 0.0;
    if (!pcg_grid_sum2(a, lz, lr, parity, target, rz_new, rr)) return;
    parity ^= 1;
    beta = rz_new / rz;
    rz = rz_new;
    rn = sqrt(rr);
    t++;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *a.out_iters = t;
    *a.out_rn = rn;
  }
}

}  // namespace aj
