// aj_setup.cuh -- setup and auxiliary kernels: CSR validation, the diagonal
// proximal matrix J (eq. J-diag, Section 3, or J = L D), precision
// conversions, the FP64 residual b - Q x, and the power iteration that
// estimates L = lambda_max(D^-1/2 Q D^-1/2).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <limits.h>
#include <stdint.h>

#include "aj_core.cuh"

namespace aj {

constexpr int kSetupThreads = 256;

// Error bits written by the validation kernels.
enum : int {
  kBadRowPtr = 1,       // row_ptr[0] != 0, decreasing, or row_ptr[n] != nnz
  kBadCol = 2,          // column index outside [0, n)
  kNonFinite = 4,       // NaN or Inf value
  kNegDiag = 8,         // negative diagonal entry (Q not PSD)
  kZeroDiagNonzero = 16 // zero diagonal but a nonzero off-diagonal entry (Q not PSD)
};

__global__ void k_check_rowptr(int n, long long nnz, const int* rp, int* flags) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i > n) return;
  const int v = rp[i];
  if (v < 0 || (long long)v > nnz) atomicOr(flags, kBadRowPtr);
  if (i == 0 && v != 0) atomicOr(flags, kBadRowPtr);
  if (i == n && (long long)v != nnz) atomicOr(flags, kBadRowPtr);
  if (i < n && rp[i + 1] < v) atomicOr(flags, kBadRowPtr);
}

// Requires a valid row_ptr.  Writes diag[i] = sum of the diagonal entries of
// row i and checks columns, finiteness and the PSD-necessary diagonal rules.
__global__ void k_check_rows(int n, const int* rp, const int* ci, const double* val, double* diag,
                             int* flags) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double d = 0.0;
  bool off_nonzero = false;
  int f = 0;
  for (int q = rp[i]; q < rp[i + 1]; q++) {
    const int c = ci[q];
    const double v = val[q];
    if (c < 0 || c >= n) f |= kBadCol;
    if (!isfinite(v)) f |= kNonFinite;
    if (c == i) d += v;
    else if (v != 0.0) off_nonzero = true;
  }
  if (d < 0.0) f |= kNegDiag;
  if (d == 0.0 && off_nonzero) f |= kZeroDiagNonzero;
  diag[i] = d;
  if (f) atomicOr(flags, f);
}

// J^{-1} in FP64.  policy 0: eq. J-diag, J_kk = Q_kk + sum_{j!=k} |Q_kj| (the
// off-diagonal magnitudes summed in CSR order); policy 1: J_kk = L Q_kk.
// A zero J_kk (all-zero row) becomes 1.
__global__ void k_jinv(int n, const int* rp, const int* ci, const double* val, const double* diag,
                       int policy, double L, double* jinv) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double j;
  if (policy == 0) {
    double off = 0.0;
    for (int q = rp[i]; q < rp[i + 1]; q++)
      if (ci[q] != i) off += fabs(val[q]);
    j = diag[i] + off;
  } else {
    j = L * diag[i];
  }
  if (j == 0.0) j = 1.0;
  jinv[i] = 1.0 / j;
}

// Scaled copies into the precision of the iteration (scale is a power of two).
__global__ void k_to_f32(long long m, const double* src, double scale, float* dst) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) dst[i] = __double2float_rn(src[i] * scale);
}
__global__ void k_to_b16(long long m, const double* src, double scale, __nv_bfloat16* dst) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) dst[i] = __double2bfloat16(src[i] * scale);
}
__global__ void k_to_dw(long long m, const double* src, double scale, float2* dst) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) {
    dw v = dw_from_double(src[i] * scale);
    dst[i] = make_float2(v.hi, v.lo);
  }
}
// Per right-hand-side scales and source buffers for the interleaved vectors.
struct RhsMap {
  double s[kMaxRhs];
  int cur[kMaxRhs];
};
__device__ __forceinline__ void to_x(double v, double* d) { *d = v; }
__device__ __forceinline__ void to_x(double v, float* d) { *d = __double2float_rn(v); }
__device__ __forceinline__ void to_x(double v, float2* d) {
  dw w = dw_from_double(v);
  *d = make_float2(w.hi, w.lo);
}
__device__ __forceinline__ double from_x(double v) { return v; }
__device__ __forceinline__ double from_x(float v) { return (double)v; }
__device__ __forceinline__ double from_x(float2 v) { return (double)v.x + (double)v.y; }

// dst[e] = src[e] * s[e % nrhs] in the iteration precision.
template <class X>
__global__ void k_to_policy(long long m, int nrhs, const double* src, RhsMap mp, X* dst) {
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < m) to_x(src[e] * mp.s[e % nrhs], dst + e);
}
// dst[e] = buf[cur[r]][e] * s[r], r = e % nrhs, back to FP64.
template <class X>
__global__ void k_from_policy(long long m, int nrhs, const X* b0, const X* b1, const X* b2,
                              RhsMap mp, double* dst) {
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m) return;
  const int r = (int)(e % nrhs);
  const int k = mp.cur[r];
  const X* src = k == 0 ? b0 : (k == 1 ? b1 : b2);
  dst[e] = from_x(src[e]) * mp.s[r];
}

// Column-major (n x nrhs) <-> interleaved (i * nrhs + r).
__global__ void k_interleave(int n, int nrhs, const double* cm, double* il) {
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)n * nrhs) return;
  const int r = (int)(e % nrhs);
  const long long i = e / nrhs;
  il[e] = cm[(long long)r * n + i];
}
__global__ void k_deinterleave(int n, int nrhs, const double* il, double* cm) {
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)n * nrhs) return;
  const int r = (int)(e % nrhs);
  const long long i = e / nrhs;
  cm[(long long)r * n + i] = il[e];
}

// FP64 residual r = b - Q x for interleaved multi-RHS vectors; per-block
// partial sums of r_r^2 and (optionally) <x, Qx>, <b, x> go to part[block][nrhs][3].
// Rows longer than long_len are left to k_residual_long (a warp per row) and
// contribute nothing here; long_len < 0 keeps every row.
__global__ void k_residual(int n, int nrhs, const int* rp, const int* ci, const double* val,
                           const double* b, const double* x, double* r_out, double* part,
                           int long_len) {
  __shared__ double sm[kMaxRhs * 3][kSetupThreads / 32];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double acc[kMaxRhs * 3];
  for (int k = 0; k < kMaxRhs * 3; k++) acc[k] = 0.0;
  if (i < n && (long_len < 0 || rp[i + 1] - rp[i] <= long_len)) {
    double s[kMaxRhs] = {0.0, 0.0, 0.0, 0.0};
    for (int q = rp[i]; q < rp[i + 1]; q++) {
      const double v = val[q];
      const long long c = ci[q];
      for (int r = 0; r < nrhs; r++) s[r] = fma(v, x[c * nrhs + r], s[r]);
    }
    for (int r = 0; r < nrhs; r++) {
      const long long e = (long long)i * nrhs + r;
      const double res = b[e] - s[r];
      if (r_out) r_out[e] = res;
      acc[r * 3 + 0] = res * res;
      acc[r * 3 + 1] = x[e] * s[r];
      acc[r * 3 + 2] = b[e] * x[e];
    }
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int k = 0; k < nrhs * 3; k++) {
    double v = acc[k];
    for (int m = 16; m >= 1; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
    if (lane == 0) sm[k][w] = v;
  }
  __syncthreads();
  if (threadIdx.x < nrhs * 3) {
    double v = 0.0;
    for (int k = 0; k < kSetupThreads / 32; k++) v += sm[threadIdx.x][k];
    part[(size_t)blockIdx.x * nrhs * 3 + threadIdx.x] = v;
  }
}

// The largest of n non-negative doubles, into *out (which starts at 0): for
// non-negative IEEE-754 values the bit patterns, read as unsigned integers,
// order as the values do, so an integer atomicMax gives the exact maximum.
__global__ void k_max_nonneg(int n, const double* v, unsigned long long* out) {
  unsigned long long m = 0ull;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    m = max(m, (unsigned long long)__double_as_longlong(v[i]));
  for (int k = 16; k >= 1; k >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, k));
  if ((threadIdx.x & 31) == 0 && m > 0ull) atomicMax(out, m);
}

// ||b_r||^2 per right-hand side (b interleaved): per-block partials in
// part[block][nrhs]; *bad = 1 if an entry is not finite.
__global__ void k_bnorm2(int n, int nrhs, const double* b, double* part, int* bad) {
  __shared__ double sm[kMaxRhs][kSetupThreads / 32];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double acc[kMaxRhs] = {0.0, 0.0, 0.0, 0.0};
  if (i < n) {
    for (int r = 0; r < nrhs; r++) {
      const double v = b[(long long)i * nrhs + r];
      if (!isfinite(v)) *bad = 1;
      acc[r] = __dmul_rn(v, v);
    }
  }
  // explicitly rounded operations (no contraction), so that another kernel
  // written with the same operations gives the same bits
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int k = 0; k < nrhs; k++) {
    double v = acc[k];
    for (int m = 16; m >= 1; m >>= 1) v = __dadd_rn(v, __shfl_xor_sync(0xffffffffu, v, m));
    if (lane == 0) sm[k][w] = v;
  }
  __syncthreads();
  if (threadIdx.x < nrhs) {
    double v = 0.0;
    for (int k = 0; k < kSetupThreads / 32; k++) v = __dadd_rn(v, sm[threadIdx.x][k]);
    part[(size_t)blockIdx.x * nrhs + threadIdx.x] = v;
  }
}

// y = D^-1/2 Q D^-1/2 x (rows with zero diagonal give 0); per-block partials
// of <x, y> and <y, y> go to part[block][2].
__global__ void k_normalized_spmv(int n, const int* rp, const int* ci, const double* val,
                                  const double* diag, const double* x, double* y, double* part) {
  __shared__ double sm[2][kSetupThreads / 32];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double xy = 0.0, yy = 0.0;
  if (i < n) {
    const double di = diag[i];
    double s = 0.0;
    if (di > 0.0) {
      for (int q = rp[i]; q < rp[i + 1]; q++) {
        const int c = ci[q];
        const double dc = diag[c];
        if (dc > 0.0) s = fma(val[q] * rsqrt(dc), x[c], s);
      }
      s *= rsqrt(di);
    }
    y[i] = s;
    xy = x[i] * s;
    yy = s * s;
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int m = 16; m >= 1; m >>= 1) {
    xy += __shfl_xor_sync(0xffffffffu, xy, m);
    yy += __shfl_xor_sync(0xffffffffu, yy, m);
  }
  if (lane == 0) { sm[0][w] = xy; sm[1][w] = yy; }
  __syncthreads();
  if (threadIdx.x < 2) {
    double v = 0.0;
    for (int k = 0; k < kSetupThreads / 32; k++) v += sm[threadIdx.x][k];
    part[(size_t)blockIdx.x * 2 + threadIdx.x] = v;
  }
}

// Gershgorin bound of D^-1/2 Q D^-1/2: per-block maxima of sum_j |Q_ij| / sqrt(D_i D_j).
__global__ void k_gershgorin(int n, const int* rp, const int* ci, const double* val,
                             const double* diag, double* part) {
  __shared__ double sm[kSetupThreads / 32];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double g = 0.0;
  if (i < n && diag[i] > 0.0) {
    for (int q = rp[i]; q < rp[i + 1]; q++) {
      const double dc = diag[ci[q]];
      if (dc > 0.0) g += fabs(val[q]) * rsqrt(dc);
    }
    g *= rsqrt(diag[i]);
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int m = 16; m >= 1; m >>= 1) g = fmax(g, __shfl_xor_sync(0xffffffffu, g, m));
  if (lane == 0) sm[w] = g;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int k = 0; k < kSetupThreads / 32; k++) v = fmax(v, sm[k]);
    part[blockIdx.x] = v;
  }
}

__global__ void k_scale(int n, double* x, double s) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] *= s;
}

// SELL-C-sigma fill (C = 32): position p of the sliced order takes the
// entries of row perm[p] in CSR order; entry k goes to sptr[p / 32] + 32 k +
// p % 32.  T is the stored value type of the iteration precision.
template <class T>
__global__ void k_sell_fill(int nsell, int cl, const int* perm, const int* rlen, const int* sptr,
                            const int* rp, const int* ci, const T* val, int* scol, T* sval) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nsell) return;
  const int i = perm[p], len = rlen[p], r0 = rp[i];
  const long long C = 1ll << cl;  // slice height
  const long long base = (long long)sptr[p >> cl] + (p & (C - 1));
  for (int k = 0; k < len; k++) {
    scol[base + C * k] = ci[r0 + k];
    sval[base + C * k] = val[r0 + k];
  }
}

// x += c * d (interleaved, FP64), used by the outer refinement loop; only the
// right-hand sides flagged in mask are updated.
__global__ void k_axpy_masked(long long m, int nrhs, unsigned mask, const double* d, double c,
                              double* x) {
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < m && ((mask >> (e % nrhs)) & 1u)) x[e] += c * d[e];
}

// Longest row of the matrix (atomicMax into *out, which starts at 0).
__global__ void k_max_row_len(int n, const int* rp, int* out) {
  int m = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    m = max(m, rp[i + 1] - rp[i]);
  for (int k = 16; k >= 1; k >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, k));
  if ((threadIdx.x & 31) == 0 && m > 0) atomicMax(out, m);
}

// Eigenvalues of the symmetric m x m matrix B (m <= 8), left on its diagonal:
// cyclic Jacobi rotations (Jacobi 1846; Golub and Van Loan, Matrix
// Computations, Sec. 8.5), each zeroing B_pq by B <- R^T B R with
// tau = (B_qq - B_pp) / (2 B_pq), t = sign(tau) / (|tau| + sqrt(1 + tau^2)),
// c = 1 / sqrt(1 + t^2), s = t c; until the off-diagonal mass is below 1e-32
// of the total (at most 60 sweeps).
__device__ void jb_jacobi_eig(double (&B)[8][8], int m) {
  for (int sw = 0; sw < 60; sw++) {
    double off = 0.0, tot = 0.0;
    for (int p = 0; p < m; p++)
      for (int q = 0; q < m; q++) {
        const double v = B[p][q] * B[p][q];
        tot += v;
        if (p != q) off += v;
      }
    if (off <= 1e-32 * tot) return;
    for (int p = 0; p < m; p++)
      for (int q = p + 1; q < m; q++) {
        const double bpq = B[p][q];
        if (bpq == 0.0) continue;
        const double tau = (B[q][q] - B[p][p]) / (2.0 * bpq);
        const double t = fabs(tau) > 1e100 ? 0.5 / tau
                                           : (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        const double c = 1.0 / sqrt(1.0 + t * t), sn = t * c;
        for (int k = 0; k < m; k++) {
          const double bkp = B[k][p], bkq = B[k][q];
          B[k][p] = c * bkp - sn * bkq;
          B[k][q] = sn * bkp + c * bkq;
        }
        for (int k = 0; k < m; k++) {
          const double bpk = B[p][k], bqk = B[q][k];
          B[p][k] = c * bpk - sn * bqk;
          B[q][k] = sn * bpk + c * bqk;
        }
      }
  }
}

// eq. J-blkdiag for blocks of bs consecutive rows (bs <= 8), one thread per
// block ib (rows r0 .. r0 + nb - 1):
//   J = Q^{ib,ib} + (sum over column blocks jb != ib, ascending, ||Q^{ib,jb}||_2) I,
// ||A||_2 = sqrt(lambda_max(A^T A)).  A block whose J has its smallest
// eigenvalue at most 1e-12 of its largest diagonal entry (a singular part of
// Q wholly inside the block, with no coupling) takes eq. J-diag's diagonal,
// whose inverse jd holds.  Row k of J^{-1} (by the Cholesky factor J = L L^T:
// column m of J^{-1} solves L y = e_m, L^T z = y) goes to out[(r0 + k) bs + m];
// the last block's rows beyond n get identity rows.  *bad = 1 if J is not
// positive definite.
__global__ void k_jblk(int n, int bs, const int* rp, const int* ci, const double* val, const double* jd,
                       double* out, int* bad) {
  const long long nblk = ((long long)n + bs - 1) / bs;
  for (long long ib = (long long)blockIdx.x * blockDim.x + threadIdx.x; ib < nblk;
       ib += (long long)gridDim.x * blockDim.x) {
    const int r0 = (int)(ib * bs);
    const int nb = min(bs, n - r0);
    double J[8][8], A[8][8];
    for (int k = 0; k < 8; k++)
      for (int m = 0; m < 8; m++) J[k][m] = 0.0;
    for (int k = 0; k < nb; k++)
      for (int q = rp[r0 + k]; q < rp[r0 + k + 1]; q++)
        if (ci[q] / bs == ib) J[k][ci[q] - r0] += val[q];
    double csum = 0.0;
    long long prev = -1;
    for (;;) {
      long long nxt = LLONG_MAX;
      for (int k = 0; k < nb; k++)
        for (int q = rp[r0 + k]; q < rp[r0 + k + 1]; q++) {
          const long long jb = ci[q] / bs;
          if (jb != ib && jb > prev && jb < nxt) nxt = jb;
        }
      if (nxt == LLONG_MAX) break;
      for (int k = 0; k < 8; k++)
        for (int m = 0; m < 8; m++) A[k][m] = 0.0;
      for (int k = 0; k < nb; k++)
        for (int q = rp[r0 + k]; q < rp[r0 + k + 1]; q++)
          if (ci[q] / bs == nxt) A[k][ci[q] - (int)(nxt * bs)] += val[q];
      double B[8][8];
      for (int p = 0; p < 8; p++)
        for (int m = 0; m < 8; m++) {
          double v = 0.0;
          for (int k = 0; k < nb; k++) v += A[k][p] * A[k][m];
          B[p][m] = v;
        }
      jb_jacobi_eig(B, bs);
      double lmax = 0.0;
      for (int p = 0; p < bs; p++) lmax = fmax(lmax, B[p][p]);
      csum += sqrt(lmax);
      prev = nxt;
    }
    for (int k = 0; k < nb; k++) J[k][k] += csum;
    // singular J: eq. J-diag for this block
    double E[8][8], dmax = 0.0;
    for (int k = 0; k < 8; k++)
      for (int m = 0; m < 8; m++) E[k][m] = J[k][m];
    for (int k = 0; k < nb; k++) dmax = fmax(dmax, J[k][k]);
    jb_jacobi_eig(E, nb);
    double lmin = 1e300;
    for (int k = 0; k < nb; k++) lmin = fmin(lmin, E[k][k]);
    double* o = out + (size_t)r0 * bs;
    if (!(lmin > 1e-12 * dmax)) {
      for (int k = 0; k < bs; k++)
        for (int m = 0; m < bs; m++) o[k * bs + m] = (k == m) ? (k < nb ? jd[r0 + k] : 1.0) : 0.0;
      continue;
    }
    // Cholesky J = L L^T (rows k >= nb are left out), then the columns of J^{-1}
    double L[8][8];
    bool ok = true;
    for (int j = 0; j < nb && ok; j++) {
      double d = J[j][j];
      for (int k = 0; k < j; k++) d -= L[j][k] * L[j][k];
      ok = d > 0.0;
      if (!ok) break;
      L[j][j] = sqrt(d);
      for (int i = j + 1; i < nb; i++) {
        double v = J[i][j];
        for (int k = 0; k < j; k++) v -= L[i][k] * L[j][k];
        L[i][j] = v / L[j][j];
      }
    }
    if (!ok) {
      *bad = 1;
      continue;
    }
    for (int mcol = 0; mcol < bs; mcol++) {
      double z[8];
      for (int i = 0; i < nb; i++) {
        double v = (i == mcol) ? 1.0 : 0.0;
        for (int k = 0; k < i; k++) v -= L[i][k] * z[k];
        z[i] = v / L[i][i];
      }
      for (int i = nb - 1; i >= 0; i--) {
        double v = z[i];
        for (int k = i + 1; k < nb; k++) v -= L[k][i] * z[k];
        z[i] = v / L[i][i];
      }
      for (int k = 0; k < bs; k++)
        o[k * bs + mcol] = k < nb ? (mcol < nb ? z[k] : 0.0) : (k == mcol ? 1.0 : 0.0);
    }
  }
}

// Whether Q is a constant-coefficient (2*dim+1)-point stencil on an N^dim grid
// with Dirichlet boundary, rows in natural order (i = x + N*y + N^2*z): every
// row holds exactly its in-grid neighbours, columns ascending, the diagonal
// entry bitwise equal to d and every other entry bitwise equal to o.  Sets
// *bad on any row that differs.
__global__ void k_check_stencil(int n, int N, int dim, const int* rp, const int* ci, const double* val,
                                double d, double o, int* bad) {
  const long long d_bits = __double_as_longlong(d), o_bits = __double_as_longlong(o);
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)t;
    const int NN = dim == 3 ? N * N : 0;
    const int ix = i % N, iy = (i / N) % N, iz = dim == 3 ? i / NN : 0;
    const bool in[7] = {dim == 3 && iz > 0, iy > 0, ix > 0, true, ix < N - 1, iy < N - 1, dim == 3 && iz < N - 1};
    const int cc[7] = {i - NN, i - N, i - 1, i, i + 1, i + N, i + NN};
    int q = rp[i];
    const int qe = rp[i + 1];
    bool ok = true;
    for (int k = 0; k < 7 && ok; k++) {
      if (!in[k]) continue;
      ok = q < qe && ci[q] == cc[k] && __double_as_longlong(val[q]) == (k == 3 ? d_bits : o_bits);
      q++;
    }
    if (!ok || q != qe) *bad = 1;
  }
}

// Summed row spans (largest minus smallest column of each row): per-block
// partial sums in part[block] (FP64, exact for spans below 2^53).
__global__ void k_row_spans(int n, const int* rp, const int* ci, double* part) {
  __shared__ double sm[kSetupThreads / 32];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double v = 0.0;
  if (i < n) {
    int lo = 0x7fffffff, hi = -1;
    for (int q = rp[i]; q < rp[i + 1]; q++) {
      lo = min(lo, ci[q]);
      hi = max(hi, ci[q]);
    }
    if (hi >= lo) v = (double)(hi - lo);
  }
  for (int m = 16; m >= 1; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < kSetupThreads / 32; k++) t += sm[k];
    part[blockIdx.x] = t;
  }
}

// The long rows of the FP64 residual: one warp per row (lanes stride over the
// entries, a fixed xor tree), eight rows per block, block partials of the same
// three sums as k_residual in part[block][nrhs][3].
__global__ void k_residual_long(int nlong, const int* rows, int nrhs, const int* rp, const int* ci,
                                const double* val, const double* b, const double* x, double* r_out,
                                double* part) {
  __shared__ double sm[kMaxRhs * 3][kSetupThreads / 32];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j = blockIdx.x * (kSetupThreads / 32) + w;
  double acc[kMaxRhs * 3];
  for (int k = 0; k < kMaxRhs * 3; k++) acc[k] = 0.0;
  if (j < nlong) {
    const int i = rows[j];
    double s[kMaxRhs] = {0.0, 0.0, 0.0, 0.0};
    for (int q = rp[i] + lane; q < rp[i + 1]; q += 32) {
      const double v = val[q];
      const long long c = ci[q];
      for (int r = 0; r < nrhs; r++) s[r] = fma(v, x[c * nrhs + r], s[r]);
    }
    for (int r = 0; r < nrhs; r++)
      for (int m = 16; m >= 1; m >>= 1) s[r] += __shfl_xor_sync(0xffffffffu, s[r], m);
    if (lane == 0)
      for (int r = 0; r < nrhs; r++) {
        const long long e = (long long)i * nrhs + r;
        const double res = b[e] - s[r];
        if (r_out) r_out[e] = res;
        acc[r * 3 + 0] = res * res;
        acc[r * 3 + 1] = x[e] * s[r];
        acc[r * 3 + 2] = b[e] * x[e];
      }
  }
  if (lane == 0)
    for (int k = 0; k < nrhs * 3; k++) sm[k][w] = acc[k];
  __syncthreads();
  if (threadIdx.x < nrhs * 3) {
    double v = 0.0;
    for (int k = 0; k < kSetupThreads / 32; k++) v += sm[threadIdx.x][k];
    part[(size_t)blockIdx.x * nrhs * 3 + threadIdx.x] = v;
  }
}

// Locality ordering.  New row i is old row perm[i]: its entries keep their
// original order (so every row sums exactly as before) and their columns are
// renamed through iperm (old -> new).  One warp per row.
__global__ void k_permute_csr(int n, const int* perm, const int* iperm, const int* rp0, const int* ci0,
                              const double* val0, const int* rp1, int* ci1, double* val1) {
  const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= n) return;
  const int i = (int)w, o = perm[i];
  const int s0 = rp0[o], len = rp0[o + 1] - s0, s1 = rp1[i];
  for (int k = lane; k < len; k += 32) {
    ci1[s1 + k] = iperm[ci0[s0 + k]];
    val1[s1 + k] = val0[s0 + k];
  }
}
// dst[i * nrhs + r] = src[perm[i] * nrhs + r]: an interleaved vector (or, with
// nrhs = 1, a per-row array) into the new order.
__global__ void k_gather_rows(int n, int nrhs, const int* perm, const double* src, double* dst) {
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)n * nrhs) return;
  const int r = (int)(e % nrhs);
  const long long i = e / nrhs;
  dst[e] = src[(long long)perm[i] * nrhs + r];
}
// cm[r * n + perm[i]] = il[i * nrhs + r]: an interleaved vector in the new
// order back to the caller's column-major layout and row order.
__global__ void k_unpermute_deinterleave(int n, int nrhs, const int* perm, const double* il, double* cm) {
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)n * nrhs) return;
  const int r = (int)(e % nrhs);
  const long long i = e / nrhs;
  cm[(long long)r * n + perm[i]] = il[e];
}

}  // namespace aj
