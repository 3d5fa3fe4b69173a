/*
 * aj_oracle.c -- plain, slow, single-threaded FP64 CPU oracle for the
 * accelerated Jacobi (AJ) method of Liang, Pang, Toh and Yang,
 * "Nesterov's Accelerated Jacobi-Type Methods for Large-scale SPSD Linear
 * Systems" (arXiv 2407.03272).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this file's library.  It shares no
 * code, header or constant with the CUDA library: it is written straight
 * from the paper so that the CUDA path can be checked against it.
 *
 * Every loop runs in index order; every row sum runs in ascending column
 * order as the CSR arrays hold it.  No blocking, no fusion, no reordering.
 * The baseline timing build (oracle/build.py, -fopenmp) spreads the loops
 * whose iterations are independent -- the rows of a product, element-wise
 * vector updates -- over threads (the OMP lines below; the correctness
 * build ignores them); every sum, a row's or a dot product's, still runs in
 * index order in one thread, so both builds give the same bits.
 *
 *   orc_spmv          out = Q y                          (the product in Alg. 3, step "x^t = ...")
 *   orc_j_absrowsum   J_kk = Q_kk + sum_{j!=k} |Q_kj|     (eq. J-diag, Section 3)
 *   orc_j_scaled_diag J_kk = c * Q_kk                      (c = L gives S = L*D - Q >= 0 when
 *                                                          L >= lambda_max(D^-1/2 Q D^-1/2);
 *                                                          c = 1/omega gives weighted Jacobi, eq. weighted-jacobi)
 *   orc_aj_solve      Algorithm alg-jacobi with the restart rule of Algorithm alg-apg-re
 *                     (Section 2.2) and, when is_restart = 0, plain Algorithm alg-apg.
 *                     J is diagonal (eq. J-diag and variants) or block diagonal
 *                     (eq. J-blkdiag, blocks given by the caller); a block update
 *                     x^i = y^i - (J^{ii})^{-1} g^i solves with the block's Cholesky factor.
 *   orc_pcg_solve     the comparator: conjugate gradients with the diagonal preconditioner
 *                     (Section 4.2), Saad's Alg. 9.1.
 *                     momentum = 0 replaces the alpha/beta extrapolation by beta = 0, which with
 *                     J = D / omega is the (weighted) Jacobi method of eqs. jacobi / weighted-jacobi.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Independent iterations over threads in the -fopenmp timing build only. */
#ifdef _OPENMP
#define OMP_ROWS _Pragma("omp parallel for schedule(static)")
#else
#define OMP_ROWS
#endif

/* out_i = sum_j Q_ij y_j, j in CSR order (ascending column). */
void orc_spmv(int64_t n, const int32_t* row_ptr, const int32_t* col,
              const double* val, const double* y, double* out) {
  OMP_ROWS
  for (int64_t i = 0; i < n; i++) {
    double s = 0.0;
    for (int32_t p = row_ptr[i]; p < row_ptr[i + 1]; p++) s += val[p] * y[col[p]];
    out[i] = s;
  }
}

/* eq. J-diag: J_kk = Q_kk + sum_{j != k} |Q_kj|.  A row with no nonzero entry
 * gets J_kk = 1 (the paper assumes no zero row; J = 1 keeps J invertible and
 * S = J - Q positive semidefinite there). */
void orc_j_absrowsum(int64_t n, const int32_t* row_ptr, const int32_t* col,
                     const double* val, double* J) {
  for (int64_t k = 0; k < n; k++) {
    double diag = 0.0, off = 0.0;
    for (int32_t p = row_ptr[k]; p < row_ptr[k + 1]; p++) {
      if (col[p] == k) diag += val[p];
      else off += fabs(val[p]);
    }
    double jk = diag + off;
    J[k] = (jk == 0.0) ? 1.0 : jk;
  }
}

/* J_kk = c * Q_kk; zero diagonal (an all-zero row of an SPSD matrix) -> 1. */
void orc_j_scaled_diag(int64_t n, const int32_t* row_ptr, const int32_t* col,
                       const double* val, double c, double* J) {
  for (int64_t k = 0; k < n; k++) {
    double diag = 0.0;
    for (int32_t p = row_ptr[k]; p < row_ptr[k + 1]; p++)
      if (col[p] == k) diag += val[p];
    double jk = c * diag;
    J[k] = (jk == 0.0) ? 1.0 : jk;
  }
}

static double dot(int64_t n, const double* a, const double* b) {
  double s = 0.0;
  for (int64_t i = 0; i < n; i++) s += a[i] * b[i];
  return s;
}

/* Stop kinds. */
#define ORC_STOP_NONE 0   /* run exactly maxit iterations */
#define ORC_STOP_RELRES 1 /* ||b - Q x^t||_2 / ||b||_2 <= tol   (||b|| = 0: absolute) */
#define ORC_STOP_OBJGAP 2 /* |f(x^t) - f*| / (1 + |f*|) <= tol  (Section 4 stopping rule) */

typedef struct {
  int64_t n;
  const int32_t* row_ptr;
  const int32_t* col;
  const double* val;
  const double* b;
  const double* J;      /* diagonal of J, length n (from orc_j_*) */
  const double* x0;     /* NULL: x^0 = 0 */
  int is_restart;       /* IsRestart of Algorithm alg-jacobi */
  int momentum;         /* 1: Nesterov alpha recurrence; 0: beta = 0 (Jacobi-type comparator) */
  int64_t K0;           /* K_0 >= 2 */
  int64_t maxit;
  int stop;             /* ORC_STOP_* */
  double tol;
  double fstar;
  const uint8_t* forced; /* optional, length maxit + 1: restart at t iff forced[t] (replay) */
  int64_t bs;           /* block size of Jblk */
  const double* Jblk;   /* optional block-diagonal J (replaces J): s = ceil(n / bs) blocks
                           J^{ii}, each bs x bs row-major; the last block's rows and
                           columns beyond n are ignored */
} orc_params;

typedef struct {
  int64_t iters;     /* t of the returned x^t */
  int64_t restarts;  /* ell */
  double relres;     /* ||b - Q x^t|| / ||b|| of the returned iterate */
  double f;          /* f(x^t) = 1/2 <x, Qx> - <b, x> */
  int converged;     /* stop test met (always 0 for ORC_STOP_NONE) */
} orc_info;

/* Per-iteration trace (all optional, each of length maxit + 1, index t):
 *   tr_alpha[t]   alpha_t as used by the momentum step of iteration t
 *   tr_beta[t]    the extrapolation coefficient used to form y^{t+1} (0 on restart)
 *   tr_d[t]       <Q y^t - b, x^t - x^{t-1}> with x^t before the restart branch
 *   tr_restart[t] 1 if iteration t restarted
 *   tr_f[t]       f(x^t) after the branch (t = 0: f(x^0))
 *   tr_relres[t]  relative residual of x^t after the branch
 *   tr_gnorm[t]   ||Q y^t - b||_2
 *   tr_gfloor[t]  || |Q| |y^t| + |b| ||_2: the scale of the rounding error in Q y^t - b (a
 *                 row sum of k terms in unit roundoff u errs by at most about k u times
 *                 that row's entry)
 *   tr_dxnorm[t]  ||x^t - x^{t-1}||_2 with x^t before the restart branch (the scale of the
 *                 restart test: |d| <= ||Q y^t - b|| ||x^t - x^{t-1}|| by Cauchy-Schwarz)
 *   tr_x          (maxit + 1) x n: x^t after the branch, row t
 *   tr_y          (maxit + 1) x n: y^t, row t (row 0 unused)
 */
typedef struct {
  double* alpha;
  double* beta;
  double* d;
  uint8_t* restart;
  double* f;
  double* relres;
  double* gnorm;
  double* x;
  double* y;
  double* dxnorm;
  double* gfloor;
} orc_trace;

static void eval_x(const orc_params* P, const double* x, double* qx, double bnorm,
                   double* relres, double* f) {
  int64_t n = P->n;
  orc_spmv(n, P->row_ptr, P->col, P->val, x, qx);
  double rr = 0.0;
  for (int64_t i = 0; i < n; i++) {
    double r = P->b[i] - qx[i];
    rr += r * r;
  }
  *relres = (bnorm > 0.0) ? sqrt(rr) / bnorm : sqrt(rr);
  *f = 0.5 * dot(n, x, qx) - dot(n, P->b, x);
}

static int stop_met(const orc_params* P, double relres, double f) {
  if (P->stop == ORC_STOP_RELRES) return relres <= P->tol;
  if (P->stop == ORC_STOP_OBJGAP) return fabs(f - P->fstar) / (1.0 + fabs(P->fstar)) <= P->tol;
  return 0;
}

/* Cholesky factor (lower triangular, row-major, m x m with leading
 * dimension ld) of the symmetric m x m matrix A, in place of L:
 *   L_jj = sqrt(A_jj - sum_{k<j} L_jk^2),  L_ij = (A_ij - sum_{k<j} L_ik L_jk) / L_jj.
 * Returns -1 if a pivot is not positive. */
static int cholesky(int64_t m, int64_t ld, const double* A, double* L) {
  for (int64_t i = 0; i < m; i++)
    for (int64_t j = 0; j < m; j++) L[i * ld + j] = 0.0;
  for (int64_t j = 0; j < m; j++) {
    double d = A[j * ld + j];
    for (int64_t k = 0; k < j; k++) d -= L[j * ld + k] * L[j * ld + k];
    if (!(d > 0.0)) return -1;
    L[j * ld + j] = sqrt(d);
    for (int64_t i = j + 1; i < m; i++) {
      double v = A[i * ld + j];
      for (int64_t k = 0; k < j; k++) v -= L[i * ld + k] * L[j * ld + k];
      L[i * ld + j] = v / L[j * ld + j];
    }
  }
  return 0;
}

/* z = (L L^T)^{-1} r: forward substitution L w = r, then back substitution L^T z = w. */
static void chol_solve(int64_t m, int64_t ld, const double* L, const double* r, double* z) {
  for (int64_t i = 0; i < m; i++) {
    double v = r[i];
    for (int64_t k = 0; k < i; k++) v -= L[i * ld + k] * z[k];
    z[i] = v / L[i * ld + i];
  }
  for (int64_t i = m - 1; i >= 0; i--) {
    double v = z[i];
    for (int64_t k = i + 1; k < m; k++) v -= L[k * ld + i] * z[k];
    z[i] = v / L[i * ld + i];
  }
}

/* Algorithm alg-jacobi (Section 3) with diagonal J:
 *   x^t = y^t + J^{-1}(b - Q y^t)
 *   restart if IsRestart and t > K_re + K_ell and <Q y^t - b, x^t - x^{t-1}> >= 0:
 *       K_re = t, K_{ell+1} = 2 K_ell, ell += 1, alpha_{t+1} = 1, alpha_t = 0,
 *       y^{t+1} = x^{t-1}, x^t = x^{t-1}
 *   else alpha_{t+1} = (1 + sqrt(1 + 4 alpha_t^2)) / 2,
 *       y^{t+1} = x^t + ((alpha_t - 1) / alpha_{t+1}) (x^t - x^{t-1})
 * with x^0 = y^1, alpha_0 = 0, alpha_1 = 1.  Returns 0, or -1 on bad input / no memory. */
int orc_aj_solve(const orc_params* P, double* x_out, orc_info* info, const orc_trace* T) {
  int64_t n = P->n;
  if (n < 0 || P->K0 < 2 || P->maxit < 0) return -1;
  double* xprev = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double)); /* x^{t-1} */
  double* x = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));     /* x^t */
  double* y = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));     /* y^t */
  double* g = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));     /* Q y^t - b */
  double* qx = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
  if (!xprev || !x || !y || !g || !qx) {
    free(xprev); free(x); free(y); free(g); free(qx);
    return -1;
  }
  /* block-diagonal J: the Cholesky factor of every block, once */
  double* Lf = NULL;
  double* zb = NULL;
  const int64_t bs = P->bs;
  if (P->Jblk) {
    const int64_t s = bs > 0 ? (n + bs - 1) / bs : 0;
    Lf = (double*)calloc((size_t)(s > 0 ? s : 1) * (size_t)(bs > 0 ? bs * bs : 1), sizeof(double));
    zb = (double*)calloc((size_t)(bs > 0 ? bs : 1), sizeof(double));
    int bad = bs < 1 || !Lf || !zb;
    for (int64_t ib = 0; ib < s && !bad; ib++) {
      const int64_t nb = (n - ib * bs < bs) ? n - ib * bs : bs;
      bad = cholesky(nb, bs, P->Jblk + ib * bs * bs, Lf + ib * bs * bs) != 0;
    }
    if (bad) {
      free(xprev); free(x); free(y); free(g); free(qx); free(Lf); free(zb);
      return -1;
    }
  }
  if (P->x0)
    for (int64_t i = 0; i < n; i++) xprev[i] = P->x0[i];
  OMP_ROWS
  for (int64_t i = 0; i < n; i++) { x[i] = xprev[i]; y[i] = xprev[i]; }

  double bnorm = sqrt(dot(n, P->b, P->b));
  double alpha = 1.0; /* alpha_1 (alpha_0 = 0 is never read again) */
  int64_t ell = 0, K = P->K0, Kre = 0;
  double relres, f;
  eval_x(P, x, qx, bnorm, &relres, &f);
  if (T && T->f) T->f[0] = f;
  if (T && T->relres) T->relres[0] = relres;
  if (T && T->x) memcpy(T->x, x, (size_t)n * sizeof(double));
  int64_t t = 0;
  int conv = stop_met(P, relres, f);
  while (!conv && t < P->maxit) {
    t++;
    if (T && T->y) memcpy(T->y + (size_t)t * n, y, (size_t)n * sizeof(double));
    /* g = Q y^t - b */
    orc_spmv(n, P->row_ptr, P->col, P->val, y, g);
    OMP_ROWS
    for (int64_t i = 0; i < n; i++) g[i] -= P->b[i];
    double gfl = 0.0; /* trace only: || |Q| |y^t| + |b| || */
    if (T && T->gfloor) {
      for (int64_t i = 0; i < n; i++) {
        double s = fabs(P->b[i]);
        for (int32_t p = P->row_ptr[i]; p < P->row_ptr[i + 1]; p++) s += fabs(P->val[p]) * fabs(y[P->col[p]]);
        gfl += s * s;
      }
      gfl = sqrt(gfl);
    }
    /* x^t = y^t + J^{-1}(b - Q y^t) = y^t - J^{-1} g */
    if (P->Jblk) {
      for (int64_t r0 = 0; r0 < n; r0 += bs) {
        const int64_t nb = (n - r0 < bs) ? n - r0 : bs;
        chol_solve(nb, bs, Lf + (r0 / bs) * bs * bs, g + r0, zb);
        for (int64_t k = 0; k < nb; k++) x[r0 + k] = y[r0 + k] - zb[k];
      }
    } else {
      OMP_ROWS
      for (int64_t i = 0; i < n; i++) x[i] = y[i] - g[i] / P->J[i];
    }
    /* restart test quantity <Q y^t - b, x^t - x^{t-1}> */
    double d = 0.0, gg = 0.0, dd = 0.0;
    for (int64_t i = 0; i < n; i++) {
      d += g[i] * (x[i] - xprev[i]);
      gg += g[i] * g[i];
      dd += (x[i] - xprev[i]) * (x[i] - xprev[i]);
    }
    int restart;
    if (P->forced) restart = P->forced[t] != 0;
    else restart = P->is_restart && (t > Kre + K) && (d >= 0.0);
    double alpha_next, beta;
    if (restart) {
      Kre = t;
      K = 2 * K;
      ell++;
      OMP_ROWS
      for (int64_t i = 0; i < n; i++) { x[i] = xprev[i]; y[i] = xprev[i]; }
      alpha_next = 1.0; /* alpha_{t+1} = 1, alpha_t = 0 */
      beta = 0.0;
    } else {
      if (P->momentum) {
        alpha_next = (1.0 + sqrt(1.0 + 4.0 * alpha * alpha)) / 2.0;
        beta = (alpha - 1.0) / alpha_next;
      } else {
        alpha_next = 1.0;
        beta = 0.0;
      }
      OMP_ROWS
      for (int64_t i = 0; i < n; i++) {
        y[i] = x[i] + beta * (x[i] - xprev[i]);
        xprev[i] = x[i];
      }
    }
    if (T && T->alpha) T->alpha[t] = alpha;
    if (T && T->beta) T->beta[t] = beta;
    if (T && T->d) T->d[t] = d;
    if (T && T->restart) T->restart[t] = (uint8_t)restart;
    if (T && T->gnorm) T->gnorm[t] = sqrt(gg);
    if (T && T->dxnorm) T->dxnorm[t] = sqrt(dd);
    if (T && T->gfloor) T->gfloor[t] = gfl;
    alpha = alpha_next;
    eval_x(P, x, qx, bnorm, &relres, &f);
    if (T && T->f) T->f[t] = f;
    if (T && T->relres) T->relres[t] = relres;
    if (T && T->x) memcpy(T->x + (size_t)t * n, x, (size_t)n * sizeof(double));
    conv = stop_met(P, relres, f);
  }
  memcpy(x_out, x, (size_t)n * sizeof(double));
  if (info) {
    info->iters = t;
    info->restarts = ell;
    info->relres = relres;
    info->f = f;
    info->converged = conv;
  }
  free(xprev); free(x); free(y); free(g); free(qx); free(Lf); free(zb);
  return 0;
}

/* Preconditioned conjugate gradients with the diagonal preconditioner
 * M = diag(Q) (a zero diagonal entry -> 1), the paper's main comparator
 * (Section 4.2, "PCG with a simple diagonal preconditioner"); the recurrence
 * of Saad, Iterative Methods for Sparse Linear Systems, Alg. 9.1:
 *   r^0 = b - Q x^0, z^0 = M^{-1} r^0, p^0 = z^0;
 *   alpha_t = <r^t, z^t> / <Q p^t, p^t>;  x^{t+1} = x^t + alpha_t p^t;
 *   r^{t+1} = r^t - alpha_t Q p^t;  z^{t+1} = M^{-1} r^{t+1};
 *   beta_t = <r^{t+1}, z^{t+1}> / <r^t, z^t>;  p^{t+1} = z^{t+1} + beta_t p^t.
 * Stops before iteration t when ||r^t||_2 <= tol ||b||_2 (the recursive
 * residual) or t = maxit.  x0 may be NULL (x^0 = 0).  rr_trace (optional,
 * length maxit + 1) receives ||r^t||_2.  Returns 0, or -1 on no memory. */
int orc_pcg_solve(int64_t n, const int32_t* row_ptr, const int32_t* col, const double* val,
                  const double* b, const double* x0, int64_t maxit, double tol, double* x_out,
                  int64_t* iters_out, double* rr_trace) {
  size_t m = (size_t)(n > 0 ? n : 1);
  double* x = (double*)calloc(m, sizeof(double));
  double* r = (double*)calloc(m, sizeof(double));
  double* z = (double*)calloc(m, sizeof(double));
  double* p = (double*)calloc(m, sizeof(double));
  double* q = (double*)calloc(m, sizeof(double));
  double* dinv = (double*)calloc(m, sizeof(double));
  if (!x || !r || !z || !p || !q || !dinv) {
    free(x); free(r); free(z); free(p); free(q); free(dinv);
    return -1;
  }
  for (int64_t k = 0; k < n; k++) {
    double d = 0.0;
    for (int32_t e = row_ptr[k]; e < row_ptr[k + 1]; e++)
      if (col[e] == k) d += val[e];
    dinv[k] = 1.0 / (d == 0.0 ? 1.0 : d);
  }
  if (x0)
    for (int64_t i = 0; i < n; i++) x[i] = x0[i];
  orc_spmv(n, row_ptr, col, val, x, q);
  for (int64_t i = 0; i < n; i++) {
    r[i] = b[i] - q[i];
    z[i] = dinv[i] * r[i];
    p[i] = z[i];
  }
  double rz = dot(n, r, z);
  const double bnorm = sqrt(dot(n, b, b));
  int64_t t = 0;
  double rn = sqrt(dot(n, r, r));
  if (rr_trace) rr_trace[0] = rn;
  while (t < maxit && !(rn <= tol * bnorm)) {
    orc_spmv(n, row_ptr, col, val, p, q);
    const double alpha = rz / dot(n, p, q);
    for (int64_t i = 0; i < n; i++) {
      x[i] += alpha * p[i];
      r[i] -= alpha * q[i];
      z[i] = dinv[i] * r[i];
    }
    const double rz_new = dot(n, r, z);
    const double beta = rz_new / rz;
    rz = rz_new;
    for (int64_t i = 0; i < n; i++) p[i] = z[i] + beta * p[i];
    t++;
    rn = sqrt(dot(n, r, r));
    if (rr_trace) rr_trace[t] = rn;
  }
  memcpy(x_out, x, (size_t)n * sizeof(double));
  if (iters_out) *iters_out = t;
  free(x); free(r); free(z); free(p); free(q); free(dinv);
  return 0;
}
