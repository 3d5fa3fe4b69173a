/*
 * aj.h -- C ABI of libaj, a GB300 (sm_103a) solver for Q x = b with sparse
 * symmetric positive semidefinite Q by the Nesterov-accelerated, adaptively
 * restarted Jacobi method of Liang, Pang, Toh and Yang (arXiv 2407.03272).
 *
 * The problem (Section 1, eqs. linear-sys and qp): Q x = b with Q SPSD and
 * b in range(Q), equivalently min f(x) = 1/2 <x, Qx> - <b, x>.
 *
 * The iteration (Algorithm alg-jacobi, Section 3, with the restart rule of
 * Algorithm alg-apg-re, Section 2.2), t = 1, 2, ...:
 *     x^t = y^t + J^{-1} (b - Q y^t)                       (J diagonal)
 *     if IsRestart and t > K_re + K_l and <Q y^t - b, x^t - x^{t-1}> >= 0:
 *         K_re = t, K_{l+1} = 2 K_l, l = l + 1, alpha_{t+1} = 1,
 *         y^{t+1} = x^t = x^{t-1}
 *     else:
 *         alpha_{t+1} = (1 + sqrt(1 + 4 alpha_t^2)) / 2
 *         y^{t+1} = x^t + ((alpha_t - 1) / alpha_{t+1}) (x^t - x^{t-1})
 * with x^0 = y^1, alpha_1 = 1.  One iteration is one fused HBM sweep on the
 * GPU: SpMV at y, J^{-1} scaling, x update, momentum extrapolation and the
 * FP64 restart/stop reductions in one persistent grid-synchronised kernel.
 *
 * Conventions for every entry point:
 *   - Return value: AJ_OK (0), a negative AJ_E* error, or AJ_PENDING (> 0,
 *     aj_poll only).  The library never aborts or exits; device-side failures
 *     (non-finite reductions, barrier timeouts) come back as status codes.
 *   - Pointers named *_on_device / on_device = 1 are CUDA device pointers of
 *     the current device; otherwise host pointers.  The caller owns every
 *     pointer it passes; the library copies what it keeps and never touches
 *     caller memory after the call returns.
 *   - Sizes are element counts unless the name says bytes.
 *   - Calls on one aj_ctx are not thread-safe; different contexts are
 *     independent.  All GPU work of a context runs on its stream
 *     (aj_set_stream; default: the legacy default stream) and every call
 *     returns only after that work has finished.
 */
#ifndef AJ_H
#define AJ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int aj_status;
#define AJ_OK 0
#define AJ_EINVAL (-1)     /* bad argument or input that is not a valid SPSD CSR matrix */
#define AJ_ENOMEM (-2)     /* device or host allocation failed, or over the memory budget */
#define AJ_ECUDA (-3)      /* a CUDA runtime call failed */
#define AJ_EMAXIT (-4)     /* maxit reached before the stop test held (x is still returned) */
#define AJ_EDIVERGED (-5)  /* residual grew by > 1e8 over its starting value: S = J - Q not PSD */
#define AJ_ENONFINITE (-6) /* a reduction became NaN or Inf */
#define AJ_ETIMEOUT (-7)   /* a device-side grid barrier gave up waiting */
#define AJ_EBUSY (-8)      /* a request can never be admitted (larger than the budget) */
#define AJ_PENDING 1       /* aj_poll: the request has not finished yet */

typedef struct aj_ctx aj_ctx;
typedef struct aj_server aj_server;

/* A square CSR matrix Q (n x n) with int32 indices, FP64 values.
 * row_ptr[0] = 0, row_ptr non-decreasing, row_ptr[n] = nnz, 0 <= col < n.
 * Column order within a row is free (duplicates are summed).  Every row
 * either has a positive diagonal entry or is entirely zero (an isolated
 * vertex of a graph Laplacian); a zero row gets J_kk = 1 (Section 3 assumes
 * no zero row; J = 1 keeps J invertible and S = J - Q PSD there). */
typedef struct {
  int64_t n;
  int64_t nnz;
  const int32_t* row_ptr;
  const int32_t* col;
  const double* val;
  int on_device; /* 1: the three arrays (and b in aj_create) are device pointers */
} aj_csr;

/* Choice of the proximal matrix J (S = J - Q must be PSD). */
#define AJ_J_ABSROWSUM 0   /* eq. J-diag: J_kk = Q_kk + sum_{j != k} |Q_kj| (the paper's default) */
#define AJ_J_SCALED_DIAG 1 /* J = L D with L >= lambda_max(D^-1/2 Q D^-1/2) (Remark remark-preconditioner) */
/* eq. J-blkdiag (Sec. 3): J = diag(J^{1,1}, ..., J^{s,s}) over blocks of
 * j_block consecutive rows (2, 4 or 8; 1 is eq. J-diag), J^{ii} = Q^{ii} +
 * (sum_{j != i} ||Q^{ij}||_2) I with each spectral norm computed exactly (up
 * to rounding) at aj_set.  A block whose J^{ii} is singular (a singular part
 * of Q wholly inside the block with no coupling, such as a small component
 * of a graph Laplacian) takes eq. J-diag's diagonal, which keeps J
 * invertible and S PSD.  The sweep applies each block's inverse: j_block
 * n-vectors of J^{-1} per sweep instead of one.  Needs CSR or STENCIL
 * storage in the caller's row order (AJ_EINVAL with AJ_FMT_SELL or
 * AJ_REORDER_RCM; AUTO choices avoid both) and rows of at most 1024 entries. */
#define AJ_J_BLKDIAG 2

#define AJ_RESTART_NONE 0     /* Algorithm alg-apg: no restart (IsRestart = False) */
#define AJ_RESTART_ADAPTIVE 1 /* Algorithm alg-apg-re restart rule (IsRestart = True) */

#define AJ_STOP_RELRES 0 /* ||b - Q x^t||_2 <= tol ||b||_2 (||b|| = 0: ||Q x^t|| <= tol) */
#define AJ_STOP_OBJGAP 1 /* |f(x^t) - f*| / (1 + |f*|) <= tol (Section 4 stopping rule) */
#define AJ_STOP_NONE 2   /* run exactly maxit iterations */

/* Arithmetic of the iteration. */
#define AJ_FP64 0    /* IEEE FP64 values, vectors and arithmetic */
#define AJ_DF64 1    /* double-float: FP64 data held as pairs of FP32 and computed on the
                        FP32 pipes with error-free transforms (~2^-48 relative per operation) */
#define AJ_FP32_IR 2 /* FP32 values and vectors inside, FP64 residual refinement outside */
#define AJ_BF16_IR 3 /* BF16 values x FP32 arithmetic inside, FP64 refinement outside */

/* How one fused sweep obtains Q y^t = Q x^{t-1} + beta (Q x^{t-1} - Q x^{t-2}).
 * All give the same iterates up to rounding (STORED and DELTA bit for bit).
 *   LAZY    sums both products over the gathered x^{t-1} and x^{t-2} (two
 *           multiply-adds per stored entry, fewest bytes);
 *   STORED  keeps u = Q x per row and re-reads u^{t-2} (one multiply-add per
 *           stored entry, two more n-vectors of traffic);
 *   DELTA   STORED that also keeps x^{t-1} - x^{t-2} per row in place of
 *           re-reading x^{t-2}, so y = x + beta (x - x_prev) costs one
 *           instruction instead of two (the kept difference is the one the
 *           update computes anyway for the restart test); AJ_FP64 only, one
 *           more n-vector written per sweep.
 *   Y       keeps y^t itself as a vector: the sweep gathers y^t, forms x^t and
 *           writes the candidate y^{t+1} = x^t + beta_{t+1} (x^t - x^{t-1})
 *           (beta_{t+1} depends on alpha_t only, known before the restart
 *           test; a restart drops the candidate and reads y^{t+1} = x^{t-1}
 *           from that iterate's buffer).  One multiply-add per stored entry,
 *           the row sum starting at -b, and six n-vectors of traffic; but the
 *           exact residual of x^{t-1} needs a second row sum.  It is formed
 *           on check sweeps only: once ||Q y^t - b|| (summed every 4th sweep,
 *           and every sweep within 10x of the stop) falls to 1.5 tol ||b||
 *           (widened by the largest residual-to-monitor ratio the checks have
 *           met), and every 32 iterations.  A solve so stops at the first
 *           checked iterate within tol: the oracle's stop iteration where the
 *           checks reach it, at most 31 iterations later otherwise.  The
 *           divergence guard reads ||Q y^t - b|| on the sweeps that sum it.
 *           Not with AJ_STOP_OBJGAP.
 * AUTO picks Y for AJ_FP64 with one right-hand side (its FP64 issue rate
 * binds on GB300, and Y runs the fewest FP64 instructions per row), DELTA for
 * AJ_FP64 with several or with AJ_STOP_OBJGAP; STORED for matrices stored as
 * SELL (irregular rows, whose gathers are random: one per entry instead of
 * two); Y for AJ_FP32_IR values in the stencil format with one right-hand
 * side and the relative-residual stop (one gathered vector instead of two:
 * 0.18 against 0.21 ms per 256^3 sweep); LAZY for the other precisions on CSR
 * and in the stencil format, where the second row sum gathers from the same
 * cached lines (measured faster on the 3-D Poisson system and on 2-D grids
 * with 4 RHS). */
#define AJ_SWEEP_AUTO 0
#define AJ_SWEEP_LAZY 1
#define AJ_SWEEP_STORED 2
#define AJ_SWEEP_DELTA 3
#define AJ_SWEEP_Y 4

/* Storage of Q for the fused sweep.  CSR: one row per thread.  SELL: the
 * SELL-C-sigma layout (C = 32 rows per slice, or 16 or 8 with one right-hand
 * side (aj_params.sell_c; 32 / C lanes share a row); rows sorted by length
 * within windows of sigma rows, each slice stored column-major so that a
 * warp's loads are coalesced), with rows longer than sell_lmax summed warp-cooperatively and
 * rows longer than 4096 entries CTA-cooperatively from CSR.  STENCIL: Q is
 * a constant-coefficient 5-point (n = N^2) or 7-point (n = N^3) stencil with
 * Dirichlet boundary in natural row order (i = x + N y + N^2 z), every row's
 * columns ascending, one diagonal and one off-diagonal value bitwise (the
 * grid Laplacians of Sec. 4); the sweep computes each row's columns and
 * values instead of loading them, in the CSR order and with the CSR values,
 * so its iterates equal those of CSR bit for bit.  aj_set checks every row on
 * the device and returns AJ_EINVAL for an explicit STENCIL on any other Q.
 * AUTO takes STENCIL where Q is one (rows not renumbered; not for AJ_FP64
 * with several right-hand sides or in the lazy form, where it measured
 * slower than CSR), keeps CSR for rows
 * of near-uniform length and otherwise times CSR and SELL candidates for a
 * few sweeps and keeps the fastest (the choice is cached per matrix shape
 * and precision for the process). */
#define AJ_FMT_AUTO 0
#define AJ_FMT_CSR 1
#define AJ_FMT_SELL 2
#define AJ_FMT_STENCIL 3

/* Row order of Q for the fused sweep (a format choice; the paper has no
 * counterpart).  RCM renumbers rows and columns by reverse Cuthill-McKee
 * (George and Liu, "Computer Solution of Large Sparse Positive Definite
 * Systems", 1981), so that the x entries a tile gathers lie close together
 * and stay in cache.  Each row keeps its entries in the caller's order, so
 * every row sum is bit for bit the one of the caller's order; only the
 * grouping of the FP64 reductions changes.  b, x0 and the returned x stay in
 * the caller's order.  AUTO applies RCM to large matrices without heavy rows
 * (n >= 16384, no row above 16x the mean length plus 16) whose current order
 * gathers from far away, and keeps it only when it shrinks the summed row
 * spans (max minus min column) at least fourfold. */
#define AJ_REORDER_AUTO 0
#define AJ_REORDER_NONE 1
#define AJ_REORDER_RCM 2

typedef struct {
  int j_policy;          /* AJ_J_ABSROWSUM (default) | AJ_J_SCALED_DIAG | AJ_J_BLKDIAG */
  double L;              /* AJ_J_SCALED_DIAG step constant; 0 = estimate by power iteration */
  double L_margin;       /* estimate used is (1 + L_margin) * lambda_hat (default 0.02) */
  int restart;           /* AJ_RESTART_ADAPTIVE (default) | AJ_RESTART_NONE */
  int momentum;          /* 1 (default): Nesterov extrapolation; 0: beta = 0 (Jacobi-type) */
  int64_t K0;            /* K_0 >= 2 (default 2) */
  double tol;            /* default 1e-8 */
  int stop;              /* AJ_STOP_RELRES (default) | AJ_STOP_OBJGAP | AJ_STOP_NONE */
  double fstar;          /* f* for AJ_STOP_OBJGAP */
  int64_t maxit;         /* iteration limit (inner iterations in total for the IR modes) */
  int precision;         /* AJ_FP64 (default) | AJ_DF64 | AJ_FP32_IR | AJ_BF16_IR */
  int format;            /* AJ_FMT_AUTO (default) | AJ_FMT_CSR | AJ_FMT_SELL | AJ_FMT_STENCIL */
  const double* x0;      /* initial point x^0 = y^1, n x nrhs column-major; NULL = 0 */
  int x0_on_device;
  double inner_tol;      /* IR modes: relative tolerance of each inner solve (default 1e-4) */
  int64_t max_outer;     /* IR modes: outer refinement steps (default 30) */
  int grid_ctas;         /* 0 = automatic; otherwise the number of persistent CTAs */
  int sweep_form;        /* AJ_SWEEP_AUTO (default) | _LAZY | _STORED | _DELTA | _Y */
  int sell_sigma;        /* AJ_FMT_SELL: sorting window sigma in rows (0 = 256) */
  int sell_lmax;         /* AJ_FMT_SELL: rows longer than this go to the warp-per-row bucket (0 = 64) */
  int reorder;           /* AJ_REORDER_AUTO (default) | AJ_REORDER_NONE | AJ_REORDER_RCM */
  int j_block;           /* AJ_J_BLKDIAG: rows per block, 1, 2, 4 or 8 (0 = 4) */
  int sell_c;            /* AJ_FMT_SELL: slice height C, 32, 16 or 8 (0 = 32): C rows per
                            warp step, 32 / C lanes share a row (one right-hand side) */
} aj_params;

/* Per-solve report. */
typedef struct {
  int64_t iters;    /* t of the returned x^t (summed over inner solves in the IR modes) */
  int64_t restarts; /* l: restarts taken */
  int64_t sweeps;   /* fused sweeps run (iterations + residual-only sweeps) */
  int64_t outer;    /* IR modes: outer steps; 0 otherwise */
  double relres;    /* ||b - Q x||_2 / ||b||_2 of the returned x, FP64 */
  double objgap;    /* |f(x) - f*| / (1 + |f*|) with the caller's f* */
  double L_used;    /* step constant used by AJ_J_SCALED_DIAG (0 otherwise) */
  double ms;        /* device time of the whole solve, milliseconds */
  double kernel_ms; /* device time of the fused iteration kernel launches alone */
  int64_t launches; /* kernels this solve launched (fused, setup and conversion kernels) */
  aj_status status; /* AJ_OK, AJ_EMAXIT, AJ_EDIVERGED, AJ_ENONFINITE or AJ_ETIMEOUT */
} aj_info;

/* What aj_set chose for the fused sweep (the autotuner's tuple under
 * AJ_FMT_AUTO).  The autotuner runs when the rows are long-tailed and the
 * system is large (n >= 65536): it times CSR and SELL with sigma in {256,
 * 4096} and sell_lmax in {64, 256}, then SELL's slice height C in {16, 8}
 * for the best of these, then 1-2 CTAs per SM below the kernel's occupancy,
 * 8 sweeps each, and caches the choice per matrix shape, precision, RHS
 * count, sweep form and order. */
typedef struct {
  int format;          /* AJ_FMT_CSR, AJ_FMT_SELL or AJ_FMT_STENCIL */
  int sell_c;          /* SELL slice height C: rows per warp step (0 unless SELL) */
  int sell_sigma;      /* SELL sorting window (0 unless SELL) */
  int sell_lmax;       /* SELL long-row threshold (0 unless SELL) */
  int lanes_per_row;   /* lanes that share a row: 32 / C for SELL with one RHS; with
                          several RHS one lane per RHS (2 or 4); else 1 */
  int rows_per_cta;    /* rows one CTA sweeps per tile */
  int threads_per_cta; /* 256 */
  int ctas_per_sm;     /* persistent CTAs per SM of the solve's launch */
  int grid;            /* persistent CTAs in all */
  int sweep_form;      /* the form in use: AJ_SWEEP_LAZY, _STORED, _DELTA or _Y */
  int tuned;           /* 1: chosen by timing candidates (or from the autotuner's cache) */
  int pad_;
  double fill_ratio;   /* stored entries over nnz (SELL padding); 1 for CSR, 0 for STENCIL */
} aj_tuning;

/* Fill *p with the defaults above. */
void aj_params_default(aj_params* p);

/* Create a solver context for Q and nrhs right-hand sides b (n x nrhs,
 * column-major; on the device iff Q->on_device).  nrhs in [1, 4].  The
 * library deep-copies Q and b into device memory laid out for the kernels;
 * it validates the CSR structure and the diagonal (AJ_EINVAL) and returns
 * AJ_ENOMEM if device memory runs out.  *out is NULL on failure. */
aj_status aj_create(const aj_csr* Q, const double* b, int nrhs, aj_ctx** out);

/* Set the solver parameters (copied).  Builds J^{-1} and, for
 * AJ_J_SCALED_DIAG with L = 0, estimates L by power iteration on
 * D^-1/2 Q D^-1/2 in FP64.  AJ_EINVAL on a bad parameter (the context keeps
 * its previous parameters); AJ_ENOMEM or AJ_ECUDA if building the arrays
 * fails, after which the context counts as never set: its next solve first
 * applies the default parameters, as on a fresh context. */
aj_status aj_set(aj_ctx* ctx, const aj_params* p);

/* The tuple of aj_tuning for the context's last successful aj_set.
 * AJ_EINVAL if ctx or out is NULL or aj_set has not succeeded yet. */
aj_status aj_get_tuning(aj_ctx* ctx, aj_tuning* out);

/* The format aj_set chose (AJ_FMT_CSR, AJ_FMT_SELL or AJ_FMT_STENCIL), its
 * sigma and long-row threshold (0 unless SELL), and the entries the sweep
 * loads per stored entry of Q (SELL padding overhead; 1.0 for CSR, 0.0 for
 * STENCIL). */
aj_status aj_get_format(aj_ctx* ctx, int* format, int* sigma, int* lmax, double* fill_ratio);

/* Whether aj_set renumbered the rows (1: reverse Cuthill-McKee order in use,
 * 0: the caller's order), and the summed row spans before and after (equal
 * when no reordering was tried). */
aj_status aj_get_order(aj_ctx* ctx, int* reordered, double* span_before, double* span_after);

/* Run all GPU work of ctx on this cudaStream_t (NULL = legacy default stream). */
aj_status aj_set_stream(aj_ctx* ctx, void* cuda_stream);

/* Solve.  x_out (n x nrhs, column-major, FP64) receives x^t on the host or
 * device.  info (may be NULL) receives the report of the last right-hand
 * side's worst status; info_per_rhs (may be NULL, nrhs entries) one report
 * per right-hand side.  Returns AJ_OK when every right-hand side met its stop
 * test, else the first failing status (x_out is still written). */
aj_status aj_solve(aj_ctx* ctx, double* x_out, int x_on_device, aj_info* info);
aj_status aj_solve_rhs(aj_ctx* ctx, double* x_out, int x_on_device, aj_info* info_per_rhs);

/* The comparator of Sec. 4.2: conjugate gradients with the diagonal
 * preconditioner M = diag(Q) (a zero diagonal entry counts as 1) on the same
 * Q and b, in FP64 (Saad, Iterative Methods for Sparse Linear Systems,
 * Alg. 9.1).  One persistent cooperative launch, two grid-synchronised passes
 * per iteration.  It stops when the recursive residual satisfies
 * ||r^t|| <= tol ||b|| or after maxit iterations.  tol, maxit, x0 and
 * grid_ctas come from aj_set; the other parameters do not apply.  ctx must
 * have one right-hand side (AJ_EINVAL otherwise).  x_out and info are as for
 * aj_solve: info->iters counts CG iterations, info->sweeps the passes over Q,
 * and relres is the FP64 residual of the returned x.  Returns AJ_OK,
 * AJ_EMAXIT, AJ_ENONFINITE, AJ_ETIMEOUT (a grid barrier gave up) or AJ_ENOMEM. */
aj_status aj_pcg_solve(aj_ctx* ctx, double* x_out, int x_on_device, aj_info* info);

/* Solve count independent contexts in ONE persistent launch (their sizes
 * may differ; each keeps its own momentum and restart state).  x_out[i] is
 * the output of ctx[i] (n_i x nrhs_i), info[i] its report (info may be NULL).
 * All contexts must share one precision and device (AJ_EINVAL otherwise) and
 * use the first context's stream.  Contexts whose sweep forms differ (AUTO
 * gives SELL matrices the stored form, CSR and stencil ones the lazy form in
 * the reduced precisions) run as one launch per sweep form, one after
 * another; every member's info then reports the whole call (ms, kernel_ms
 * and launches summed over the forms).  The return value is AJ_OK or the
 * first solver status (AJ_EMAXIT, AJ_EDIVERGED, AJ_ENONFINITE) of a member,
 * with every x_out and info written; any other error ends the call, and then
 * only the members of the forms that had already run have their x_out and
 * info written. */
aj_status aj_solve_batch(aj_ctx* const* ctx, int count, double* const* x_out, int x_on_device,
                         aj_info* info);

/* Continuous-batching server (no counterpart in the paper; it serves many
 * independent solves of Algorithm alg-jacobi at once).  A host thread runs
 * rounds: one batched persistent launch over every admitted request, each
 * running at most a few sweeps (about 1-4 ms of device time per round) from
 * its device-resident iterate, momentum and restart state.  After a round the
 * requests that met their stop test (or failed) are retired and queued
 * requests are admitted, first fit in submission order, while the device
 * memory of the admitted requests stays within hbm_budget_bytes and at most
 * max_slots are admitted.  Cutting a solve into rounds does not change its
 * arithmetic: a request computes exactly what aj_solve computes for the same
 * system with grid_ctas equal to its gang size (see aj_solve_batch).
 * The server runs on the device current at creation, on its own stream. */
aj_status aj_server_create(size_t hbm_budget_bytes, int max_slots, aj_server** out);
/* Queue an existing context (its device memory counts against the budget
 * while admitted).  Non-blocking.  The server uses ctx until aj_poll reports
 * the request finished; the caller must not touch ctx until then.
 * AJ_EBUSY if ctx alone exceeds the budget. */
aj_status aj_submit(aj_server* s, aj_ctx* ctx, uint64_t* ticket);
/* Queue a solve from the caller's data (Q, b as for aj_create, p as for
 * aj_set; NULL p = defaults).  The server copies Q, b and p->x0 at once into
 * host memory of its own; it allocates the device state only when the request
 * is admitted and frees it when the request retires, so the budget bounds the
 * device memory the server uses.  AJ_EBUSY if the request alone exceeds the
 * budget. */
aj_status aj_submit_csr(aj_server* s, const aj_csr* Q, const double* b, int nrhs,
                        const aj_params* p, uint64_t* ticket);
/* AJ_PENDING until the request has finished; then writes x_out (host, n x
 * nrhs column-major; may be NULL) and info (may be NULL; info->ms is the
 * wall time from submission to completion) and returns the solve's status.
 * A finished request is reported once; an unknown ticket gives AJ_EINVAL. */
aj_status aj_poll(aj_server* s, uint64_t ticket, double* x_out, aj_info* info);
/* Block until the request has finished or timeout_ms has passed (< 0: no
 * limit).  AJ_OK when it has finished (collect it with aj_poll), AJ_PENDING
 * on timeout. */
aj_status aj_server_wait(aj_server* s, uint64_t ticket, double timeout_ms);
/* Server counters: rounds run, requests admitted and completed, the largest
 * number admitted at once in a round and the largest admitted device memory
 * (both show requests sharing the GPU), current use and queue length, and
 * the device time of all rounds. */
typedef struct {
  uint64_t rounds;
  uint64_t admitted;
  uint64_t completed;
  int64_t peak_active;
  uint64_t peak_bytes;
  uint64_t in_use_bytes;
  int64_t queued;
  double kernel_ms;
} aj_server_stats;
aj_status aj_server_get_stats(aj_server* s, aj_server_stats* out);
/* Stop the server after its current round; unfinished requests are dropped
 * (contexts submitted with aj_submit get their stream back). */
void aj_server_destroy(aj_server* s);

/* Solver state (x^t, x^{t-1}, alpha_t, t, l, K_l, K_re per right-hand side)
 * for checkpoint/resume.  aj_get_state with buf = NULL writes the size to
 * *size; aj_set_state restores it so that the next aj_solve continues the
 * run as if it had not stopped. */
aj_status aj_get_state(aj_ctx* ctx, void* buf, size_t* size);
aj_status aj_set_state(aj_ctx* ctx, const void* buf, size_t size);

/* Iterations t (1-based) at which the last solve of right-hand side rhs
 * restarted; writes at most cap entries and the total count to *count. */
aj_status aj_restart_log(aj_ctx* ctx, int rhs, int64_t* iters, int64_t cap, int64_t* count);

void aj_destroy(aj_ctx* ctx);
const char* aj_strerror(aj_status s);

/* ---- Allocation-free solve.  The paper has no counterpart: this entry point
 * exists for callers that must not allocate device memory, for instance
 *   - a latency-critical service whose other streams would stall on the
 *     implicit device synchronisation of cudaMalloc / cudaFree;
 *   - a process whose device memory is reserved up front by a framework's
 *     caching allocator, where a foreign cudaMalloc can fail at run time;
 *   - deployments that fix every device buffer when the library loads.
 * It runs the same FP64 fused solve as aj_create + aj_set + aj_solve for ONE
 * right-hand side (same J, restart rule, stop test and kernel), but takes all
 * of its scratch -- J^{-1}, the three iterate buffers, the two Q x buffers of
 * the stored sweep form, the per-CTA partial sums, the grid-barrier counter,
 * the error word and the solver state -- from one fixed device array inside
 * libaj of about 6.1 MB, sized for
 * n <= AJ_NOALLOC_MAX_N.  Every GPU that loads libaj holds that array until
 * the process exits.  The call allocates nothing: no cudaMalloc, cudaFree or
 * allocating library routine.
 *
 *   Q       CSR on the current device (Q->on_device must be 1); read only.
 *   b       n device doubles; read only.
 *   p       parameters as for aj_set; precision must be AJ_FP64 (the sweep
 *           form is always AJ_SWEEP_STORED, which computes the same iterates
 *           as the other FP64 forms up to rounding and, bit for bit, as
 *           AJ_SWEEP_DELTA;
 *           p->reorder is ignored: rows keep the caller's order), and
 *           AJ_J_SCALED_DIAG needs p->L > 0 (no power-iteration estimate);
 *           p->x0, if given, must be a device pointer (x0_on_device = 1).
 *   x_out   n device doubles; receives the returned iterate x^t.
 *   info    may be NULL; iters, restarts, sweeps, relres (FP64 residual of
 *           x^t from the fused sweep), objgap (AJ_STOP_OBJGAP only, else 0),
 *           status; ms and kernel_ms are the host wall time of the call.
 *   cuda_stream  cudaStream_t to run on (NULL = legacy default stream).
 * Returns as aj_solve; AJ_ENOMEM when n > AJ_NOALLOC_MAX_N (the problem does
 * not fit the fixed array), AJ_EINVAL for a bad argument or matrix.  The call
 * returns after its GPU work has finished.
 *
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current) and the kernel's
 * occupancy; make that first call before any stream capture begins.  Every
 * call copies its status and solver state to the host and synchronises
 * cuda_stream before it returns.  Every call on a device shares the one
 * array, and it keeps the last call's contents (each call re-initialises what
 * must start at zero): calls whose GPU work overlaps -- from two host
 * threads, or on two streams -- race on it and must be serialised by the
 * caller. */
#define AJ_NOALLOC_MAX_N 131072
aj_status aj_solve_noalloc(const aj_csr* Q, const double* b, const aj_params* p, double* x_out,
                           aj_info* info, void* cuda_stream);

/* Diagnostics: number of CUDA kernels libaj has launched in this process. */
uint64_t aj_kernel_launches(void);

/* Diagnostics: lookups in this process of aj_set's two caches, keyed by the
 * matrix, whose hits skip host work: the locality ordering (RCM test, keyed
 * by the sparsity pattern's hash) and the autotuner's choice (keyed by n,
 * nnz, the row-length moments, precision, RHS count, sweep form and order).
 * Any pointer may be NULL. */
void aj_cache_stats(uint64_t* order_hits, uint64_t* order_misses, uint64_t* tune_hits, uint64_t* tune_misses);

/* ---- Failure-detection test hooks.  The paper has no counterpart: they let
 * a test drive the library's error paths without faulting a GPU.
 *
 * aj_test_barrier_stall: the next persistent solve launched in this process
 * (aj_solve, aj_solve_rhs) runs with every grid-barrier wait limited to
 * timeout_ms (0 < timeout_ms <= 4000; the default limit is 4 s), and its CTA
 * number `cta` withholds its arrival at the first barrier.  Every other wait
 * then runs out, the kernel records the timeout and returns, and the solve
 * returns AJ_ETIMEOUT; the context stays usable and its next solve runs
 * normally.  A `cta` at or beyond the launch's grid withholds nothing;
 * cta = -1 disarms the hook.  One shot: the hook is cleared by the launch
 * that takes it.  AJ_EINVAL for a bad argument.
 *
 * aj_test_alloc_fail: the device allocation that comes after `after` more
 * successful ones (0: the very next) fails as if the device were out of
 * memory, once; the call that needed it returns AJ_ENOMEM having released
 * what it had allocated.  after = -1 disarms the hook.  AJ_EINVAL if
 * after < -1.
 *
 * Both hooks are process-wide and meant for single-threaded tests. */
aj_status aj_test_barrier_stall(int cta, double timeout_ms);
aj_status aj_test_alloc_fail(int64_t after);

#ifdef __cplusplus
}
#endif

#endif /* AJ_H */
