/*
 * trs.h -- C ABI of libtrs, a GB300 (sm_103a) solver for the block-sparse
 * Jacobian systems of a fully implicit thermal reservoir model, after Liu &
 * Chen, "A Scalable Thermal Reservoir Simulator for Giant Models on Parallel
 * Computers" (arXiv 1812.03952).
 *
 * The system A x = b has b x b blocks numbered cell by cell with the well
 * (bottom-hole-pressure) unknowns after the cells (Sec. "Linear Solver",
 * Eq. mat-ja; Sec. "Linear System": well equations placed last).  A well's
 * BHP is entry 0 of its padded b x b block; entries 1..b-1 of a well block
 * are padding that the caller fills with an identity diagonal and zero RHS.
 *
 * The solve is restarted flexible GMRES, right-preconditioned by CPR-FPF
 * (Sec. "Preconditioners", Algorithm pc-fpf) applied to the ABF-decoupled
 * matrix D^-1 A (Sec. "Decoupling Methods", Eqs. decoupled-eq and
 * decoupled-abf), with a pressure-AMG stage and a multicolour block ILU(0)
 * (or ILU(1)) "F" stage; BiCGSTAB is offered beside FGMRES.  All arithmetic
 * runs in CUDA kernels on the current device.
 *
 * Conventions for every entry point:
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream); device work is ordered on it.  Calls that return results to
 *     the host synchronise that stream.  The library's kernels use
 *     programmatic dependent launch: each waits for the work before it in
 *     the stream to complete before touching memory, so ordering with the
 *     caller's own work on the stream is ordinary stream order.
 *   - "device pointer" arguments must point to memory of the current device,
 *     "host pointer" arguments to host memory.  Vectors are FP64 arrays of
 *     n_block_rows * b entries, block by block, owned by the caller; device
 *     vectors must be 16-byte aligned (cudaMalloc and the PyTorch allocator
 *     return 256-byte aligned memory), else TRS_ERR_INVALID.
 *   - Handles (trs_bsr, trs_cpr) are owned by the library and released with
 *     the matching *_destroy call.
 *   - Every call returns a trs_status; no exception, abort or device trap
 *     crosses the boundary.  trs_last_error() returns a thread-local
 *     message describing the last failure.
 */
#ifndef TRS_H
#define TRS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t trs_status;

#define TRS_OK 0
#define TRS_ERR_INVALID (-1)          /* bad argument or malformed matrix */
#define TRS_ERR_OOM (-2)              /* device allocation failed */
#define TRS_ERR_CUDA (-3)             /* CUDA runtime error */
#define TRS_ERR_SINGULAR_BLOCK (-4)   /* a diagonal block (or ILU pivot block) is singular */
#define TRS_ERR_NAN (-5)              /* NaN or Inf met in a residual norm */
#define TRS_ERR_NOT_CONVERGED (-6)    /* iteration limit reached; stats and x hold the last iterate */
#define TRS_ERR_BREAKDOWN (-7)        /* Krylov breakdown without convergence */
#define TRS_ERR_COARSENING (-8)       /* AMG coarsening stalled above the dense limit */
#define TRS_ERR_UNSUPPORTED (-9)      /* block size or option outside the supported set */

/* Preconditioner precision. */
#define TRS_FP64 0          /* everything in FP64 */
#define TRS_FP32_PREC 1     /* CPR stored and applied in FP32; Krylov basis, residuals,
                               Givens/least squares and the coarsest LU stay FP64 */

typedef struct trs_bsr trs_bsr;
typedef struct trs_cpr trs_cpr;

/* CPR stage ordering (trs_cpr_opts.stages), Sec. "Preconditioners".  With
 * f = D^-1 v, F = block ILU(0) of Ã and P = one AMG V-cycle on A_PP:
 *   FPF (Algorithm pc-fpf): y = F^-1 f; y += Pi_p P (f - Ã y)_p; z = y + F^-1 (f - Ã y);
 *   FP:  the first two steps, z = y;
 *   PF:  y = Pi_p P f_p; z = y + F^-1 (f - Ã y). */
#define TRS_CPR_FPF 0
#define TRS_CPR_FP 1
#define TRS_CPR_PF 2

/* Decoupling D^-1 A (trs_cpr_opts.decoupling), Sec. "Decoupling Methods":
 *   ABF: D_i = A_ii (Eq. decoupled-abf), inverted by Gauss-Jordan elimination
 *        with partial row pivoting, which is also the GJE decoupling;
 *   NONE: D_i = I;
 *   FRS: D_i^-1 = R, ones in the first row and on the diagonal (Eq.
 *        decoupled-frs): every equation is added into the pressure row;
 *   FRS_ABF: the two-stage FRS+ABF, D_i^-1 = (R A_ii)^-1 R.
 * The dynamic row sum (DRS) of the paper is defined only by citation and is
 * not offered. */
#define TRS_DEC_ABF 0
#define TRS_DEC_NONE 1
#define TRS_DEC_FRS 2
#define TRS_DEC_FRS_ABF 3

/* Level of fill of the block ILU stage F (trs_cpr_opts.ilu_fill).  The
 * paper's subdomain solves may be block ILU(k), and its recommended level is
 * k = 1 (Sec. "Preconditioners", the RAS paragraph).
 *   TRS_ILU0: block ILU(0) on the pattern of Ã, rows in the colour-major
 *     order of a Jones-Plassmann colouring (about 6 colours on a 7-point
 *     grid);
 *   TRS_ILU1: block ILU(1): the pattern of Ã plus every (i, j) with a
 *     neighbour k ordered before both (level of fill 1), rows in the
 *     colour-major order of a distance-2 colouring: grid cell (x, y, z)
 *     takes colour (x + 2y + 3z) mod 7, the other rows (wells), in index
 *     order, the first colour from 7 on not taken by an earlier such row
 *     that is adjacent to them or shares a neighbour with them.  Needs a
 *     matrix created with grid_dims; TRS_ERR_UNSUPPORTED when two rows of
 *     one colour are coupled in the factor pattern (a cell coupled to
 *     another cell outside its 7-point star).  The fill pattern is built on
 *     the host once, at trs_cpr_setup. */
#define TRS_ILU0 0
#define TRS_ILU1 1

typedef struct {
  int32_t precision;     /* TRS_FP64 or TRS_FP32_PREC */
  double theta;          /* AMG strength threshold (default 0.08) */
  int32_t coarse_max;    /* stop coarsening at <= coarse_max rows (default 64) */
  int32_t max_levels;    /* default 12 */
  int32_t cheb_degree;   /* Chebyshev smoother degree (default 2) */
  uint32_t seed;         /* seed of the MIS-2 and colouring priorities */
  int32_t stages;        /* TRS_CPR_FPF (default), TRS_CPR_FP or TRS_CPR_PF */
  int32_t decoupling;    /* TRS_DEC_ABF (default), TRS_DEC_NONE, TRS_DEC_FRS, TRS_DEC_FRS_ABF */
  int32_t ilu_fill;      /* level of fill of the block ILU stage: TRS_ILU0 (default) or TRS_ILU1 */
} trs_cpr_opts;

/* Krylov method (trs_solve_opts.method). */
#define TRS_FGMRES 0        /* restarted flexible GMRES with CGS2 */
#define TRS_BICGSTAB 1      /* BiCGSTAB (van der Vorst), the solver of the paper's runs */

typedef struct {
  double rtol;           /* stop when ||b - A x||_2 <= rtol ||b||_2 (true FP64 residual) */
  int32_t restart;       /* FGMRES subspace size per cycle, 1..64 (default 30) */
  int32_t maxit;         /* total iteration limit (default 1000; one BiCGSTAB
                            iteration applies A and M twice) */
  int32_t use_x0;        /* 1: x holds the initial guess; 0: start from x = 0 */
  int32_t method;        /* TRS_FGMRES (default) or TRS_BICGSTAB: read by
                            trs_solve_adjoint; the named solve calls set it */
  int32_t time_phases;   /* 1: time the preconditioner, operator SpMV and
                            orthogonalisation phases with CUDA events on the
                            solve's stream (trs_solve_stats.ms_precond ...);
                            0 (default): no events between the launches */
} trs_solve_opts;

typedef struct {
  int32_t iters;         /* Arnoldi steps (FGMRES) or iterations (BiCGSTAB) */
  int32_t restarts;      /* cycles after the first */
  int32_t converged;
  int32_t amg_levels;
  int32_t n_colours;
  double est_relres;     /* recurrence residual / ||b|| at the last step */
  double true_relres;    /* ||b - A x|| / ||b|| of the returned x, FP64 */
  double ms_setup;       /* device time of the last trs_cpr_setup/update */
  double ms_solve;       /* device time of this solve */
  /* With opts.time_phases = 1 (else 0): device time of the CPR applications
   * (with the D^-1 scaling), of the operator SpMVs w = A z, and of the
   * orthogonalisation and vector updates (FGMRES: CGS2 and the Givens step;
   * BiCGSTAB: the vector updates with their fused dot products), and the
   * number of operator SpMV launches timed. */
  double ms_precond;
  double ms_spmv;
  double ms_orth;
  int64_t spmv_launches;
} trs_solve_stats;

typedef struct {
  int64_t n_block_rows;
  int32_t b;
  int64_t nnzb;
  int64_t n_cells;       /* rows on the structured 7-point grid (0 if none) */
  int32_t grid[3];
} trs_bsr_info;

typedef struct {
  int32_t n_levels;
  int32_t n_colours;
  int32_t precision;
  int64_t level_rows[16];
  int64_t level_nnz[16];
  double level_lambda[16]; /* Gershgorin bound of D^-1 A per level */
} trs_cpr_info;

/* ------------------------------------------------------------------ matrix */

/* Creates a device block matrix from a general BSR on the host.
 * n_block_rows, b: block rows and block size (b in 1..5).
 * row_ptr[n_block_rows+1] (int64), col_idx[nnzb] (int32): host pointers;
 *   columns sorted and unique in each row, every row holds its diagonal
 *   block, the block pattern is structurally symmetric.
 * values: host pointer to nnzb*b*b doubles, each block row-major, or NULL
 *   (zeros; fill later with trs_bsr_update_values).
 * grid_dims: host pointer to {nx, ny, nz} when the first nx*ny*nz rows are
 *   the cells of a structured grid (cell c = x + nx*(y + ny*z)) whose
 *   couplings are the 7-point neighbours; other blocks (wells) go to a
 *   general tail.  NULL: every row is stored in the general form.
 *   The kernels are built for the grid form: in the general form every row
 *   takes the paths meant for the few long well rows (a warp or a block per
 *   row), which are correct but slow (on a 1M-cell 7-point system about 11x
 *   for the SpMV and 46x for a CPR-FGMRES solve).
 * Errors: TRS_ERR_INVALID (checked on the host before any upload),
 *   TRS_ERR_UNSUPPORTED, TRS_ERR_OOM, TRS_ERR_CUDA.  Inputs stay caller-owned. */
trs_status trs_bsr_create(int64_t n_block_rows, int32_t b, const int64_t *row_ptr,
                          const int32_t *col_idx, const double *values, const int32_t *grid_dims,
                          void *stream, trs_bsr **out);

/* Creates the block pattern of the synthetic thermal Jacobian: an nx*ny*nz
 * grid with the 7-point two-point-flux stencil (Sec. "Numerical Methods"),
 * plus n_wells well rows coupled to their perforated cells (Sec. "Well
 * Modeling").  perf_well[n_perf], perf_cell[n_perf]: host pointers; a well
 * perforates a cell at most once.  Values are zero until trs_bsr_assemble. */
trs_status trs_bsr_create_synthetic(int32_t nx, int32_t ny, int32_t nz, int32_t b, int32_t n_wells,
                                    int64_t n_perf, const int32_t *perf_well,
                                    const int32_t *perf_cell, void *stream, trs_bsr **out);

/* Assembles the values of a matrix made by trs_bsr_create_synthetic.
 * perm: device pointer, n_cells doubles: permeability k (mD) if
 *   perm_is_log == 0, else theta = ln k.
 * T_f = c_t * 2 k_i k_j / (k_i + k_j) on every internal face (k scaled by
 *   kvkh on z faces; T_f = 0 when k_i + k_j = 0): harmonic mean of Sec.
 *   "Numerical Methods".  M: device, [n_cells][6][b][b] mobility block of
 *   each directed face (directions -z,-y,-x,+x,+y,+z).  acc: device,
 *   [n_cells][b][b].  A_ij = -T_f M_ij; A_ii = acc_i + sum_j T_f M_ij
 *   + well terms.  wi: device [n_perf]; lam: device [n_perf][b].
 *   Peaceman rate (Eq. well-model): cell row c gets +wi*lam[r] in its own
 *   pressure column and -wi*lam[r] in the well's BHP column; well row
 *   (fixed-rate form sum_m Q_m = c) gets sum_m wi_m*Lam_m on its diagonal
 *   and -wi_m*Lam_m in column (c_m, 0), Lam_m = sum_r lam_m[r]. */
trs_status trs_bsr_assemble(trs_bsr *A, const double *perm, int32_t perm_is_log, double kvkh,
                            double c_t, const double *M, const double *acc, const double *wi,
                            const double *lam, void *stream);

/* trs_bsr_assemble with the inputs (perm, M, acc, wi, lam) in host memory:
 * the library copies them into a device staging area that the matrix keeps
 * (allocated at the first call) and assembles from there; the copies are
 * ordered on `stream` and are part of the call.  Pinned host memory lets the
 * copies run asynchronously.  Same sizes and errors as trs_bsr_assemble. */
trs_status trs_bsr_assemble_host(trs_bsr *A, const double *perm, int32_t perm_is_log, double kvkh,
                                 double c_t, const double *M, const double *acc, const double *wi,
                                 const double *lam, void *stream);

/* Replaces all values.  values: nnzb*b*b doubles in the matrix's canonical
 * BSR order (rows ascending, columns ascending; the order of trs_bsr_pattern),
 * on the device if values_on_device, else on the host. */
trs_status trs_bsr_update_values(trs_bsr *A, const double *values, int32_t values_on_device,
                                 void *stream);

/* Copies the values out in canonical BSR order (device or host pointer). */
trs_status trs_bsr_get_values(const trs_bsr *A, double *values, int32_t values_on_device,
                              void *stream);

/* Multiplies every diagonal block by a per-row factor: A_ii <- s_i A_ii.
 * s: device pointer, n_block_rows doubles. */
trs_status trs_bsr_scale_diagonal(trs_bsr *A, const double *s, void *stream);

/* Pattern of the canonical BSR order: row_ptr[n+1], col_idx[nnzb] (host). */
trs_status trs_bsr_pattern(const trs_bsr *A, int64_t *row_ptr, int32_t *col_idx);
trs_status trs_bsr_get_info(const trs_bsr *A, trs_bsr_info *info);

/* y = alpha * op(A) x + beta * y, op = transpose ? A^T : A; x, y: device
 * pointers, FP64.  The product with A is the block SpMV of the Krylov
 * operator (sparse BLAS of Sec. "Linear Solver"); A^T is a gather of the
 * transposed blocks (no explicit transpose is formed). */
trs_status trs_bsr_spmv(const trs_bsr *A, double alpha, const double *x, double beta, double *y,
                        int32_t transpose, void *stream);

/* Forms A^T explicitly as a new matrix (blocks transposed). */
trs_status trs_bsr_transpose(const trs_bsr *A, void *stream, trs_bsr **out);

/* Refreshes the values of AT = trs_bsr_transpose(A0) from A, which must have
 * A0's pattern (for example A0 itself after new values): (A^T)_ij = (A_ji)^T. */
trs_status trs_bsr_transpose_values(const trs_bsr *A, trs_bsr *AT, void *stream);

void trs_bsr_destroy(trs_bsr *A);

/* ---------------------------------------------------------- preconditioner */

/* Fills *opts with the defaults (FP64, theta 0.08, coarse_max 64, 12 levels,
 * Chebyshev degree 2). */
void trs_cpr_default_opts(trs_cpr_opts *opts);

/* Builds CPR-FPF for A: ABF decoupling D_i = A_ii inverted by Gauss-Jordan
 * with row pivoting (GJE), Ã = D^-1 A; pressure matrix A_p = (Ã_ij)_00;
 * aggregation AMG of A_p (strength, MIS-2, unsmoothed aggregates, Galerkin
 * P^T A P, Chebyshev smoothing, dense LU at the coarsest level);
 * multicolouring and block ILU(0) of Ã (block ILU(1) with opts->ilu_fill =
 * TRS_ILU1).  The handle keeps a reference to nothing of A; A may change
 * afterwards (see trs_cpr_update).
 * Errors: TRS_ERR_SINGULAR_BLOCK, TRS_ERR_COARSENING, TRS_ERR_INVALID,
 * TRS_ERR_UNSUPPORTED, TRS_ERR_OOM, TRS_ERR_CUDA. */
trs_status trs_cpr_setup(const trs_bsr *A, const trs_cpr_opts *opts, void *stream,
                         trs_cpr **out);

/* Refreshes M for new values of A with the same pattern.  reuse_amg = 1
 * keeps the AMG aggregates (the strength graph, MIS-2 and aggregation, so P
 * and every coarse pattern) and recomputes all values: the decoupling, the
 * pressure matrix, every Galerkin product, the smoother bounds, the
 * coarsest inverse and the ILU(0) factors; reuse_amg = 0 rebuilds
 * everything. */
trs_status trs_cpr_update(trs_cpr *M, const trs_bsr *A, int32_t reuse_amg, void *stream);

/* z = M^-1 v = CPR(Ã)^-1 (D^-1 v): one application of the preconditioner
 * (device pointers, FP64; computed in the handle's precision). */
trs_status trs_cpr_apply(const trs_cpr *M, const double *v, double *z, void *stream);

trs_status trs_cpr_get_info(const trs_cpr *M, trs_cpr_info *info);

/* Setup objects copied to host memory, for inspection and tests:
 * aggregates of level l (n_l int32, -1 = not aggregated); colours
 * (n_block_rows int32); decoupled blocks Ã in canonical BSR order and
 * D^-1 (n_block_rows*b*b), FP64; level-l pressure operator in CSR
 * (row_ptr n_l+1 int64, col nnz int32, val nnz double). */
trs_status trs_cpr_get_aggregates(const trs_cpr *M, int32_t level, int32_t *agg);
trs_status trs_cpr_get_colours(const trs_cpr *M, int32_t *colour);
trs_status trs_cpr_get_decoupled(const trs_cpr *M, double *vt, double *dinv);
trs_status trs_cpr_get_level(const trs_cpr *M, int32_t level, int64_t *row_ptr, int32_t *col,
                             double *val);

/* Applies one AMG V-cycle of the pressure hierarchy to r (device pointers,
 * n_0 doubles): e = AMG(A_p)^-1 r. */
trs_status trs_cpr_vcycle(const trs_cpr *M, const double *r, double *e, void *stream);

void trs_cpr_destroy(trs_cpr *M);

/* ------------------------------------------------------------------ solves */

void trs_solve_default_opts(trs_solve_opts *opts);

/* Solves A x = b by FGMRES(restart) right-preconditioned with M (built from
 * A).  b, x: device pointers.  Convergence is decided on the true FP64
 * residual.  TRS_ERR_NOT_CONVERGED still fills stats and leaves the last
 * iterate in x. */
trs_status trs_fgmres_solve(const trs_bsr *A, const trs_cpr *M, const double *b, double *x,
                            const trs_solve_opts *opts, void *stream, trs_solve_stats *stats);

/* The same solve with b and x in host memory; the copies are part of the
 * call.  The device copies of b and x are kept by M after the first call
 * (2 * n_block_rows * b doubles); pinned host memory lets the copies run
 * asynchronously.  The call synchronises `stream`. */
trs_status trs_fgmres_solve_host(const trs_bsr *A, const trs_cpr *M, const double *b_host,
                                 double *x_host, const trs_solve_opts *opts, void *stream,
                                 trs_solve_stats *stats);

/* Solves A x = b by BiCGSTAB right-preconditioned with M: the Krylov
 * method of every run in the paper (Sec. "Numerical Studies", subsections
 * "Numerical Performance" and "Scalability").  Same arguments, errors and true-residual test as
 * trs_fgmres_solve; opts->restart is not used.  A cycle ends when the
 * recurrence residual meets rtol, or on breakdown (rho = 0 or omega = 0); the
 * next cycle restarts from the true FP64 residual with r^ = r. */
trs_status trs_bicgstab_solve(const trs_bsr *A, const trs_cpr *M, const double *b, double *x,
                              const trs_solve_opts *opts, void *stream, trs_solve_stats *stats);

/* trs_bicgstab_solve with b and x in host memory; the copies are part of
 * the call. */
trs_status trs_bicgstab_solve_host(const trs_bsr *A, const trs_cpr *M, const double *b_host,
                                   double *x_host, const trs_solve_opts *opts, void *stream,
                                   trs_solve_stats *stats);

/* Adjoint of x = A^-1 b for a loss L(x) with g = dL/dx: solves
 * A^T lambda = g with opts->method (FGMRES by default) and M_T (a CPR built on A^T, e.g. from
 * trs_bsr_transpose), so dL/db = lambda; if dA is not NULL it receives
 * dL/dA_ij = -lambda_i x_j^T for every stored block in canonical BSR
 * order.  g, x, lambda, dA: device pointers. */
trs_status trs_solve_adjoint(const trs_bsr *A, const trs_bsr *AT, const trs_cpr *M_T,
                             const double *g, const double *x, double *lambda, double *dA,
                             const trs_solve_opts *opts, void *stream, trs_solve_stats *stats);

/* Residual r = b - A x and its 2-norm without allocating anything.
 * The paper has no counterpart: this call is for callers that must not
 * allocate device memory while they run (for instance loops that cannot
 * afford the device-wide synchronisation of cudaMalloc/cudaFree, or
 * processes whose device memory belongs to their own pool allocator).
 * x, b, r: device pointers (n*b doubles, caller-owned, r must not alias x or
 * b); norm: host pointer that receives ||r||_2.  The call copies the norm to
 * *norm and synchronises `stream` before it returns.  The reduction scratch
 * is a static device array of 778,752 bytes inside the library (the partial
 * sums of at most 1,216 blocks, a counter and the result), held by every
 * GPU that loads the library until the process exits; the blocks stride over
 * the rows, so every matrix the library accepts fits.  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress), so that
 * first call should come before any stream capture.  Every call on a device
 * shares the one array, so calls that overlap on the GPU (other streams,
 * other threads) race; the counter is cleared at the start of each call.
 * No cudaMalloc, cudaFree or allocating library routine is called. */
trs_status trs_residual_norm_noalloc(const trs_bsr *A, const double *x, const double *b, double *r,
                                     double *norm, void *stream);

/* dA = -lambda_i x_j^T on every stored block (canonical order). */
trs_status trs_outer_product(const trs_bsr *A, const double *lambda, const double *x, double *dA,
                             void *stream);

/* Gradient of L with respect to theta = ln k for a matrix assembled by
 * trs_bsr_assemble with the same perm/kvkh/c_t/M:
 *   dL/dT_f = lambda_i^T M_if (x_j - x_i) + lambda_j^T M_jf' (x_i - x_j),
 *   dL/dtheta_i = sum_f dL/dT_f T_f k_j / (k_i + k_j).
 * (the outer product -lambda x^T contracted with dA/dT_f, formed without
 * storing dA).  dtheta: device pointer, n_cells doubles (overwritten). */
trs_status trs_chain_theta(const trs_bsr *A, const double *perm, int32_t perm_is_log,
                           double kvkh, double c_t, const double *M, const double *lambda,
                           const double *x, double *dtheta, void *stream);

/* ------------------------------------------------ thermal model Jacobian */

/* Parameters of the thermal model assembled by trs_thermal_assemble (Sec.
 * "Mathematical Model").  Units: p kPa, T C, lengths m, time day, amounts
 * gmol, energy kJ, permeability mD, viscosity cP. */
typedef struct {
  double dx, dy, dz;          /* cell sizes */
  double depth_top;           /* depth of the top face of layer 0 (z grows downward) */
  double dt;                  /* time step of the backward Euler discretisation */
  double kvkh;                /* vertical / horizontal permeability ratio */
  double gravity;             /* m/s^2 (0 switches gravity off) */
  double phi_ref, cpor, ctpor, p_ref, T_ref;  /* phi = phi_ref (1 + cpor (p - p_ref) - ctpor (T - T_ref)) */
  double cp1_r, cp2_r;        /* rock U_r = cp1_r (T - T_ref) + cp2_r / 2 (T^2 - T_ref^2), kJ/m^3 */
  double kt_w, kt_o, kt_g, kt_r;  /* thermal conductivities, kJ/(m day C) */
  double rho_w_ref, cp_w, ct1_w, ct2_w, cpt_w;  /* water molar density correlation (Sec. "Density") */
  double mw_w;                /* molar mass of water, kg/gmol */
  double avisc_w, bvisc_w;    /* mu_w = avisc_w exp(bvisc_w / T_K), cP */
  double kv1, kv2, kv3, kv4, kv5;  /* K_W = (kv1/p + kv2 p + kv3) exp(kv4 / (T - kv5)) */
  double per_eps;             /* PER: K*_W = S_w / (S_w + per_eps) K_W */
  double tc_w, pc_w;          /* critical temperature (C) and pressure (kPa) of water (Redlich-Kwong) */
  double cpg[5];              /* H_gW = integral from T_ref of sum_k cpg[k] t^k, kJ/gmol */
  double hvr, ev;             /* heat of vaporisation hvr (tc_w - T)^ev */
  double rho_o_ref, cp_o, ct1_o, ct2_o, cpt_o;  /* oil component density correlation */
  double mw_o;                /* molar mass of the oil component */
  double avisc_o, bvisc_o;    /* mu_o = avisc_o exp(bvisc_o / T_K) */
  double cpl1_o;              /* H_o = cpl1_o (T - T_ref) (liquid-based enthalpy) */
  double mug_a, mug_b;        /* mu_g = mug_a + mug_b T */
  double h_inj;               /* enthalpy of the steam the injectors inject, kJ/gmol */
  double R_gas;               /* gas constant, kJ/(gmol K) */
} trs_thermal_params;

/* Jacobian and residual of one Newton step of the thermal model for a
 * matrix made by trs_bsr_create_synthetic with b = 4: one component set,
 * water in the water and gas phases and one heavy-oil component in the oil
 * phase (Sec. "Mathematical Model").  Unknowns per cell (p, S_w, S_g, T);
 * equations: water and oil moles (Eq. eq4.2), energy (Eq. eq4.3) and the gas
 * constraint K*_W(p, T, S_w) - 1 = 0 where gas exists, S_g = 0 where not
 * (Sec. "Spatial Discretization").  Backward Euler in time; two-point fluxes
 * with the harmonic mean of the permeabilities and upstream k_r rho / mu and
 * enthalpy per phase; conduction with the harmonic mean of the bulk
 * conductivities; densities, Redlich-Kwong gas, viscosities, porosity,
 * tables with Stone's model II, enthalpies by the paper's correlations.
 * Wells (Sec. "Well Modeling"): well_type[w] = 0, an injector at the fixed
 * rate well_target[w] (gmol/day) with Q = wi (p_b - p) of steam
 * (unweighted mobility); 1, a producer at the fixed BHP well_target[w] (kPa)
 * with Q_a = wi c lambda_a (p_b - p) from the cell's mobilities.
 * Host pointers: prm; swt (nswt x 3: S_w, k_rw, k_row) and slt (nslt x 3:
 * S_l, k_rg, k_rog), 2..32 rows with increasing saturations.  Device
 * pointers: perm (n_cells, mD), u and u_old ((n_cells + n_wells) * 4: cells
 * (p, S_w, S_g, T), wells (p_b, 0, 0, 0)), gas (n_cells bytes), wi (n_perf),
 * well_type (n_wells int32), well_target (n_wells), residual (out, n * 4:
 * R(u), with R = u on the padding entries of well blocks).  The values of
 * A become dR/du.  The matrix keeps a scratch of 50 doubles per cell for
 * the cell properties (allocated at the first call).
 * Errors: TRS_ERR_INVALID, TRS_ERR_UNSUPPORTED (b != 4), TRS_ERR_OOM,
 * TRS_ERR_CUDA. */
trs_status trs_thermal_assemble(trs_bsr *A, const trs_thermal_params *prm, const double *swt, int32_t nswt,
                                const double *slt, int32_t nslt, const double *perm, const double *u,
                                const double *u_old, const uint8_t *gas, const double *wi,
                                const int32_t *well_type, const double *well_target, double *residual,
                                void *stream);

/* --------------------------------------------------------------- misc */
const char *trs_last_error(void);
const char *trs_version(void);

/* Number of CUDA kernels this library has launched in this process (all
 * devices, all threads), for accounting of launch counts. */
uint64_t trs_kernel_launches(void);

/* Device timing of the operator SpMV (w = A z_j) launches inside FGMRES, by
 * CUDA events on the solve's stream.  enable = 1 resets the totals and starts
 * timing; enable = 0 stops.  Either call first returns the totals so far
 * (host pointers, may be NULL).  Process-wide; not for concurrent solves. */
trs_status trs_profile_spmv(int32_t enable, double *total_ms, int64_t *launches);

/* Testing the bounded waits.  The Gram-Schmidt kernels of FGMRES stage their
 * basis tiles through bulk copies completed on mbarriers, and every wait for
 * a tile gives up after a fixed number of polls: the kernel then makes its
 * sums NaN, waits (bounded) for its copies still in flight and returns, and
 * the solve ends with TRS_ERR_NAN.  With extra_bytes > 0 each stage expects
 * that many bytes more than its copies deliver, so every wait runs out (about
 * a second per launch) and that path can be tested; 0 restores normal
 * operation.  Process-wide; extra_bytes must be 0..65536 and a multiple of
 * 16, else TRS_ERR_INVALID. */
trs_status trs_test_stall_staged_copies(int32_t extra_bytes);

#ifdef __cplusplus
}
#endif
#endif
