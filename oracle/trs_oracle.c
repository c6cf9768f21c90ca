/*
 * trs_oracle.c -- plain FP64 CPU oracle (see trs_oracle.h).
 *
 * TEST INFRASTRUCTURE ONLY: used by tests, the smoke check and the CPU
 * baseline leg of the benchmark, never by the product path.
 *
 * Every routine is a direct, sequential statement of the operation it names,
 * written for readability and checked against the paper's definitions and
 * closed forms by the CPU test-suite.  No blocking, fusion or reordering
 * beyond what each definition states.  Compiled with -ffp-contract=off so
 * that a*b+c is always a rounded product followed by a rounded sum.
 *
 * Paper passages followed (Liu & Chen, arXiv 1812.03952):
 *   - block Jacobian numbered cell by cell, wells after cells:
 *     Sec. "Linear Solver" (Eq. mat-ja) and Sec. "Linear System" mapping;
 *   - harmonic-mean geometric transmissibility, zero on boundary faces:
 *     Sec. "Numerical Methods" (transmissibility paragraph);
 *   - Peaceman well term Q = WI * mobility * (p_b - p) and the fixed-rate
 *     well equation sum_m Q_m = c: Sec. "Well Modeling" (Eq. well-model,
 *     fixed-rate constraint);
 *   - decoupling (D^-1 A) x = D^-1 b, ABF D = blockdiag(A_ii), GJE with row
 *     pivoting: Sec. "Decoupling Methods" (Eqs. decoupled-eq, decoupled-abf);
 *   - CPR-FPF: smoother, residual, pressure AMG correction, residual,
 *     smoother: Sec. "Preconditioners" (Algorithm pc-fpf and its prose);
 *   - one AMG V-cycle per application (maxit 1): Fig. fig-ds-amg-par;
 *   - GMRES-type Krylov outer solver: Sec. "Linear Solver".
 * Where the paper is silent (aggregation AMG, Chebyshev smoothing, block
 * ILU(0) with multicolouring, FGMRES with CGS2, adjoint) the routine states
 * the reading it implements.
 */
#include "trs_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_NOT_CONVERGED 1
#define ORC_INVALID (-1)
#define ORC_SINGULAR (-2)
#define ORC_STALLED (-3)
#define ORC_NOMEM (-4)
#define ORC_COLOURS (-5)

#define ORC_MAX_LEVELS 16
#define ORC_DENSE_MAX 4096
#define ORC_MAX_COLOURS 64

/* allocation count that is never zero */
static size_t nz1(int64_t v) { return v > 0 ? (size_t)v : 1; }

/* face directions (dx, dy, dz), ordered by ascending neighbour index */
static const int DIR[6][3] = {{0, 0, -1}, {0, -1, 0}, {-1, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
static int opposite_dir(int d) { return 5 - d; }

/* Binary search of column j in row i of a CSR pattern; -1 if absent. */
static int64_t find_entry(const int64_t *rp, const int32_t *col, int64_t i, int64_t j) {
  int64_t lo = rp[i], hi = rp[i + 1] - 1;
  while (lo <= hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (col[mid] == j) return mid;
    if (col[mid] < j) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

/* murmur3 32-bit finaliser (Appleby, MurmurHash3 "fmix32"); used only to
 * give every node a reproducible pseudo-random priority. */
static uint32_t fmix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}
static uint64_t node_key(int64_t i, uint32_t seed) {
  return ((uint64_t)fmix32((uint32_t)i ^ seed) << 32) | (uint64_t)(uint32_t)i;
}

/* ======================================================================
 * Assembly of the synthetic Newton-step Jacobian.
 *
 * Geometric transmissibility of the face between cells i and j (unit cell
 * size and face area), harmonic mean of the permeabilities, zero when both
 * vanish and zero (no face) on the boundary -- Sec. "Numerical Methods":
 *     T = c_t * (2 k_i k_j) / (k_i + k_j),   k scaled by kv/kh on z faces.
 * The upstream fluid factor of the paper is replaced by a given mobility
 * block M (one per directed face):  A_ij = -T M_ij,  and the cell's own
 * block collects the accumulation block and the opposite of every flux
 * block:  A_ii = Acc_i + sum_j T M_ij   (so a uniform state carries no flux).
 * Wells, from the Peaceman rate Q = WI * lam * (p_bhp - p_cell)
 * (Eq. well-model) and the fixed-rate well equation sum_m Q_m = c:
 *     cell row c:  A_cc(r,0) += WI_m lam_m[r],  A_cw(r,0) = -WI_m lam_m[r];
 *     well row w:  A_ww(0,0) = sum_m WI_m Lam_m,  A_wc(0,0) = -WI_m Lam_m,
 *                  Lam_m = sum_r lam_m[r];  A_ww(s,s) = 1 for s >= 1 (padding).
 * Summation order (fixed): Acc, then the faces in direction order, then the
 * perforations of the cell in ascending perforation index.
 * ====================================================================== */
static double face_transmissibility(const double *k, double kvkh, double c_t, int64_t i,
                                    int64_t j, int vertical) {
  double ki = k[i], kj = k[j];
  if (vertical) { ki = kvkh * ki; kj = kvkh * kj; }
  double den = ki + kj;
  if (den == 0.0) return 0.0;
  double num = (2.0 * ki) * kj;
  return c_t * (num / den);
}

static int64_t neighbour(int nx, int ny, int nz, int64_t c, int d) {
  int64_t x = c % nx, y = (c / nx) % ny, z = c / ((int64_t)nx * ny);
  int64_t X = x + DIR[d][0], Y = y + DIR[d][1], Z = z + DIR[d][2];
  if (X < 0 || X >= nx || Y < 0 || Y >= ny || Z < 0 || Z >= nz) return -1;
  return X + (int64_t)nx * (Y + (int64_t)ny * Z);
}

static int cmp_i32(const void *a, const void *b) {
  int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  return (x > y) - (x < y);
}

/* per-row list of perforation indices, cells first then wells */
typedef struct { int64_t *ptr; int64_t *idx; } perf_lists;

static int build_perf_lists(int64_t n_c, int nw, int64_t np, const int32_t *pw, const int32_t *pc,
                            perf_lists *cell, perf_lists *well) {
  cell->ptr = calloc((size_t)n_c + 1, sizeof(int64_t));
  well->ptr = calloc((size_t)nw + 1, sizeof(int64_t));
  cell->idx = malloc(sizeof(int64_t) * (size_t)(np > 0 ? np : 1));
  well->idx = malloc(sizeof(int64_t) * (size_t)(np > 0 ? np : 1));
  if (!cell->ptr || !well->ptr || !cell->idx || !well->idx) return ORC_NOMEM;
  for (int64_t m = 0; m < np; m++) {
    if (pc[m] < 0 || pc[m] >= n_c || pw[m] < 0 || pw[m] >= nw) return ORC_INVALID;
    cell->ptr[pc[m] + 1]++;
    well->ptr[pw[m] + 1]++;
  }
  for (int64_t i = 0; i < n_c; i++) cell->ptr[i + 1] += cell->ptr[i];
  for (int w = 0; w < nw; w++) well->ptr[w + 1] += well->ptr[w];
  int64_t *fc = calloc((size_t)n_c, sizeof(int64_t));
  int64_t *fw = calloc((size_t)(nw > 0 ? nw : 1), sizeof(int64_t));
  for (int64_t m = 0; m < np; m++) {  /* ascending m within each list */
    cell->idx[cell->ptr[pc[m]] + fc[pc[m]]++] = m;
    well->idx[well->ptr[pw[m]] + fw[pw[m]]++] = m;
  }
  free(fc);
  free(fw);
  return ORC_OK;
}
static void free_perf_lists(perf_lists *a) { free(a->ptr); free(a->idx); }

int64_t orc_assembly_nnzb(int nx, int ny, int nz, int nw, int64_t np, const int32_t *perf_well,
                          const int32_t *perf_cell) {
  int64_t n_c = (int64_t)nx * ny * nz, nnz = 0;
  (void)perf_well; (void)perf_cell;
  for (int64_t c = 0; c < n_c; c++) {
    nnz += 1;
    for (int d = 0; d < 6; d++) nnz += neighbour(nx, ny, nz, c, d) >= 0;
  }
  return nnz + 2 * np + nw;
}

int orc_assemble(int nx, int ny, int nz, int b, const double *k, double kvkh, double c_t,
                 const double *M, const double *acc, int nw, int64_t np,
                 const int32_t *perf_well, const int32_t *perf_cell, const double *wi,
                 const double *lam, int64_t *rp, int32_t *col, double *val) {
  const int64_t n_c = (int64_t)nx * ny * nz, bb = (int64_t)b * b;
  perf_lists pcell, pwell;
  int st = build_perf_lists(n_c, nw, np, perf_well, perf_cell, &pcell, &pwell);
  if (st) return st;
  int64_t pos = 0;
  rp[0] = 0;
  /* cell rows */
  for (int64_t c = 0; c < n_c; c++) {
    int64_t diag_pos = -1;
    /* columns in ascending order: -z,-y,-x, self, +x,+y,+z, then wells */
    for (int d = 0; d < 3; d++) {
      int64_t j = neighbour(nx, ny, nz, c, d);
      if (j >= 0) col[pos++] = (int32_t)j;
    }
    diag_pos = pos;
    col[pos++] = (int32_t)c;
    for (int d = 3; d < 6; d++) {
      int64_t j = neighbour(nx, ny, nz, c, d);
      if (j >= 0) col[pos++] = (int32_t)j;
    }
    int64_t nperf = pcell.ptr[c + 1] - pcell.ptr[c];
    int32_t *wcols = col + pos;
    for (int64_t t = 0; t < nperf; t++) wcols[t] = (int32_t)(n_c + perf_well[pcell.idx[pcell.ptr[c] + t]]);
    qsort(wcols, (size_t)nperf, sizeof(int32_t), cmp_i32);
    for (int64_t t = 1; t < nperf; t++)
      if (wcols[t] == wcols[t - 1]) { free_perf_lists(&pcell); free_perf_lists(&pwell); return ORC_INVALID; }
    pos += nperf;
    rp[c + 1] = pos;
    /* values */
    for (int64_t p = rp[c]; p < rp[c + 1]; p++) memset(val + p * bb, 0, sizeof(double) * (size_t)bb);
    double *Aii = val + diag_pos * bb;
    memcpy(Aii, acc + c * bb, sizeof(double) * (size_t)bb);
    for (int d = 0; d < 6; d++) {
      int64_t j = neighbour(nx, ny, nz, c, d);
      if (j < 0) continue;
      double T = face_transmissibility(k, kvkh, c_t, c, j, d == 0 || d == 5);
      const double *Mij = M + (c * 6 + d) * bb;
      int64_t p = find_entry(rp, col, c, j);
      for (int64_t e = 0; e < bb; e++) {
        double flux = T * Mij[e];
        val[p * bb + e] = -flux;
        Aii[e] = Aii[e] + flux;
      }
    }
    for (int64_t t = pcell.ptr[c]; t < pcell.ptr[c + 1]; t++) {
      int64_t m = pcell.idx[t];
      int64_t p = find_entry(rp, col, c, n_c + perf_well[m]);
      for (int r = 0; r < b; r++) {
        double q = wi[m] * lam[m * b + r];
        Aii[r * b + 0] = Aii[r * b + 0] + q;
        val[p * bb + r * b + 0] = -q;
      }
    }
  }
  /* well rows */
  for (int w = 0; w < nw; w++) {
    int64_t row = n_c + w, start = pos;
    int64_t nperf = pwell.ptr[w + 1] - pwell.ptr[w];
    for (int64_t t = 0; t < nperf; t++) col[pos++] = perf_cell[pwell.idx[pwell.ptr[w] + t]];
    col[pos++] = (int32_t)row;
    qsort(col + start, (size_t)(pos - start), sizeof(int32_t), cmp_i32);
    rp[row + 1] = pos;
    for (int64_t p = start; p < pos; p++) memset(val + p * bb, 0, sizeof(double) * (size_t)bb);
    int64_t dp = find_entry(rp, col, row, row);
    double *Aww = val + dp * bb;
    double sum = 0.0;
    for (int64_t t = pwell.ptr[w]; t < pwell.ptr[w + 1]; t++) {
      int64_t m = pwell.idx[t];
      double Lam = 0.0;
      for (int r = 0; r < b; r++) Lam = Lam + lam[m * b + r];
      double q = wi[m] * Lam;
      sum = sum + q;
      int64_t p = find_entry(rp, col, row, perf_cell[m]);
      val[p * bb] = -q;
    }
    Aww[0] = sum;
    for (int s = 1; s < b; s++) Aww[s * b + s] = 1.0;
  }
  free_perf_lists(&pcell);
  free_perf_lists(&pwell);
  return ORC_OK;
}

/* ======================================================================
 * Block sparse matrix-vector products (sparse BLAS of Sec. "Linear Solver";
 * y = a*A*x + b*y of Fig. fig-mv).  Row sums in ascending column order.
 * ====================================================================== */
void orc_bsr_spmv(int64_t n, int b, const int64_t *rp, const int32_t *col, const double *val,
                  const double *x, double *y, double alpha, double beta) {
  const int64_t bb = (int64_t)b * b;
  double *acc = malloc(sizeof(double) * (size_t)b);
  for (int64_t i = 0; i < n; i++) {
    for (int r = 0; r < b; r++) acc[r] = 0.0;
    for (int64_t p = rp[i]; p < rp[i + 1]; p++) {
      const double *blk = val + p * bb, *xj = x + (int64_t)col[p] * b;
      for (int r = 0; r < b; r++)
        for (int s = 0; s < b; s++) acc[r] = acc[r] + blk[r * b + s] * xj[s];
    }
    for (int r = 0; r < b; r++) {
      double yi = (beta == 0.0) ? 0.0 : beta * y[i * b + r];
      y[i * b + r] = alpha * acc[r] + yi;
    }
  }
  free(acc);
}

void orc_bsr_spmv_t(int64_t n, int b, const int64_t *rp, const int32_t *col, const double *val,
                    const double *x, double *y, double alpha, double beta) {
  const int64_t bb = (int64_t)b * b;
  double *t = calloc((size_t)(n * b), sizeof(double));
  for (int64_t i = 0; i < n; i++)
    for (int64_t p = rp[i]; p < rp[i + 1]; p++) {
      const double *blk = val + p * bb, *xi = x + i * b;
      double *tj = t + (int64_t)col[p] * b;
      for (int s = 0; s < b; s++)
        for (int r = 0; r < b; r++) tj[s] = tj[s] + blk[r * b + s] * xi[r];
    }
  for (int64_t e = 0; e < n * b; e++) {
    double yi = (beta == 0.0) ? 0.0 : beta * y[e];
    y[e] = alpha * t[e] + yi;
  }
  free(t);
}

/* (A^T)_ij = (A_ji)^T, rows of the transpose with sorted columns. */
int orc_bsr_transpose(int64_t n, int b, const int64_t *rp, const int32_t *col, const double *val,
                      int64_t *rpT, int32_t *colT, double *valT) {
  const int64_t bb = (int64_t)b * b;
  for (int64_t i = 0; i <= n; i++) rpT[i] = 0;
  for (int64_t p = 0; p < rp[n]; p++) {
    if (col[p] < 0 || col[p] >= n) return ORC_INVALID;
    rpT[col[p] + 1]++;
  }
  for (int64_t i = 0; i < n; i++) rpT[i + 1] += rpT[i];
  int64_t *fill = calloc((size_t)n, sizeof(int64_t));
  for (int64_t i = 0; i < n; i++)           /* ascending i => sorted columns */
    for (int64_t p = rp[i]; p < rp[i + 1]; p++) {
      int64_t j = col[p], q = rpT[j] + fill[j]++;
      colT[q] = (int32_t)i;
      for (int r = 0; r < b; r++)
        for (int s = 0; s < b; s++) valT[q * bb + s * b + r] = val[p * bb + r * b + s];
    }
  free(fill);
  return ORC_OK;
}

int orc_pattern_symmetric(int64_t n, const int64_t *rp, const int32_t *col) {
  for (int64_t i = 0; i < n; i++)
    for (int64_t p = rp[i]; p < rp[i + 1]; p++)
      if (find_entry(rp, col, col[p], i) < 0) return 0;
  return 1;
}

/* ======================================================================
 * Decoupling, Sec. "Decoupling Methods".
 *
 * Gauss-Jordan elimination on [D | I] with row pivoting only (GJE): at
 * column c the pivot row is the one of largest |D(r,c)|, r >= c, the first
 * such row on ties; the pivot row is scaled by the reciprocal of the pivot
 * (one division per column), then the multiple D(r,c) of it is subtracted
 * from every other row.  The right half
 * becomes D^-1.  ABF (Eq. decoupled-abf) uses D_i = A_ii; the decoupled
 * blocks are  Ã_ij = D_i^-1 A_ij, with Ã_ii set to the identity.  The
 * products sum over the inner index in ascending order.
 * ====================================================================== */
int orc_gj_inverse(int b, const double *D, double *inv) {
  double a[64], m[64];
  if (b < 1 || b > 8) return ORC_INVALID;
  for (int e = 0; e < b * b; e++) { a[e] = D[e]; m[e] = 0.0; }
  for (int r = 0; r < b; r++) m[r * b + r] = 1.0;
  for (int c = 0; c < b; c++) {
    int p = c;
    double best = fabs(a[c * b + c]);
    for (int r = c + 1; r < b; r++)
      if (fabs(a[r * b + c]) > best) { best = fabs(a[r * b + c]); p = r; }
    if (best == 0.0 || !isfinite(best)) return ORC_SINGULAR;
    if (p != c)
      for (int s = 0; s < b; s++) {
        double t = a[c * b + s]; a[c * b + s] = a[p * b + s]; a[p * b + s] = t;
        t = m[c * b + s]; m[c * b + s] = m[p * b + s]; m[p * b + s] = t;
      }
    const double rpiv = 1.0 / a[c * b + c];
    for (int s = 0; s < b; s++) { a[c * b + s] = a[c * b + s] * rpiv; m[c * b + s] = m[c * b + s] * rpiv; }
    for (int r = 0; r < b; r++) {
      if (r == c) continue;
      double f = a[r * b + c];
      for (int s = 0; s < b; s++) {
        a[r * b + s] = a[r * b + s] - f * a[c * b + s];
        m[r * b + s] = m[r * b + s] - f * m[c * b + s];
      }
    }
  }
  for (int e = 0; e < b * b; e++) inv[e] = m[e];
  return ORC_OK;
}

/* C = A * B for b x b row-major blocks, inner index ascending */
static void block_mul(int b, const double *A, const double *B, double *C) {
  for (int r = 0; r < b; r++)
    for (int s = 0; s < b; s++) {
      double acc = A[r * b] * B[s];
      for (int t = 1; t < b; t++) acc = acc + A[r * b + t] * B[t * b + s];
      C[r * b + s] = acc;
    }
}

static void block_vec(int b, const double *A, const double *x, double *y) {
  for (int r = 0; r < b; r++) {
    double acc = A[r * b] * x[0];
    for (int t = 1; t < b; t++) acc = acc + A[r * b + t] * x[t];
    y[r] = acc;
  }
}

/* Decoupling D^-1 A of Eq. decoupled-eq, block row by block row, with the
 * left factor D_i^-1 chosen by `mode` (Sec. "Decoupling Methods"):
 *   ORC_DEC_ABF      D_i^-1 = A_ii^-1 (Eq. decoupled-abf; the inverse by
 *                    Gauss-Jordan elimination with partial row pivoting, so
 *                    the same operator also serves for GJE); Ã_ii = I exactly;
 *   ORC_DEC_NONE     D_i^-1 = I, Ã = A;
 *   ORC_DEC_FRS      D_i^-1 = R (Eq. decoupled-frs: ones in the first row and
 *                    on the diagonal), which adds every row into the pressure
 *                    row;
 *   ORC_DEC_FRS_ABF  the two-stage FRS+ABF: A' = R A, then ABF of A', so
 *                    D_i^-1 = (R A_ii)^-1 R and Ã_ii = I exactly.
 * Every product is block_mul (inner index ascending). */
int orc_decouple_mode(int64_t n, int b, const int64_t *rp, const int32_t *col, const double *val,
                      int mode, double *vt, double *dinv) {
  if (mode < ORC_DEC_ABF || mode > ORC_DEC_FRS_ABF || b < 1 || b > ORC_MAX_B) return ORC_INVALID;
  const int64_t bb = (int64_t)b * b;
  double R[ORC_MAX_B * ORC_MAX_B], Ai[ORC_MAX_B * ORC_MAX_B], Rd[ORC_MAX_B * ORC_MAX_B];
  for (int r = 0; r < b; r++)
    for (int c = 0; c < b; c++) R[r * b + c] = (r == 0 || r == c) ? 1.0 : 0.0;
  const int unit = (mode == ORC_DEC_ABF || mode == ORC_DEC_FRS_ABF);
  for (int64_t i = 0; i < n; i++) {
    int64_t dp = find_entry(rp, col, i, i);
    if (dp < 0) return ORC_INVALID;
    double *Di = dinv + i * bb;
    if (mode == ORC_DEC_NONE) {
      for (int e = 0; e < bb; e++) Di[e] = (e % (b + 1) == 0) ? 1.0 : 0.0;
    } else if (mode == ORC_DEC_FRS) {
      for (int e = 0; e < bb; e++) Di[e] = R[e];
    } else if (mode == ORC_DEC_ABF) {
      int st = orc_gj_inverse(b, val + dp * bb, Di);
      if (st) return st;
    } else {
      block_mul(b, R, val + dp * bb, Rd);
      int st = orc_gj_inverse(b, Rd, Ai);
      if (st) return st;
      block_mul(b, Ai, R, Di);
    }
    for (int64_t p = rp[i]; p < rp[i + 1]; p++) {
      if (p == dp && unit) {
        for (int e = 0; e < bb; e++) vt[p * bb + e] = 0.0;
        for (int r = 0; r < b; r++) vt[p * bb + r * b + r] = 1.0;
      } else if (mode == ORC_DEC_FRS_ABF) {
        block_mul(b, R, val + p * bb, Rd);
        block_mul(b, Ai, Rd, vt + p * bb);
      } else {
        block_mul(b, Di, val + p * bb, vt + p * bb);
      }
    }
  }
  return ORC_OK;
}

int orc_decouple(int64_t n, int b, const int64_t *rp, const int32_t *col, const double *val,
                 double *vt, double *dinv) {
  return orc_decouple_mode(n, b, rp, col, val, ORC_DEC_ABF, vt, dinv);
}

/* Pressure matrix A_PP of Algorithm pc-fpf: entry (0,0) of every decoupled
 * block (the BHP is entry 0 of a padded well block). */
void orc_pressure_matrix(int64_t n, int b, const int64_t *rp, const int32_t *col,
                         const double *vt, double *ap) {
  (void)col;
  const int64_t bb = (int64_t)b * b;
  for (int64_t p = 0; p < rp[n]; p++) ap[p] = vt[p * bb];
}

/* ======================================================================
 * Pressure AMG.  The paper uses BoomerAMG (Fig. fig-ds-amg-par) and keeps
 * one V-cycle per preconditioner application.  The reading implemented
 * here is unsmoothed aggregation:
 *   strength: j != i is strong when s_ij = max(|a_ij|, |a_ji|) > 0 and
 *     s_ij >= theta * sqrt(|a_ii * a_jj|)  (a_ji = 0 if not stored);
 *   MIS-2 of the strength graph by synchronous rounds of two max-sweeps of
 *     the tuple (state, key), states OUT < UNDECIDED < IN, key_i =
 *     fmix32(i ^ seed) << 32 | i; nodes without strong neighbours are left
 *     out of the coarse space (zero row of P);
 *   aggregates: roots numbered in index order; a root's strong neighbours
 *     join it; every other node joins, among its strong neighbours that
 *     joined in that first pass, the one of largest |a_ij| (smaller
 *     aggregate id on ties);
 *   A_c = P^T A P with P piecewise constant: A_c[I][J] = running sum, over
 *     fine rows i of I in ascending order and their stored entries in
 *     ascending column order with agg[col] = J, starting from 0.0;
 *   coarsen while n > coarse_max, fewer than max_levels levels, and
 *     n_coarse < 0.9 n; the coarsest matrix is solved by dense LU;
 *   smoothing: Chebyshev polynomial of D^-1 A (Saad, "Iterative Methods for
 *     Sparse Linear Systems", Alg. 12.1) on [0.3 lam, lam], lam = max_i
 *     (sum_j |a_ij|) / |a_ii| (Gershgorin), one pre- and one post-sweep.
 * ====================================================================== */
static double diag_of(const int64_t *rp, const int32_t *col, const double *val, int64_t i) {
  int64_t p = find_entry(rp, col, i, i);
  return p < 0 ? 0.0 : val[p];
}

int64_t orc_strength(int64_t n, const int64_t *rp, const int32_t *col, const double *val,
                     double theta, int64_t *srp, int32_t *scol) {
  int64_t q = 0;
  srp[0] = 0;
  for (int64_t i = 0; i < n; i++) {
    double aii = diag_of(rp, col, val, i);
    for (int64_t p = rp[i]; p < rp[i + 1]; p++) {
      int64_t j = col[p];
      if (j == i) continue;
      double ajj = diag_of(rp, col, val, j);
      int64_t pt = find_entry(rp, col, j, i);
      double aij = fabs(val[p]), aji = pt < 0 ? 0.0 : fabs(val[pt]);
      double s = aij > aji ? aij : aji;
      double thr = theta * sqrt(fabs(aii * ajj));
      if (s > 0.0 && s >= thr) scol[q++] = (int32_t)j;
    }
    srp[i + 1] = q;
  }
  return q;
}

enum { ST_OUT = 0, ST_UNDECIDED = 1, ST_IN = 2 };

typedef struct { int8_t s; uint64_t key; } tuple_t;
static int tuple_gt(tuple_t a, tuple_t b) { return a.s > b.s || (a.s == b.s && a.key > b.key); }

int orc_mis2(int64_t n, const int64_t *srp, const int32_t *scol, uint32_t seed, int8_t *state) {
  tuple_t *t0 = malloc(sizeof(tuple_t) * nz1(n));
  tuple_t *t1 = malloc(sizeof(tuple_t) * nz1(n));
  tuple_t *t2 = malloc(sizeof(tuple_t) * nz1(n));
  for (int64_t i = 0; i < n; i++) state[i] = (srp[i + 1] > srp[i]) ? ST_UNDECIDED : ST_OUT;
  int rounds = 0;
  for (;;) {
    int64_t undecided = 0;
    for (int64_t i = 0; i < n; i++) undecided += state[i] == ST_UNDECIDED;
    if (!undecided) break;
    rounds++;
    for (int64_t i = 0; i < n; i++) { t0[i].s = state[i]; t0[i].key = node_key(i, seed); }
    for (int64_t i = 0; i < n; i++) {
      tuple_t m = t0[i];
      for (int64_t p = srp[i]; p < srp[i + 1]; p++) if (tuple_gt(t0[scol[p]], m)) m = t0[scol[p]];
      t1[i] = m;
    }
    for (int64_t i = 0; i < n; i++) {
      tuple_t m = t1[i];
      for (int64_t p = srp[i]; p < srp[i + 1]; p++) if (tuple_gt(t1[scol[p]], m)) m = t1[scol[p]];
      t2[i] = m;
    }
    for (int64_t i = 0; i < n; i++) {
      if (state[i] != ST_UNDECIDED) continue;
      if (t2[i].s == t0[i].s && t2[i].key == t0[i].key) state[i] = ST_IN;
      else if (t2[i].s == ST_IN) state[i] = ST_OUT;
    }
  }
  free(t0); free(t1); free(t2);
  return rounds;
}

int64_t orc_aggregate(int64_t n, const int64_t *rp, const int32_t *col, const double *val,
                      const int64_t *srp, const int32_t *scol, const int8_t *state, int32_t *agg) {
  int64_t n_agg = 0;
  for (int64_t i = 0; i < n; i++) agg[i] = (state[i] == ST_IN) ? (int32_t)(n_agg++) : -1;
  /* pass 1: strong neighbours of a root join it */
  int32_t *first = malloc(sizeof(int32_t) * nz1(n));
  for (int64_t i = 0; i < n; i++) {
    first[i] = agg[i];
    if (agg[i] >= 0) continue;
    for (int64_t p = srp[i]; p < srp[i + 1]; p++)
      if (state[scol[p]] == ST_IN) { first[i] = agg[scol[p]]; break; }
  }
  /* pass 2: the rest join the first-pass neighbour of largest |a_ij| */
  for (int64_t i = 0; i < n; i++) {
    agg[i] = first[i];
    if (first[i] >= 0 || srp[i + 1] == srp[i]) continue;
    double best = -1.0;
    int32_t pick = -1;
    for (int64_t p = srp[i]; p < srp[i + 1]; p++) {
      int64_t j = scol[p];
      if (first[j] < 0) continue;
      double a = fabs(val[find_entry(rp, col, i, j)]);
      if (a > best || (a == best && first[j] < pick)) { best = a; pick = first[j]; }
    }
    agg[i] = pick;
  }
  free(first);
  return n_agg;
}

static void members_of(int64_t n, const int32_t *agg, int64_t n_agg, int64_t **mptr, int64_t **midx) {
  int64_t *ptr = calloc((size_t)n_agg + 1, sizeof(int64_t));
  for (int64_t i = 0; i < n; i++) if (agg[i] >= 0) ptr[agg[i] + 1]++;
  for (int64_t a = 0; a < n_agg; a++) ptr[a + 1] += ptr[a];
  int64_t *idx = malloc(sizeof(int64_t) * nz1(ptr[n_agg]));
  int64_t *f = calloc((size_t)n_agg + 1, sizeof(int64_t));
  for (int64_t i = 0; i < n; i++) if (agg[i] >= 0) idx[ptr[agg[i]] + f[agg[i]]++] = i;
  free(f);
  *mptr = ptr;
  *midx = idx;
}

/* Shared walk for the count and the fill of P^T A P. */
static int64_t galerkin_walk(int64_t n, const int64_t *rp, const int32_t *col, const double *val,
                             const int32_t *agg, int64_t n_agg, int64_t *crp, int32_t *ccol,
                             double *cval) {
  int64_t *mptr, *midx;
  members_of(n, agg, n_agg, &mptr, &midx);
  double *acc = calloc(nz1(n_agg), sizeof(double));
  int64_t *mark = malloc(sizeof(int64_t) * nz1(n_agg));
  int32_t *touched = malloc(sizeof(int32_t) * nz1(n_agg));
  for (int64_t a = 0; a < n_agg; a++) mark[a] = -1;
  int64_t nnz = 0;
  if (crp) crp[0] = 0;
  for (int64_t I = 0; I < n_agg; I++) {
    int64_t nt = 0;
    for (int64_t t = mptr[I]; t < mptr[I + 1]; t++) {
      int64_t i = midx[t];
      for (int64_t p = rp[i]; p < rp[i + 1]; p++) {
        int32_t J = agg[col[p]];
        if (J < 0) continue;
        if (mark[J] != I) { mark[J] = I; acc[J] = 0.0; touched[nt++] = J; }
        if (val) acc[J] = acc[J] + val[p];
      }
    }
    qsort(touched, (size_t)nt, sizeof(int32_t), cmp_i32);
    if (ccol)
      for (int64_t t = 0; t < nt; t++) { ccol[nnz + t] = touched[t]; cval[nnz + t] = acc[touched[t]]; }
    nnz += nt;
    if (crp) crp[I + 1] = nnz;
  }
  free(mptr); free(midx); free(acc); free(mark); free(touched);
  return nnz;
}

int64_t orc_galerkin_nnz(int64_t n, const int64_t *rp, const int32_t *col, const int32_t *agg,
                         int64_t n_agg) {
  return galerkin_walk(n, rp, col, NULL, agg, n_agg, NULL, NULL, NULL);
}

void orc_galerkin(int64_t n, const int64_t *rp, const int32_t *col, const double *val,
                  const int32_t *agg, int64_t n_agg, int64_t *crp, int32_t *ccol, double *cval) {
  galerkin_walk(n, rp, col, val, agg, n_agg, crp, ccol, cval);
}

double orc_gershgorin(int64_t n, const int64_t *rp, const int32_t *col, const double *val) {
  double lam = 0.0;
  for (int64_t i = 0; i < n; i++) {
    double s = 0.0;
    for (int64_t p = rp[i]; p < rp[i + 1]; p++) s = s + fabs(val[p]);
    double q = s / fabs(diag_of(rp, col, val, i));
    if (q > lam) lam = q;
  }
  return lam;
}

static void csr_residual(int64_t n, const int64_t *rp, const int32_t *col, const double *val,
                         const double *r, const double *e, double *res) {
  for (int64_t i = 0; i < n; i++) {
    double s = 0.0;
    for (int64_t p = rp[i]; p < rp[i + 1]; p++) s = s + val[p] * e[col[p]];
    res[i] = r[i] - s;
  }
}

/* Chebyshev acceleration of the Jacobi iteration for A e = r (Saad, Alg.
 * 12.1 applied to D^-1 A on [alpha, beta] = [0.3 lam, lam]), `degree`
 * corrections starting from e (or from e = 0 when zero_init). */
void orc_chebyshev(int64_t n, const int64_t *rp, const int32_t *col, const double *val,
                   double lam_max, int degree, const double *r, double *e, int zero_init) {
  double alpha = 0.3 * lam_max, beta = lam_max;
  double theta = (beta + alpha) / 2.0, delta = (beta - alpha) / 2.0;
  double sigma = theta / delta, rho = 1.0 / sigma;
  double *res = malloc(sizeof(double) * nz1(n));
  double *d = malloc(sizeof(double) * nz1(n));
  double *dinv = malloc(sizeof(double) * nz1(n));
  double *ad = malloc(sizeof(double) * nz1(n));
  for (int64_t i = 0; i < n; i++) dinv[i] = 1.0 / diag_of(rp, col, val, i);
  if (zero_init) {
    for (int64_t i = 0; i < n; i++) { e[i] = 0.0; res[i] = r[i]; }
  } else {
    csr_residual(n, rp, col, val, r, e, res);
  }
  for (int64_t i = 0; i < n; i++) d[i] = (dinv[i] * res[i]) / theta;
  for (int k = 1; k <= degree; k++) {
    for (int64_t i = 0; i < n; i++) e[i] = e[i] + d[i];
    if (k == degree) break;
    for (int64_t i = 0; i < n; i++) {
      double s = 0.0;
      for (int64_t p = rp[i]; p < rp[i + 1]; p++) s = s + val[p] * d[col[p]];
      ad[i] = s;
    }
    for (int64_t i = 0; i < n; i++) res[i] = res[i] - ad[i];
    double rho_new = 1.0 / (2.0 * sigma - rho);
    double c1 = rho_new * rho, c2 = (2.0 * rho_new) / delta;
    for (int64_t i = 0; i < n; i++) d[i] = c1 * d[i] + c2 * (dinv[i] * res[i]);
    rho = rho_new;
  }
  free(res); free(d); free(dinv); free(ad);
}

/* Dense LU with partial pivoting (row of largest |a|, first on ties). */
int orc_dense_lu(int64_t n, double *a, int32_t *piv) {
  for (int64_t k = 0; k < n; k++) {
    int64_t p = k;
    double best = fabs(a[k * n + k]);
    for (int64_t i = k + 1; i < n; i++)
      if (fabs(a[i * n + k]) > best) { best = fabs(a[i * n + k]); p = i; }
    if (best == 0.0 || !isfinite(best)) return ORC_SINGULAR;
    piv[k] = (int32_t)p;
    if (p != k)
      for (int64_t j = 0; j < n; j++) { double t = a[k * n + j]; a[k * n + j] = a[p * n + j]; a[p * n + j] = t; }
    for (int64_t i = k + 1; i < n; i++) {
      double l = a[i * n + k] / a[k * n + k];
      a[i * n + k] = l;
      for (int64_t j = k + 1; j < n; j++) a[i * n + j] = a[i * n + j] - l * a[k * n + j];
    }
  }
  return ORC_OK;
}

void orc_dense_lu_solve(int64_t n, const double *lu, const int32_t *piv, double *x) {
  for (int64_t k = 0; k < n; k++)
    if (piv[k] != k) { double t = x[k]; x[k] = x[piv[k]]; x[piv[k]] = t; }
  for (int64_t i = 0; i < n; i++) {
    double s = x[i];
    for (int64_t j = 0; j < i; j++) s = s - lu[i * n + j] * x[j];
    x[i] = s;
  }
  for (int64_t i = n - 1; i >= 0; i--) {
    double s = x[i];
    for (int64_t j = i + 1; j < n; j++) s = s - lu[i * n + j] * x[j];
    x[i] = s / lu[i * n + i];
  }
}

typedef struct {
  int64_t n;
  int64_t *rp;
  int32_t *col;
  double *val;
  int32_t *agg;    /* NULL on the coarsest level */
  int64_t n_agg;
  double lam;
} orc_level;

typedef struct {
  int nlev;
  int cheb_degree;
  orc_level lev[ORC_MAX_LEVELS];
  double *lu;
  int32_t *piv;
} orc_amg;

void orc_amg_free(void *hv) {
  orc_amg *h = hv;
  if (!h) return;
  for (int l = 0; l < h->nlev; l++) {
    free(h->lev[l].rp); free(h->lev[l].col); free(h->lev[l].val); free(h->lev[l].agg);
  }
  free(h->lu); free(h->piv); free(h);
}

void *orc_amg_setup(int64_t n, const int64_t *rp, const int32_t *col, const double *val,
                    double theta, int coarse_max, int max_levels, int cheb_degree, uint32_t seed,
                    int *status) {
  orc_amg *h = calloc(1, sizeof(orc_amg));
  *status = ORC_OK;
  if (max_levels < 1 || max_levels > ORC_MAX_LEVELS) max_levels = ORC_MAX_LEVELS;
  h->cheb_degree = cheb_degree;
  int64_t nnz = rp[n];
  orc_level *L0 = &h->lev[0];
  L0->n = n;
  L0->rp = malloc(sizeof(int64_t) * (size_t)(n + 1));
  L0->col = malloc(sizeof(int32_t) * nz1(nnz));
  L0->val = malloc(sizeof(double) * nz1(nnz));
  memcpy(L0->rp, rp, sizeof(int64_t) * (size_t)(n + 1));
  memcpy(L0->col, col, sizeof(int32_t) * (size_t)nnz);
  memcpy(L0->val, val, sizeof(double) * (size_t)nnz);
  h->nlev = 1;
  for (int l = 0;; l++) {
    orc_level *F = &h->lev[l];
    F->lam = orc_gershgorin(F->n, F->rp, F->col, F->val);
    if (F->n <= coarse_max || l + 1 >= max_levels) break;
    int64_t fnnz = F->rp[F->n];
    int64_t *srp = malloc(sizeof(int64_t) * (size_t)(F->n + 1));
    int32_t *scol = malloc(sizeof(int32_t) * nz1(fnnz));
    int8_t *state = malloc(nz1(F->n));
    int32_t *agg = malloc(sizeof(int32_t) * nz1(F->n));
    orc_strength(F->n, F->rp, F->col, F->val, theta, srp, scol);
    orc_mis2(F->n, srp, scol, seed ^ (0x9E3779B9u * (uint32_t)(l + 1)), state);
    int64_t n_agg = orc_aggregate(F->n, F->rp, F->col, F->val, srp, scol, state, agg);
    free(srp); free(scol); free(state);
    if (n_agg == 0 || 10 * n_agg >= 9 * F->n) { free(agg); break; }
    F->agg = agg;
    F->n_agg = n_agg;
    orc_level *C = &h->lev[l + 1];
    int64_t cnnz = orc_galerkin_nnz(F->n, F->rp, F->col, agg, n_agg);
    C->n = n_agg;
    C->rp = malloc(sizeof(int64_t) * (size_t)(n_agg + 1));
    C->col = malloc(sizeof(int32_t) * nz1(cnnz));
    C->val = malloc(sizeof(double) * nz1(cnnz));
    orc_galerkin(F->n, F->rp, F->col, F->val, agg, n_agg, C->rp, C->col, C->val);
    h->nlev = l + 2;
  }
  orc_level *Lc = &h->lev[h->nlev - 1];
  if (Lc->n > ORC_DENSE_MAX) { *status = ORC_STALLED; orc_amg_free(h); return NULL; }
  h->lu = calloc(nz1(Lc->n * Lc->n), sizeof(double));
  h->piv = malloc(sizeof(int32_t) * nz1(Lc->n));
  for (int64_t i = 0; i < Lc->n; i++)
    for (int64_t p = Lc->rp[i]; p < Lc->rp[i + 1]; p++) h->lu[i * Lc->n + Lc->col[p]] = Lc->val[p];
  int st = orc_dense_lu(Lc->n, h->lu, h->piv);
  if (st) { *status = st; orc_amg_free(h); return NULL; }
  return h;
}

int orc_amg_levels(const void *hv) { return ((const orc_amg *)hv)->nlev; }
int64_t orc_amg_level_n(const void *hv, int l) { return ((const orc_amg *)hv)->lev[l].n; }
int64_t orc_amg_level_nnz(const void *hv, int l) {
  const orc_level *L = &((const orc_amg *)hv)->lev[l];
  return L->rp[L->n];
}
void orc_amg_level_copy(const void *hv, int l, int64_t *rp, int32_t *col, double *val) {
  const orc_level *L = &((const orc_amg *)hv)->lev[l];
  memcpy(rp, L->rp, sizeof(int64_t) * (size_t)(L->n + 1));
  memcpy(col, L->col, sizeof(int32_t) * (size_t)L->rp[L->n]);
  memcpy(val, L->val, sizeof(double) * (size_t)L->rp[L->n]);
}
void orc_amg_level_agg(const void *hv, int l, int32_t *agg) {
  const orc_level *L = &((const orc_amg *)hv)->lev[l];
  if (L->agg) memcpy(agg, L->agg, sizeof(int32_t) * (size_t)L->n);
}
double orc_amg_level_lambda(const void *hv, int l) { return ((const orc_amg *)hv)->lev[l].lam; }

/* One V-cycle for A_0 e = r from e = 0: pre-smooth, residual, restrict
 * (r_c[I] = sum over members of I in ascending order), recurse, prolong
 * (e_i += e_c[agg_i]), post-smooth; dense LU solve on the coarsest level. */
static void vcycle_level(const orc_amg *h, int l, const double *r, double *e) {
  const orc_level *L = &h->lev[l];
  if (l == h->nlev - 1) {
    memcpy(e, r, sizeof(double) * (size_t)L->n);
    orc_dense_lu_solve(L->n, h->lu, h->piv, e);
    return;
  }
  orc_chebyshev(L->n, L->rp, L->col, L->val, L->lam, h->cheb_degree, r, e, 1);
  double *res = malloc(sizeof(double) * (size_t)L->n);
  csr_residual(L->n, L->rp, L->col, L->val, r, e, res);
  double *rc = calloc((size_t)L->n_agg, sizeof(double));
  double *ec = calloc((size_t)L->n_agg, sizeof(double));
  for (int64_t i = 0; i < L->n; i++)     /* ascending i: members in order */
    if (L->agg[i] >= 0) rc[L->agg[i]] = rc[L->agg[i]] + res[i];
  vcycle_level(h, l + 1, rc, ec);
  for (int64_t i = 0; i < L->n; i++)
    if (L->agg[i] >= 0) e[i] = e[i] + ec[L->agg[i]];
  orc_chebyshev(L->n, L->rp, L->col, L->val, L->lam, h->cheb_degree, r, e, 0);
  free(res); free(rc); free(ec);
}

void orc_amg_vcycle(const void *hv, const double *r, double *e) { vcycle_level(hv, 0, r, e); }

/* ======================================================================
 * Multicolouring (Jones-Plassmann with first-fit colours) of the block
 * pattern, and block ILU(0) in colour-major order.  The paper's "F" stage
 * is RAS with ILUT/ILU(k) subdomain solves (Sec. "Preconditioners"); the
 * reading here is a single-domain block ILU(0) made parallel by a
 * multicolour ordering:
 *   colouring: in every synchronous round, each uncoloured node whose key
 *     beats the keys of all its uncoloured neighbours takes the smallest
 *     colour not used by an already coloured neighbour;
 *   order: rows sorted by (colour, index);
 *   ILU(0) (IKJ form) restricted to the block pattern: for row i, for each
 *     earlier-ordered k of the row in ascending order, L_ik = W_ik U_kk^-1,
 *     then W_ij -= L_ik U_kj for every later-ordered j of row i with
 *     (k, j) stored; U_ii^-1 is kept (Gauss-Jordan inverse).
 * ====================================================================== */
int orc_colour_jp(int64_t n, const int64_t *rp, const int32_t *col, uint32_t seed, int32_t *colour) {
  int8_t *ready = malloc(nz1(n));
  for (int64_t i = 0; i < n; i++) colour[i] = -1;
  int64_t left = n;
  int ncol = 0;
  while (left > 0) {
    for (int64_t i = 0; i < n; i++) {
      ready[i] = 0;
      if (colour[i] >= 0) continue;
      uint64_t ki = node_key(i, seed);
      int ok = 1;
      for (int64_t p = rp[i]; p < rp[i + 1] && ok; p++) {
        int64_t j = col[p];
        if (j != i && colour[j] < 0 && node_key(j, seed) > ki) ok = 0;
      }
      ready[i] = (int8_t)ok;
    }
    for (int64_t i = 0; i < n; i++) {
      if (!ready[i]) continue;
      uint64_t used = 0;
      for (int64_t p = rp[i]; p < rp[i + 1]; p++) {
        int64_t j = col[p];
        if (j != i && colour[j] >= 0) used |= (uint64_t)1 << colour[j];
      }
      int c = 0;
      while (c < ORC_MAX_COLOURS && (used >> c) & 1) c++;
      if (c >= ORC_MAX_COLOURS) { free(ready); return ORC_COLOURS; }
      colour[i] = c;
      if (c + 1 > ncol) ncol = c + 1;
      left--;
    }
  }
  free(ready);
  return ncol;
}

typedef struct {
  int64_t n;
  int b;
  const int64_t *rp;  /* borrowed from the owner of the pattern */
  const int32_t *col;
  int64_t *rp_own;
  int32_t *col_own;
  double *F;          /* L_ij / U_ij per stored entry, U_ii^-1 on the diagonal */
  int64_t *pos;       /* position of each row in the colour-major order */
  int64_t *order;     /* rows in colour-major order */
} orc_ilu;

void orc_bilu0_free(void *hv) {
  orc_ilu *h = hv;
  if (!h) return;
  free(h->rp_own); free(h->col_own); free(h->F); free(h->pos); free(h->order); free(h);
}

typedef struct { int64_t key; int64_t p; } kp_t;
static int cmp_kp(const void *a, const void *b) {
  int64_t x = ((const kp_t *)a)->key, y = ((const kp_t *)b)->key;
  return (x > y) - (x < y);
}

void *orc_bilu0_setup(int64_t n, int b, const int64_t *rp, const int32_t *col, const double *vt,
                      const int32_t *colour, int *status) {
  const int64_t bb = (int64_t)b * b, nnz = rp[n];
  orc_ilu *h = calloc(1, sizeof(orc_ilu));
  *status = ORC_OK;
  h->n = n; h->b = b;
  h->rp_own = malloc(sizeof(int64_t) * (size_t)(n + 1));
  h->col_own = malloc(sizeof(int32_t) * nz1(nnz));
  memcpy(h->rp_own, rp, sizeof(int64_t) * (size_t)(n + 1));
  memcpy(h->col_own, col, sizeof(int32_t) * (size_t)nnz);
  h->rp = h->rp_own; h->col = h->col_own;
  h->F = malloc(sizeof(double) * nz1(nnz * bb));
  memcpy(h->F, vt, sizeof(double) * (size_t)(nnz * bb));
  h->pos = malloc(sizeof(int64_t) * nz1(n));
  h->order = malloc(sizeof(int64_t) * nz1(n));
  /* colour-major order, ascending index within a colour (stable counting sort) */
  int maxc = 0;
  for (int64_t i = 0; i < n; i++) if (colour[i] + 1 > maxc) maxc = colour[i] + 1;
  int64_t *cnt = calloc((size_t)maxc + 1, sizeof(int64_t));
  for (int64_t i = 0; i < n; i++) cnt[colour[i] + 1]++;
  for (int c = 0; c < maxc; c++) cnt[c + 1] += cnt[c];
  for (int64_t i = 0; i < n; i++) { h->pos[i] = cnt[colour[i]]++; h->order[h->pos[i]] = i; }
  free(cnt);
  double *Lblk = malloc(sizeof(double) * (size_t)bb), *prod = malloc(sizeof(double) * (size_t)bb);
  int64_t maxrow = 0;
  for (int64_t i = 0; i < n; i++) if (rp[i + 1] - rp[i] > maxrow) maxrow = rp[i + 1] - rp[i];
  kp_t *lower = malloc(sizeof(kp_t) * nz1(maxrow));
  for (int64_t t = 0; t < n; t++) {
    int64_t i = h->order[t];
    int64_t nl = 0;
    for (int64_t p = rp[i]; p < rp[i + 1]; p++)
      if (h->pos[col[p]] < h->pos[i]) { lower[nl].key = h->pos[col[p]]; lower[nl].p = p; nl++; }
    qsort(lower, (size_t)nl, sizeof(kp_t), cmp_kp);
    for (int64_t u = 0; u < nl; u++) {
      int64_t p = lower[u].p, kk = col[p];
      int64_t kd = find_entry(rp, col, kk, kk);
      block_mul(b, h->F + p * bb, h->F + kd * bb, Lblk);       /* W_ik U_kk^-1 */
      memcpy(h->F + p * bb, Lblk, sizeof(double) * (size_t)bb);
      for (int64_t q = rp[i]; q < rp[i + 1]; q++) {
        int64_t j = col[q];
        if (h->pos[j] <= h->pos[kk]) continue;
        int64_t r = find_entry(rp, col, kk, j);
        if (r < 0) continue;
        block_mul(b, Lblk, h->F + r * bb, prod);
        for (int e = 0; e < bb; e++) h->F[q * bb + e] = h->F[q * bb + e] - prod[e];
      }
    }
    int64_t dp = find_entry(rp, col, i, i);
    double inv[64];
    int st = orc_gj_inverse(b, h->F + dp * bb, inv);
    if (st) { *status = st; free(Lblk); free(prod); free(lower); orc_bilu0_free(h); return NULL; }
    memcpy(h->F + dp * bb, inv, sizeof(double) * (size_t)bb);
  }
  free(Lblk); free(prod); free(lower);
  return h;
}

void orc_bilu0_solve(const void *hv, const double *r, double *y) {
  const orc_ilu *h = hv;
  const int b = h->b;
  const int64_t bb = (int64_t)b * b, n = h->n;
  double t[8], u[8];
  for (int64_t s = 0; s < n; s++) {             /* forward: y_i = r_i - sum L_ik y_k */
    int64_t i = h->order[s];
    for (int c = 0; c < b; c++) t[c] = r[i * b + c];
    for (int64_t p = h->rp[i]; p < h->rp[i + 1]; p++) {
      int64_t k = h->col[p];
      if (h->pos[k] >= h->pos[i]) continue;
      block_vec(b, h->F + p * bb, y + k * b, u);
      for (int c = 0; c < b; c++) t[c] = t[c] - u[c];
    }
    for (int c = 0; c < b; c++) y[i * b + c] = t[c];
  }
  for (int64_t s = n - 1; s >= 0; s--) {        /* backward: y_i = U_ii^-1 (y_i - sum U_ij y_j) */
    int64_t i = h->order[s];
    int64_t dp = -1;
    for (int c = 0; c < b; c++) t[c] = y[i * b + c];
    for (int64_t p = h->rp[i]; p < h->rp[i + 1]; p++) {
      int64_t j = h->col[p];
      if (j == i) { dp = p; continue; }
      if (h->pos[j] < h->pos[i]) continue;
      block_vec(b, h->F + p * bb, y + j * b, u);
      for (int c = 0; c < b; c++) t[c] = t[c] - u[c];
    }
    block_vec(b, h->F + dp * bb, t, u);
    for (int c = 0; c < b; c++) y[i * b + c] = u[c];
  }
}

void orc_bilu0_factors(const void *hv, double *F) {
  const orc_ilu *h = hv;
  memcpy(F, h->F, sizeof(double) * (size_t)(h->rp[h->n] * h->b * h->b));
}

/* ======================================================================
 * Block ILU(1).  The paper's subdomain solves may be block ILU(k), and the
 * level it recommends is k = 1 (Sec. "Preconditioners", the RAS paragraph).
 * Reading for a single-domain, multicolour form:
 *   order: a distance-2 colouring, so that the rows of one colour are still
 *     uncoupled once the level-1 fill is added: grid cell (x, y, z) takes
 *     colour (x + 2y + 3z) mod 7 (the 7-point neighbours of a cell differ
 *     from it by +-1, +-2, +-3 mod 7 and cells two steps apart by a nonzero
 *     sum of two of those, |sum| <= 6); every other row (the wells), in
 *     index order, takes the first colour 7, 8, ... not taken by an earlier
 *     such row that is adjacent to it or shares a neighbour with it; rows
 *     are sorted by (colour, index) as for ILU(0);
 *   pattern: level of fill at most 1 (Saad, Iterative Methods for Sparse
 *     Linear Systems, Sec. 10.3.3, lev_ij = min over k of lev_ik + lev_kj
 *     + 1): the stored pattern plus every (i, j) with a neighbour k ordered
 *     before both i and j and (i, k), (k, j) stored; an entry made from a
 *     fill entry has level >= 2 and is dropped;
 *   numeric: the IKJ factorisation of orc_bilu0_setup on that pattern, the
 *     fill entries starting from zero.
 * The parallel sweeps need the rows of one colour uncoupled in the factor
 * pattern; orc_bilu_colours_independent checks it.
 * ====================================================================== */
int orc_colour_geo(int nx, int ny, int nz, int64_t n, const int64_t *rp, const int32_t *col,
                   int32_t *colour) {
  const int64_t nc = (int64_t)nx * ny * nz;
  if (nx < 1 || ny < 1 || nz < 1 || nc > n) return ORC_INVALID;
  for (int64_t i = 0; i < nc; i++) {
    const int64_t x = i % nx, y = (i / nx) % ny, z = i / ((int64_t)nx * ny);
    colour[i] = (int32_t)((x + 2 * y + 3 * z) % 7);
  }
  int ncol = 0;
  for (int64_t i = 0; i < nc; i++) if (colour[i] + 1 > ncol) ncol = colour[i] + 1;
  for (int64_t w = nc; w < n; w++) {
    uint64_t used = 0;
    for (int64_t p = rp[w]; p < rp[w + 1]; p++) {
      const int64_t k = col[p];
      if (k == w) continue;
      if (k >= nc && k < w) used |= (uint64_t)1 << (colour[k] - 7);
      for (int64_t q = rp[k]; q < rp[k + 1]; q++) {
        const int64_t j = col[q];
        if (j >= nc && j < w) used |= (uint64_t)1 << (colour[j] - 7);
      }
    }
    int c = 0;
    while (c < ORC_MAX_COLOURS - 7 && (used >> c) & 1) c++;
    if (c >= ORC_MAX_COLOURS - 7) return ORC_COLOURS;
    colour[w] = 7 + c;
    if (colour[w] + 1 > ncol) ncol = colour[w] + 1;
  }
  return ncol;
}

/* The level-1 pattern of (rp, col) in the order pos: rows sorted by column. */
static void ilu1_pattern(int64_t n, const int64_t *rp, const int32_t *col, const int64_t *pos,
                         int64_t **rp1_out, int32_t **col1_out) {
  int64_t *stamp = malloc(sizeof(int64_t) * nz1(n));
  for (int64_t i = 0; i < n; i++) stamp[i] = -1;
  int64_t *rp1 = malloc(sizeof(int64_t) * (size_t)(n + 1));
  rp1[0] = 0;
  for (int pass = 0; pass < 2; pass++) {
    int32_t *col1 = pass ? *col1_out : NULL;
    for (int64_t i = 0; i < n; i++) stamp[i] = -1;
    for (int64_t i = 0; i < n; i++) {
      int64_t cnt = 0, base = pass ? rp1[i] : 0;
      for (int64_t p = rp[i]; p < rp[i + 1]; p++) {
        stamp[col[p]] = i;
        if (pass) col1[base + cnt] = col[p];
        cnt++;
      }
      for (int64_t p = rp[i]; p < rp[i + 1]; p++) {
        const int64_t k = col[p];
        if (pos[k] >= pos[i]) continue;
        for (int64_t q = rp[k]; q < rp[k + 1]; q++) {
          const int64_t j = col[q];
          if (pos[j] <= pos[k] || stamp[j] == i) continue;
          stamp[j] = i;
          if (pass) col1[base + cnt] = (int32_t)j;
          cnt++;
        }
      }
      if (!pass) rp1[i + 1] = rp1[i] + cnt;
      else
        for (int64_t a = base + 1; a < base + cnt; a++) {   /* insertion sort of the row */
          int32_t v = col1[a];
          int64_t b2 = a - 1;
          while (b2 >= base && col1[b2] > v) { col1[b2 + 1] = col1[b2]; b2--; }
          col1[b2 + 1] = v;
        }
    }
    if (!pass) *col1_out = malloc(sizeof(int32_t) * nz1(rp1[n]));
  }
  free(stamp);
  *rp1_out = rp1;
}

void *orc_biluk_setup(int64_t n, int b, const int64_t *rp, const int32_t *col, const double *vt,
                      const int32_t *colour, int level, int *status) {
  if (level == 0) return orc_bilu0_setup(n, b, rp, col, vt, colour, status);
  if (level != 1) { *status = ORC_INVALID; return NULL; }
  const int64_t bb = (int64_t)b * b;
  /* positions of the colour-major order (the same stable sort as ILU(0)) */
  int maxc = 0;
  for (int64_t i = 0; i < n; i++) if (colour[i] + 1 > maxc) maxc = colour[i] + 1;
  int64_t *cnt = calloc((size_t)maxc + 1, sizeof(int64_t));
  int64_t *pos = malloc(sizeof(int64_t) * nz1(n));
  for (int64_t i = 0; i < n; i++) cnt[colour[i] + 1]++;
  for (int c = 0; c < maxc; c++) cnt[c + 1] += cnt[c];
  for (int64_t i = 0; i < n; i++) pos[i] = cnt[colour[i]]++;
  free(cnt);
  int64_t *rp1;
  int32_t *col1;
  ilu1_pattern(n, rp, col, pos, &rp1, &col1);
  free(pos);
  double *vt1 = calloc(nz1(rp1[n] * bb), sizeof(double));
  for (int64_t i = 0; i < n; i++)
    for (int64_t p = rp1[i]; p < rp1[i + 1]; p++) {
      const int64_t src = find_entry(rp, col, i, col1[p]);
      if (src >= 0) memcpy(vt1 + p * bb, vt + src * bb, sizeof(double) * (size_t)bb);
    }
  void *h = orc_bilu0_setup(n, b, rp1, col1, vt1, colour, status);
  free(rp1); free(col1); free(vt1);
  return h;
}

int64_t orc_bilu_nnz(const void *hv) {
  const orc_ilu *h = hv;
  return h->rp[h->n];
}

void orc_bilu_pattern(const void *hv, int64_t *rp, int32_t *col) {
  const orc_ilu *h = hv;
  memcpy(rp, h->rp, sizeof(int64_t) * (size_t)(h->n + 1));
  memcpy(col, h->col, sizeof(int32_t) * (size_t)h->rp[h->n]);
}

int orc_bilu_colours_independent(const void *hv, const int32_t *colour) {
  const orc_ilu *h = hv;
  for (int64_t i = 0; i < h->n; i++)
    for (int64_t p = h->rp[i]; p < h->rp[i + 1]; p++)
      if (h->col[p] != i && colour[h->col[p]] == colour[i]) return 0;
  return 1;
}

/* ======================================================================
 * CPR-FPF (Algorithm pc-fpf; its listing is garbled -- the third line
 * repeats the first and r is undefined -- so the five steps of the prose are
 * followed):  with f = D^-1 v (decoupling as a right-preconditioner factor,
 * M^-1 = CPR(Ã)^-1 D^-1, which gives the same x as solving Eq.
 * decoupled-eq and keeps the Krylov residual equal to b - A x):
 *   y1 = F^-1 f;            r1 = f - Ã y1;
 *   y2 = y1 + Pi_p AMG(A_p)^-1 Pi_r r1;
 *   r2 = f - Ã y2;          z  = y2 + F^-1 r2;
 * Pi_r takes entry 0 (pressure) of every block, Pi_p adds into entry 0.
 * ====================================================================== */
typedef struct {
  int64_t n;
  int b;
  int64_t *rp;
  int32_t *col;
  double *vt;
  double *dinv;
  void *amg;
  void *ilu;
  int32_t *colour;
  int n_colours;
  int stages;
} orc_cpr;

void orc_cpr_free(void *hv) {
  orc_cpr *h = hv;
  if (!h) return;
  orc_amg_free(h->amg);
  orc_bilu0_free(h->ilu);
  free(h->rp); free(h->col); free(h->vt); free(h->dinv); free(h->colour); free(h);
}

void *orc_cpr_setup(int64_t n, int b, const int64_t *rp, const int32_t *col, const double *val,
                    const orc_cpr_opts *opts, int *status) {
  const int64_t bb = (int64_t)b * b, nnz = rp[n];
  *status = ORC_OK;
  if (!orc_pattern_symmetric(n, rp, col)) { *status = ORC_INVALID; return NULL; }
  orc_cpr *h = calloc(1, sizeof(orc_cpr));
  h->n = n; h->b = b;
  h->rp = malloc(sizeof(int64_t) * (size_t)(n + 1));
  h->col = malloc(sizeof(int32_t) * nz1(nnz));
  memcpy(h->rp, rp, sizeof(int64_t) * (size_t)(n + 1));
  memcpy(h->col, col, sizeof(int32_t) * (size_t)nnz);
  h->vt = malloc(sizeof(double) * nz1(nnz * bb));
  h->dinv = malloc(sizeof(double) * nz1(n * bb));
  if (opts->stages < ORC_CPR_FPF || opts->stages > ORC_CPR_PF) { *status = ORC_INVALID; orc_cpr_free(h); return NULL; }
  h->stages = opts->stages;
  int st = orc_decouple_mode(n, b, rp, col, val, opts->decoupling, h->vt, h->dinv);
  if (st) { *status = st; orc_cpr_free(h); return NULL; }
  double *ap = malloc(sizeof(double) * nz1(nnz));
  orc_pressure_matrix(n, b, rp, col, h->vt, ap);
  h->amg = orc_amg_setup(n, rp, col, ap, opts->theta, opts->coarse_max, opts->max_levels,
                         opts->cheb_degree, opts->seed, &st);
  free(ap);
  if (!h->amg) { *status = st; orc_cpr_free(h); return NULL; }
  h->colour = malloc(sizeof(int32_t) * nz1(n));
  if (opts->ilu_fill != 0 && opts->ilu_fill != 1) { *status = ORC_INVALID; orc_cpr_free(h); return NULL; }
  int nc = opts->ilu_fill == 0
               ? orc_colour_jp(n, rp, col, opts->seed ^ 0x85EBCA77u, h->colour)
               : orc_colour_geo(opts->grid[0], opts->grid[1], opts->grid[2], n, rp, col, h->colour);
  if (nc < 0) { *status = nc; orc_cpr_free(h); return NULL; }
  h->n_colours = nc;
  h->ilu = orc_biluk_setup(n, b, h->rp, h->col, h->vt, h->colour, opts->ilu_fill, &st);
  if (!h->ilu) { *status = st; orc_cpr_free(h); return NULL; }
  if (!orc_bilu_colours_independent(h->ilu, h->colour)) { *status = ORC_INVALID; orc_cpr_free(h); return NULL; }
  return h;
}

/* z = CPR(Ã)^-1 D^-1 v.  With f = D^-1 v, F = the block ILU(0) of Ã,
 * P = AMG(A_PP)^-1 one V-cycle, Pi_r = restriction to the pressure entries
 * and Pi_p = prolongation into them (entry 0 of every block):
 *   FPF (Algorithm pc-fpf): y1 = F^-1 f; r1 = f - Ã y1;
 *        y2 = y1 + Pi_p P Pi_r r1; r2 = f - Ã y2; z = y2 + F^-1 r2;
 *   FP:  the first three steps, z = y2;
 *   PF:  y1 = Pi_p P Pi_r f; r1 = f - Ã y1; z = y1 + F^-1 r1.
 * (CPR-FP and CPR-PF are the two-stage orderings the paper compares with
 * CPR-FPF, Sec. "Preconditioners" and the tables of Sec. "Numerical
 * Performance".) */
void orc_cpr_apply(const void *hv, const double *v, double *z) {
  const orc_cpr *h = hv;
  const int64_t n = h->n, N = n * h->b;
  const int b = h->b;
  const int64_t bb = (int64_t)b * b;
  double *f = calloc((size_t)N, sizeof(double)), *y = calloc((size_t)N, sizeof(double));
  double *r = malloc(sizeof(double) * (size_t)N);
  double *rp_ = calloc((size_t)n, sizeof(double)), *ep = calloc((size_t)n, sizeof(double));
  for (int64_t i = 0; i < n; i++) block_vec(b, h->dinv + i * bb, v + i * b, f + i * b);
  if (h->stages == ORC_CPR_PF) {
    for (int64_t i = 0; i < n; i++) rp_[i] = f[i * b];
    orc_amg_vcycle(h->amg, rp_, ep);
    for (int64_t i = 0; i < n; i++) y[i * b] = ep[i];                       /* y1, y = 0 elsewhere */
    memcpy(r, f, sizeof(double) * (size_t)N);
    orc_bsr_spmv(n, b, h->rp, h->col, h->vt, y, r, -1.0, 1.0);              /* r1 */
    orc_bilu0_solve(h->ilu, r, z);
    for (int64_t e = 0; e < N; e++) z[e] = y[e] + z[e];
  } else {
    orc_bilu0_solve(h->ilu, f, y);                                           /* y1 */
    memcpy(r, f, sizeof(double) * (size_t)N);
    orc_bsr_spmv(n, b, h->rp, h->col, h->vt, y, r, -1.0, 1.0);              /* r1 */
    for (int64_t i = 0; i < n; i++) rp_[i] = r[i * b];
    orc_amg_vcycle(h->amg, rp_, ep);
    for (int64_t i = 0; i < n; i++) y[i * b] = y[i * b] + ep[i];            /* y2 */
    if (h->stages == ORC_CPR_FP) {
      memcpy(z, y, sizeof(double) * (size_t)N);
    } else {
      memcpy(r, f, sizeof(double) * (size_t)N);
      orc_bsr_spmv(n, b, h->rp, h->col, h->vt, y, r, -1.0, 1.0);            /* r2 */
      orc_bilu0_solve(h->ilu, r, z);
      for (int64_t e = 0; e < N; e++) z[e] = y[e] + z[e];
    }
  }
  free(f); free(y); free(r); free(rp_); free(ep);
}

int orc_cpr_info(const void *hv, int *n_levels, int *n_colours) {
  const orc_cpr *h = hv;
  *n_levels = orc_amg_levels(h->amg);
  *n_colours = h->n_colours;
  return 0;
}
const void *orc_cpr_amg(const void *hv) { return ((const orc_cpr *)hv)->amg; }
void orc_cpr_colours(const void *hv, int32_t *colour) {
  const orc_cpr *h = hv;
  memcpy(colour, h->colour, sizeof(int32_t) * (size_t)h->n);
}
void orc_cpr_decoupled(const void *hv, double *vt, double *dinv) {
  const orc_cpr *h = hv;
  const int64_t bb = (int64_t)h->b * h->b;
  memcpy(vt, h->vt, sizeof(double) * (size_t)(h->rp[h->n] * bb));
  memcpy(dinv, h->dinv, sizeof(double) * (size_t)(h->n * bb));
}
void orc_cpr_ilu_factors(const void *hv, double *F) { orc_bilu0_factors(((const orc_cpr *)hv)->ilu, F); }

const void *orc_cpr_ilu(const void *hv) { return ((const orc_cpr *)hv)->ilu; }

/* ======================================================================
 * Restarted flexible GMRES (Saad 1993) with right preconditioning and
 * classical Gram-Schmidt applied twice (CGS2); the paper's Krylov layer
 * offers GMRES-type solvers (Sec. "Linear Solver").  Readings:
 *   h_{j+1,j} = ||w|| after the second pass; happy breakdown when
 *   h_{j+1,j} <= 1e-14 ||A z_j||; Givens rotations c = a/d, s = h/d,
 *   d = sqrt(a^2 + h^2); stop a cycle when |g_{j+1}| <= rtol ||b||, form
 *   x += Z y, compute the true residual and restart while it is above
 *   rtol ||b|| and fewer than maxit iterations were spent.
 * ====================================================================== */
static double dot(int64_t N, const double *a, const double *b) {
  double s = 0.0;
  for (int64_t i = 0; i < N; i++) s = s + a[i] * b[i];
  return s;
}

int orc_fgmres(int64_t n, int b, const int64_t *rp, const int32_t *col, const double *val,
               const void *cpr, const double *rhs, double *x, double rtol, int restart, int maxit,
               orc_stats *st, double *hist, int hist_cap) {
  const int64_t N = n * b;
  const int m = restart;
  memset(st, 0, sizeof(*st));
  double bnorm = sqrt(dot(N, rhs, rhs));
  if (bnorm == 0.0) {
    for (int64_t e = 0; e < N; e++) x[e] = 0.0;
    st->converged = 1;
    return ORC_OK;
  }
  double *V = malloc(sizeof(double) * (size_t)(N * (m + 1)));
  double *Z = malloc(sizeof(double) * (size_t)(N * m));
  double *w = malloc(sizeof(double) * (size_t)N), *r = malloc(sizeof(double) * (size_t)N);
  double *H = calloc((size_t)((m + 1) * m), sizeof(double));
  double *cs = malloc(sizeof(double) * (size_t)m), *sn = malloc(sizeof(double) * (size_t)m);
  double *g = malloc(sizeof(double) * (size_t)(m + 1)), *yv = malloc(sizeof(double) * (size_t)m);
  double *h1 = malloc(sizeof(double) * (size_t)(m + 1)), *h2 = malloc(sizeof(double) * (size_t)(m + 1));
  if (!V || !Z || !w || !r || !H) { free(V); free(Z); free(w); free(r); free(H); return ORC_NOMEM; }
  int iters = 0, converged = 0, status = ORC_OK;
  double relres = 0.0;
  int nh = 0;
  for (;;) {
    memcpy(r, rhs, sizeof(double) * (size_t)N);
    orc_bsr_spmv(n, b, rp, col, val, x, r, -1.0, 1.0);
    double beta = sqrt(dot(N, r, r));
    relres = beta / bnorm;
    st->true_relres = relres;
    if (nh < hist_cap && iters == 0 && hist) hist[nh++] = relres;
    if (relres <= rtol) { converged = 1; break; }
    if (iters >= maxit) break;
    if (!isfinite(beta)) { status = ORC_SINGULAR; break; }
    for (int64_t e = 0; e < N; e++) V[e] = r[e] / beta;
    for (int i = 0; i <= m; i++) g[i] = 0.0;
    g[0] = beta;
    int j, jdone = 0;
    for (j = 0; j < m; j++) {
      double *vj = V + (int64_t)j * N, *zj = Z + (int64_t)j * N;
      orc_cpr_apply(cpr, vj, zj);
      for (int64_t e = 0; e < N; e++) w[e] = 0.0;
      orc_bsr_spmv(n, b, rp, col, val, zj, w, 1.0, 0.0);
      double wnorm0 = sqrt(dot(N, w, w));
      for (int k = 0; k <= j; k++) h1[k] = dot(N, V + (int64_t)k * N, w);
      for (int k = 0; k <= j; k++) {
        const double *vk = V + (int64_t)k * N;
        for (int64_t e = 0; e < N; e++) w[e] = w[e] - h1[k] * vk[e];
      }
      for (int k = 0; k <= j; k++) h2[k] = dot(N, V + (int64_t)k * N, w);
      for (int k = 0; k <= j; k++) {
        const double *vk = V + (int64_t)k * N;
        for (int64_t e = 0; e < N; e++) w[e] = w[e] - h2[k] * vk[e];
      }
      for (int k = 0; k <= j; k++) H[k * m + j] = h1[k] + h2[k];
      double hn = sqrt(dot(N, w, w));
      H[(j + 1) * m + j] = hn;
      for (int k = 0; k < j; k++) {
        double a = H[k * m + j], c = H[(k + 1) * m + j];
        H[k * m + j] = cs[k] * a + sn[k] * c;
        H[(k + 1) * m + j] = -sn[k] * a + cs[k] * c;
      }
      double a = H[j * m + j], c = H[(j + 1) * m + j];
      double d = sqrt(a * a + c * c);
      cs[j] = a / d;
      sn[j] = c / d;
      H[j * m + j] = d;
      H[(j + 1) * m + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      iters++;
      relres = fabs(g[j + 1]) / bnorm;
      if (hist && nh < hist_cap) hist[nh++] = relres;
      int breakdown = hn <= 1e-14 * wnorm0;
      if (!breakdown) {
        double *v1 = V + (int64_t)(j + 1) * N;
        for (int64_t e = 0; e < N; e++) v1[e] = w[e] / hn;
      }
      if (relres <= rtol || iters >= maxit || breakdown) { jdone = j + 1; break; }
    }
    if (!jdone) jdone = m;
    /* back substitution H y = g, then x += Z y */
    for (int i = jdone - 1; i >= 0; i--) {
      double s = g[i];
      for (int k = i + 1; k < jdone; k++) s = s - H[i * m + k] * yv[k];
      yv[i] = s / H[i * m + i];
    }
    for (int k = 0; k < jdone; k++) {
      const double *zk = Z + (int64_t)k * N;
      for (int64_t e = 0; e < N; e++) x[e] = x[e] + yv[k] * zk[e];
    }
    st->restarts++;
    st->est_relres = relres;
  }
  if (st->restarts > 0) st->restarts--;
  st->iters = iters;
  st->converged = converged;
  free(V); free(Z); free(w); free(r); free(H); free(cs); free(sn); free(g); free(yv); free(h1); free(h2);
  if (status) return status;
  return converged ? ORC_OK : ORC_NOT_CONVERGED;
}

/* ======================================================================
 * BiCGSTAB (van der Vorst 1992), right-preconditioned with the same
 * CPR-FPF: the Krylov solver of every run in the paper (Examples num-sagd,
 * sca-230m, ...; Sec. "Linear Solver" lists it among the solvers).  With
 * shadow residual r^ = r0 and rho = <r^, r>:
 *   p = r + beta (p - omega v), beta = (rho / rho_old)(alpha / omega);
 *   p^ = M^-1 p;  v = A p^;  alpha = rho / <r^, v>;  s = r - alpha v;
 *   (if ||s|| <= rtol ||b||: x += alpha p^ and stop)
 *   s^ = M^-1 s;  t = A s^;  omega = <t, s> / <t, t>;
 *   x += alpha p^ + omega s^;  r = s - omega t.
 * A recurrence residual below rtol is confirmed on the true residual; if
 * the true residual is still above, the iteration restarts from it.
 * ====================================================================== */
int orc_bicgstab(int64_t n, int b, const int64_t *rp, const int32_t *col, const double *val,
                 const void *cpr, const double *rhs, double *x, double rtol, int maxit, orc_stats *st,
                 double *hist, int hist_cap) {
  const int64_t N = n * b;
  memset(st, 0, sizeof(*st));
  double bnorm = sqrt(dot(N, rhs, rhs));
  if (bnorm == 0.0) {
    for (int64_t e = 0; e < N; e++) x[e] = 0.0;
    st->converged = 1;
    return ORC_OK;
  }
  double *r = malloc(sizeof(double) * (size_t)N), *rh = malloc(sizeof(double) * (size_t)N);
  double *p = calloc((size_t)N, sizeof(double)), *v = calloc((size_t)N, sizeof(double));
  double *ph = malloc(sizeof(double) * (size_t)N), *s = malloc(sizeof(double) * (size_t)N);
  double *sh = malloc(sizeof(double) * (size_t)N), *t = malloc(sizeof(double) * (size_t)N);
  int iters = 0, nh = 0, cycles = 0, converged = 0, status = ORC_OK;
  double relres = 1.0;
  /* Every cycle starts from the true residual of the current x, and the
   * solve ends there too, so true_relres always belongs to the returned x. */
  for (;;) {
    memcpy(r, rhs, sizeof(double) * (size_t)N);
    orc_bsr_spmv(n, b, rp, col, val, x, r, -1.0, 1.0);
    relres = sqrt(dot(N, r, r)) / bnorm;
    st->true_relres = relres;
    if (hist && nh < hist_cap && iters == 0) hist[nh++] = relres;
    if (!isfinite(relres)) { status = ORC_SINGULAR; break; }
    if (relres <= rtol) { converged = 1; break; }
    if (iters >= maxit) break;
    cycles++;
    memcpy(rh, r, sizeof(double) * (size_t)N);
    for (int64_t e = 0; e < N; e++) { p[e] = 0.0; v[e] = 0.0; }
    double rho_old = 1.0, alpha = 1.0, omega = 1.0;
    while (iters < maxit) {
      const double rho = dot(N, rh, r);
      if (rho == 0.0 || !isfinite(rho)) break;          /* breakdown: restart */
      const double beta = (rho / rho_old) * (alpha / omega);
      for (int64_t e = 0; e < N; e++) p[e] = r[e] + beta * (p[e] - omega * v[e]);
      orc_cpr_apply(cpr, p, ph);
      for (int64_t e = 0; e < N; e++) v[e] = 0.0;
      orc_bsr_spmv(n, b, rp, col, val, ph, v, 1.0, 0.0);
      alpha = rho / dot(N, rh, v);
      for (int64_t e = 0; e < N; e++) s[e] = r[e] - alpha * v[e];
      iters++;
      const double snorm = sqrt(dot(N, s, s)) / bnorm;
      if (snorm <= rtol) {                               /* half step suffices */
        for (int64_t e = 0; e < N; e++) x[e] = x[e] + alpha * ph[e];
        relres = snorm;
        if (hist && nh < hist_cap) hist[nh++] = relres;
        break;
      }
      orc_cpr_apply(cpr, s, sh);
      for (int64_t e = 0; e < N; e++) t[e] = 0.0;
      orc_bsr_spmv(n, b, rp, col, val, sh, t, 1.0, 0.0);
      omega = dot(N, t, s) / dot(N, t, t);
      for (int64_t e = 0; e < N; e++) x[e] = x[e] + alpha * ph[e] + omega * sh[e];
      for (int64_t e = 0; e < N; e++) r[e] = s[e] - omega * t[e];
      relres = sqrt(dot(N, r, r)) / bnorm;
      if (hist && nh < hist_cap) hist[nh++] = relres;
      rho_old = rho;
      if (relres <= rtol || omega == 0.0 || !isfinite(relres)) break;
    }
    st->est_relres = relres;
  }
  st->restarts = cycles > 0 ? cycles - 1 : 0;
  st->iters = iters;
  st->converged = converged;
  free(r); free(rh); free(p); free(v); free(ph); free(s); free(sh); free(t);
  if (status) return status;
  return converged ? ORC_OK : ORC_NOT_CONVERGED;
}

/* ======================================================================
 * Adjoint.  For L(x) with x = A^-1 b and g = dL/dx: A^T lambda = g gives
 * dL/db = lambda and dL/dA_ij = -lambda_i x_j^T on every stored block.
 * Chain to theta = log k through the assembly above: for the face between
 * i and j (direction d from i, opposite d' from j)
 *   dL/dT = <G_ii - G_ij, M_i,d> + <G_jj - G_ji, M_j,d'>,
 *   dT/dtheta_i = T k_j / (k_i + k_j)   (harmonic mean, both faces scaled
 *   alike by kv/kh, which cancels in the ratio).
 * ====================================================================== */
void orc_outer_product(int64_t n, int b, const int64_t *rp, const int32_t *col,
                       const double *lambda, const double *x, double *dA) {
  const int64_t bb = (int64_t)b * b;
  for (int64_t i = 0; i < n; i++)
    for (int64_t p = rp[i]; p < rp[i + 1]; p++) {
      int64_t j = col[p];
      for (int r = 0; r < b; r++)
        for (int s = 0; s < b; s++) dA[p * bb + r * b + s] = -(lambda[i * b + r] * x[j * b + s]);
    }
}

int orc_chain_theta(int nx, int ny, int nz, int b, const double *k, double kvkh, double c_t,
                    const double *M, const int64_t *rp, const int32_t *col, const double *dA,
                    double *dtheta) {
  const int64_t n_c = (int64_t)nx * ny * nz, bb = (int64_t)b * b;
  for (int64_t i = 0; i < n_c; i++) dtheta[i] = 0.0;
  for (int64_t i = 0; i < n_c; i++)
    for (int d = 3; d < 6; d++) {       /* each face once, from its lower cell */
      int64_t j = neighbour(nx, ny, nz, i, d);
      if (j < 0) continue;
      int vertical = (d == 5);
      double T = face_transmissibility(k, kvkh, c_t, i, j, vertical);
      int64_t pii = find_entry(rp, col, i, i), pij = find_entry(rp, col, i, j);
      int64_t pjj = find_entry(rp, col, j, j), pji = find_entry(rp, col, j, i);
      if (pii < 0 || pij < 0 || pjj < 0 || pji < 0) return ORC_INVALID;
      const double *Mi = M + (i * 6 + d) * bb, *Mj = M + (j * 6 + opposite_dir(d)) * bb;
      double s = 0.0;
      for (int e = 0; e < bb; e++) s = s + (dA[pii * bb + e] - dA[pij * bb + e]) * Mi[e];
      for (int e = 0; e < bb; e++) s = s + (dA[pjj * bb + e] - dA[pji * bb + e]) * Mj[e];
      double ki = k[i], kj = k[j];
      if (ki + kj == 0.0) continue;
      dtheta[i] = dtheta[i] + s * (T * (kj / (ki + kj)));
      dtheta[j] = dtheta[j] + s * (T * (ki / (ki + kj)));
    }
  return ORC_OK;
}
