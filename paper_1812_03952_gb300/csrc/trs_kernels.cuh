// Kernel launchers of libtrs (internal).
#pragma once

#include "trs_internal.cuh"

namespace trs {

#define TRS_DISPATCH_B(bval, ...)                                                           \
  switch (bval) {                                                                           \
    case 1: { constexpr int B = 1; __VA_ARGS__; } break;                                     \
    case 2: { constexpr int B = 2; __VA_ARGS__; } break;                                     \
    case 3: { constexpr int B = 3; __VA_ARGS__; } break;                                     \
    case 4: { constexpr int B = 4; __VA_ARGS__; } break;                                     \
    case 5: { constexpr int B = 5; __VA_ARGS__; } break;                                     \
    default: throw Error(TRS_ERR_UNSUPPORTED, "block size must be 1..5");                   \
  }

// Multicolour block ILU(0) factors, rows stored in colour-major positions.
template <class T>
struct IluView {
  Geom g;
  const int32_t *crow;    // [n_rows] row at position q
  const uint8_t *emask;   // [nc] natural-order slot presence
  const uint8_t *lmask;   // [n_rows] bit s: slot s holds an L block (neighbour earlier)
  const int64_t *ftptr;   // [n_rows+1] tail by position
  const int32_t *ftcol;   // natural column
  const uint8_t *ftlow;   // 1: L block, 0: U block
  const T *fell;          // [7 (+18)][n_rows][bb] by position (blocks contiguous); slot 3 = U_ii^-1
  const T *ftval;         // [nft][bb]
  const uint32_t *fmask;  // [n_rows] ILU(1): bit s, fill slot s (fell slot 7 + s) present; NULL for ILU(0)
  const uint32_t *flmask; // [n_rows] ILU(1): bit s, fill slot s holds an L block
};

// Scalar operator of one AMG level: ELL-7 + tail (level 0) or CSR.
template <class T>
struct ScalarOp {
  int is_ell;
  int64_t n;
  // ELL form
  Geom g;
  const uint8_t *emask;
  const int64_t *tptr;
  const int32_t *tcol;
  const T *ell;    // [7][nc]
  const T *tval;   // [ntail]
  // CSR form
  const int64_t *rp;
  const int32_t *col;
  const T *val;
};

// Coarse part of the AMG hierarchy run by one block (levels with few rows).
constexpr int kMaxCheb = 8;
#ifndef TRS_COARSE_FUSE_ROWS
#define TRS_COARSE_FUSE_ROWS 1024
#endif
constexpr int kCoarseFuseRows = TRS_COARSE_FUSE_ROWS;

template <class T>
struct CoarseLevel {
  int64_t n;
  const int64_t *rp;
  const int32_t *col;
  const T *val;
  const T *dinv;
  const int32_t *agg;       // aggregates into the next level (not on the coarsest)
  const int64_t *mptr;      // members of the next level's rows
  const int32_t *midx;
  T inv_theta;
  T c1[kMaxCheb];
  T c2[kMaxCheb];
  T *r, *e, *res, *d, *dn;
};

template <class T>
struct CoarseHierarchy {
  int l0, nlev, deg;        // levels l0 .. nlev-1 run in one block; Chebyshev degree
  const double *cinv;       // inverse of the coarsest operator
  CoarseLevel<T> lv[kMaxLevels];
};

template <class T>
void launch_vcycle_coarse(const CoarseHierarchy<T> &h, cudaStream_t s);


// Reduction scratch: per-block partial sums and a ticket counter.
struct RedScratch {
  double *partial;        // [grid][kMaxRestart + 16]
  unsigned int *counter;  // one word, zero between uses
  int grid;
};

// ---------------------------------------------------------------- k_solve
template <class TA, class TX>
void launch_spmv(int b, const MatView<TA> &A, const TX *x, double *y, double alpha, double beta,
                 cudaStream_t s);
void launch_true_residual(int b, const MatView<double> &A, const double *x, const double *rhs,
                          double *r, const RedScratch &red, double *out_norm2, cudaStream_t s);
void launch_norm2(const double *x, int64_t n, const RedScratch &red, double *out, cudaStream_t s);

template <class T>
// colour, y0: if not NULL, rows of colour 0 also get y0 = f (their forward ILU(0) sweep)
void launch_dscale(int b, int64_t n_rows, const double *w, const double *hnorm2, double *vout,
                   const T *dinv, T *f, const int32_t *colour, T *y0, cudaStream_t s);
template <class T>
void launch_ilu_fwd(int b, const IluView<T> &F, const T *rhs, T *y, int64_t q0, int64_t q1,
                    int64_t q2, cudaStream_t s);
template <class T, class TZ>
void launch_ilu_bwd(int b, const IluView<T> &F, T *y, int64_t q0, int64_t q1, int64_t q2,
                    const T *y1, const T *e0, TZ *zout, const T *rhs, cudaStream_t s);
// CPR residuals on Ã; unit = 1 when every diagonal block of Ã is I (ABF,
// FRS+ABF), so that y_i is added instead of multiplied; y1 may be NULL (zero).
template <class T>
void launch_resid_p(int b, const MatView<T> &At, const T *atp, const T *f, const T *y, T *rp, int unit,
                    cudaStream_t s);
template <class T>
void launch_resid_full(int b, const MatView<T> &At, const T *f, const T *y1, const T *e0, T *r,
                       int unit, const int32_t *colour, T *x0, cudaStream_t s);
// z = y1 + Pi_p e0 (FP64 out) and rp = Pi_r f, for the CPR-FP and CPR-PF orderings
template <class T>
void launch_cpr_combine(int b, int64_t n, const T *y1, const T *e0, double *z, cudaStream_t s);
template <class T>
void launch_pressure_of(int b, int64_t n, const T *f, T *rp, cudaStream_t s);

template <class T>
void launch_cheb_resid_init(const ScalarOp<T> &op, const T *r, const T *e, const T *dinv,
                            double inv_theta, T *res, T *d, cudaStream_t s);
template <class T>
void launch_cheb_step(const ScalarOp<T> &op, const T *res_in, T *res_out, const T *d,
                      const T *dinv, double c1, double c2, T *dn, T *e, int last, cudaStream_t s);
// fused forms: first step from e = 0 with its initialisation; restriction
// of the fine residual r - A e
template <class T>
void launch_cheb_first(const ScalarOp<T> &op, const T *r, const T *dinv, double inv_theta, double c1,
                       double c2, T *res_out, T *d_out, T *dn, T *e, int last, cudaStream_t s);
template <class T>
void launch_restrict_resid(const ScalarOp<T> &op, int64_t nc, const int64_t *mptr, const int32_t *midx,
                           const T *r, const T *e, T *rc, cudaStream_t s);
template <class T>
void launch_prolong(int64_t n, const int32_t *agg, const T *ec, T *e, cudaStream_t s);
template <class T>
void launch_dense_gemv(int64_t n, const double *Minv, const T *r, T *e, cudaStream_t s);

void launch_multidot(const double *V, int64_t N, int K, const double *w, const RedScratch &red,
                     double *out, cudaStream_t s);
void launch_cgs_update(const double *V, int64_t N, int K, const double *h, double *w,
                       int want_dots, const RedScratch &red, double *out, cudaStream_t s);
void launch_cgs_dots(const double *V, int64_t N, int K, const double *w, const RedScratch &red,
                     double *out, cudaStream_t s);
void launch_cgs_update_dots(const double *V, int64_t N, int K, const double *h, double *w,
                            const RedScratch &red, double *out, cudaStream_t s);
void launch_givens(int j, int m, double *H, const double *h1, const double *h2,
                   const double *hn2, const double *wn2, double *cs, double *sn, double *g,
                   double *hnorm_out, double *relres_out, double inv_bnorm, cudaStream_t s);
void launch_lsq(int jdone, int m, const double *H, const double *g, double *y, cudaStream_t s);
template <class TZ>
void launch_xupdate(const TZ *Z, int64_t N, int K, const double *y, double *x, cudaStream_t s);
void launch_scale_copy(const double *r, const double *norm2, double *v, int64_t N, cudaStream_t s);

template <class TS, class TD>
void launch_cast(const TS *src, TD *dst, int64_t n, cudaStream_t s);

// BiCGSTAB scalars, kept on the device between the kernels of one iteration.
struct BicgScalars {
  double rho, rho_old, alpha, omega;   // recurrence coefficients
  double rv, ss, ts, tt, rr;           // <r^,v>, ||s||^2, <t,s>, <t,t>, ||r||^2
  double half;                         // 1: ||s|| met the tolerance (x += alpha p^ only)
  double bnorm, rtol;
};
void launch_bicg_start(BicgScalars *sc, const double *rr, double bnorm, double rtol, cudaStream_t s);
template <class T>
void launch_bicg_dir(int b, int64_t n, const double *r, const double *v, double *p, const BicgScalars *sc,
                     int first, const T *dinv, T *f, const int32_t *colour, T *y0, cudaStream_t s);
// blocks of one k_bicg_spmv launch (its partial sums take 2 doubles each)
int64_t bicg_spmv_blocks(const Geom &g);
void launch_bicg_spmv(int b, const MatView<double> &A, const double *x, double *y, const double *w, int nd,
                      double *part, unsigned int *counter, BicgScalars *sc, cudaStream_t s);
void launch_bicg_s(int64_t N, const double *r, const double *v, double *sv, const RedScratch &red,
                   BicgScalars *sc, cudaStream_t s);
void launch_bicg_xr(int64_t N, const double *ph, const double *sh, const double *sv, const double *t,
                    const double *rh, double *x, double *r, const RedScratch &red, BicgScalars *sc,
                    cudaStream_t s);

// ---------------------------------------------------------------- k_setup
void launch_scatter_values(int64_t nnzb, int bb, const int64_t *map, const double *uval,
                           int64_t nc, double *ell, double *tval, cudaStream_t s);
// values in canonical BSR order from the ELL/tail storage; aos = 1 for the
// per-slot block-contiguous layout [7][nc][bb] of the decoupled matrix
void launch_gather_values(int64_t nnzb, int bb, const int64_t *map, const double *ell,
                          const double *tval, int64_t nc, double *uval, cudaStream_t s, int aos = 0);
void launch_assemble(int b, trs_bsr *A, const double *perm, int perm_is_log, double kvkh,
                     double c_t, const double *M, const double *acc, const double *wi,
                     const double *lam, cudaStream_t s);
void launch_scale_diagonal(int b, trs_bsr *A, const double *sc, cudaStream_t s);
// at_ell: Ã's ELL part [7][nc][bb]; at_p: its pressure rows (row 0 of every block) [7][b][nc]
void launch_decouple(int b, const MatView<double> &A, const int64_t *tdiag, int mode, double *at_ell,
                     double *at_p, double *at_tval, double *dinv, double *ap_ell, double *ap_tval, int *err,
                     cudaStream_t s);

// exclusive scan of n int64 values (in place allowed), total written to *total (device)
void exclusive_scan(const int64_t *in, int64_t *out, int64_t n, int64_t *total, cudaStream_t s);

}  // namespace trs

namespace trs {

// Scalar CSR matrix on the device (AMG levels, FP64 during setup).
struct Csr {
  int64_t n = 0, nnz = 0;
  DBuf<int64_t> rp;
  DBuf<int32_t> col;
  DBuf<double> val;
};

void launch_ap_csr_rowlen(const Geom &g, const uint8_t *emask, const int64_t *tptr, int64_t *len,
                          cudaStream_t s);
void launch_ap_csr_fill(const Geom &g, const uint8_t *emask, const int64_t *tptr, const int32_t *tcol,
                        const double *ap_ell, const double *ap_tval, const int64_t *rp, int32_t *col,
                        double *val, cudaStream_t s);
// position and value of each row's diagonal entry (-1 and 0.0 if absent)
void launch_diag_pos(int64_t n, const int64_t *rp, const int32_t *col, const double *val, int64_t *dpos,
                     double *dval, cudaStream_t s);
void launch_strength(int64_t n, const int64_t *rp, const int32_t *col, const double *val,
                     const double *dval, double theta, uint8_t *sflag, int32_t *sdeg, cudaStream_t s);
void launch_mis2_init(int64_t n, const int32_t *sdeg, int8_t *state, cudaStream_t s);
void launch_mis2_sweep(int64_t n, const int64_t *rp, const int32_t *col, const uint8_t *sflag,
                       const int8_t *state, uint32_t seed, uint64_t *out_w, cudaStream_t s);
// the second sweep and the decision in one launch (the undecided rows are
// added to *undecided)
void launch_mis2_sweep_decide(int64_t n, const int64_t *rp, const int32_t *col, const uint8_t *sflag, int8_t *state,
                              const uint64_t *w1, uint32_t seed, unsigned long long *undecided, cudaStream_t s);
void launch_in_flag(int64_t n, const int8_t *state, int64_t *flag, cudaStream_t s);
void launch_agg_pass1(int64_t n, const int64_t *rp, const int32_t *col, const uint8_t *sflag,
                      const int32_t *sdeg, const int8_t *state, const int64_t *rootid, int32_t *first,
                      cudaStream_t s);
void launch_agg_pass2(int64_t n, const int64_t *rp, const int32_t *col, const double *val,
                      const uint8_t *sflag, const int32_t *sdeg, const int32_t *first, int32_t *agg,
                      cudaStream_t s);
void launch_members(int64_t n, const int32_t *agg, int64_t n_agg, DBuf<int64_t> &mptr,
                    DBuf<int32_t> &midx, cudaStream_t s);
void launch_galerkin(const Csr &F, const int32_t *agg, int64_t n_agg, const int64_t *mptr,
                     const int32_t *midx, Csr &C, cudaStream_t s);
void launch_gershgorin_dinv(const Csr &A, const int64_t *dpos, double *dinv, unsigned long long *lam_bits,
                            cudaStream_t s);
int launch_dense_inverse(const Csr &A, DBuf<double> &inv, cudaStream_t s);
int launch_colour(const Geom &g, const uint8_t *emask, const int64_t *tptr, const int32_t *tcol,
                  uint32_t seed, int32_t *colour, cudaStream_t s);
void launch_colour_order(const Geom &g, const int32_t *colour, int ncol, std::vector<int64_t> &cptr,
                         std::vector<int64_t> &cmid, int32_t *crow, int64_t *pos, cudaStream_t s);
void launch_ilu_structure(const Geom &g, const uint8_t *emask, const int64_t *tptr, const int32_t *tcol,
                          const int32_t *crow, const int64_t *pos, uint8_t *lmask, DBuf<int64_t> &ftptr,
                          DBuf<int32_t> &ftcol, DBuf<uint8_t> &ftlow, DBuf<int64_t> &ftsrc,
                          cudaStream_t s);
template <class T>
void launch_ilu_init(int b, const Geom &g, const uint8_t *emask, const int32_t *crow, const T *at_ell,
                     const T *at_tval, const int64_t *ftsrc, int64_t nft, int nslots, T *fell, T *ftval,
                     cudaStream_t s);
// Symbolic IKJ plan of the long rows (rows held in the tail: wells, general
// rows), built once per pattern: for long row r, its earlier-ordered
// entries k in ascending position (L_u: index in the row, L_pk: position of
// row k) and, for each, the pairs (k, j) of row k with j later than k and
// stored in row r (P_dst: index in row r; P_src: the block of U_kj, as an
// element offset into the tail values if >= 0, or ~offset into the slot
// array, stride n_rows).  diag: index of the diagonal in the row.
struct LongRowPlan {
  const int64_t *Lptr = nullptr;   // [nlong + 1]
  const int32_t *diag = nullptr;   // [nlong]
  const int32_t *Lu = nullptr;
  const int64_t *Lpk = nullptr;
  const int64_t *Pptr = nullptr;   // [nL + 1]
  const int32_t *Pdst = nullptr;
  const int64_t *Psrc = nullptr;
};
// Per colour: the first long row of the colour in the plan and the largest
// entry, L and pair counts of its rows (they size the shared memory).
struct LongRowColour {
  int64_t first = 0, max_ne = 0, max_nl = 0, max_np = 0;
};
template <class T>
void launch_ilu_factor_colour(int b, const Geom &g, const uint8_t *emask, const int32_t *crow,
                              const int64_t *pos, const int64_t *ftptr, const int32_t *ftcol,
                              const uint8_t *ftlow, const uint32_t *fmask, T *fell, T *ftval, int64_t q0,
                              int64_t q1,
                              int64_t q2, const LongRowPlan *plan, const LongRowColour *pc, int *err,
                              cudaStream_t s);
void launch_decouple_mixed(int b, const MatView<double> &A, const int64_t *tdiag, int mode,
                           float *at_ell, float *at_p, float *at_tval, float *dinv, double *ap_ell,
                           double *ap_tval, int *err, cudaStream_t s);

// ------------------------------------------------------------- k_adjoint
void launch_spmv_t(int b, const trs_bsr &A, const double *x, double *y, double alpha, double beta,
                   cudaStream_t s);
// AT's values from A's; AT made by trs_bsr_transpose (tsrc and ttail set)
void launch_transpose_values(const trs_bsr &A, trs_bsr &AT, cudaStream_t s);
void launch_outer_product(int b, const trs_bsr &A, const double *lambda, const double *x, double *dA,
                          cudaStream_t s);
void launch_chain_theta(int b, const trs_bsr &A, const double *perm, int perm_is_log, double kvkh,
                        double c_t, const double *M, const double *lambda, const double *x,
                        double *dtheta, cudaStream_t s);

}  // namespace trs
