/*
 * trs_oracle.h -- plain FP64 CPU oracle for the CPR-FPF preconditioned FGMRES
 * solve of one Newton-step block Jacobian of a thermal reservoir model
 * (Liu & Chen, arXiv 1812.03952).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or helper with the CUDA library; the two are written
 * independently from the paper and from the readings listed with each
 * function in trs_oracle.c.
 *
 * Matrices are general block CSR ("BSR"): n block rows, b x b blocks stored
 * row-major, rp[n+1] (int64) row pointers, col[nnzb] (int32) sorted column
 * indices, val[nnzb*b*b].  Vectors hold n*b doubles, block by block.
 *
 * Return codes: 0 = success, 1 = not converged, -1 = invalid input,
 * -2 = singular block / matrix, -3 = coarsening stalled, -4 = out of memory,
 * -5 = too many colours.
 */
#ifndef TRS_ORACLE_H
#define TRS_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- synthetic Jacobian assembly (TPFA stencil + Peaceman-type wells) ---- */
int64_t orc_assembly_nnzb(int nx, int ny, int nz, int nw, int64_t np,
                          const int32_t *perf_well, const int32_t *perf_cell);
int orc_assemble(int nx, int ny, int nz, int b, const double *k, double kvkh, double c_t,
                 const double *M, const double *acc, int nw, int64_t np,
                 const int32_t *perf_well, const int32_t *perf_cell, const double *wi,
                 const double *lam, int64_t *rp, int32_t *col, double *val);

/* ---- block sparse kernels ---- */
void orc_bsr_spmv(int64_t n, int b, const int64_t *rp, const int32_t *col, const double *val,
                  const double *x, double *y, double alpha, double beta);
void orc_bsr_spmv_t(int64_t n, int b, const int64_t *rp, const int32_t *col, const double *val,
                    const double *x, double *y, double alpha, double beta);
int orc_bsr_transpose(int64_t n, int b, const int64_t *rp, const int32_t *col, const double *val,
                      int64_t *rpT, int32_t *colT, double *valT);
int orc_pattern_symmetric(int64_t n, const int64_t *rp, const int32_t *col);

/* ---- decoupling ---- */
#define ORC_MAX_B 8
#define ORC_DEC_ABF 0      /* D_i = A_ii (ABF; GJE computes the same operator) */
#define ORC_DEC_NONE 1     /* no decoupling */
#define ORC_DEC_FRS 2      /* full row sum */
#define ORC_DEC_FRS_ABF 3  /* FRS, then ABF */
int orc_gj_inverse(int b, const double *D, double *inv);
int orc_decouple_mode(int64_t n, int b, const int64_t *rp, const int32_t *col, const double *val,
                      int mode, double *vt, double *dinv);
int orc_decouple(int64_t n, int b, const int64_t *rp, const int32_t *col, const double *val,
                 double *vt, double *dinv);
void orc_pressure_matrix(int64_t n, int b, const int64_t *rp, const int32_t *col,
                         const double *vt, double *ap);

/* ---- aggregation AMG on a scalar CSR matrix ---- */
int64_t orc_strength(int64_t n, const int64_t *rp, const int32_t *col, const double *val,
                     double theta, int64_t *srp, int32_t *scol);
int orc_mis2(int64_t n, const int64_t *srp, const int32_t *scol, uint32_t seed, int8_t *state);
int64_t orc_aggregate(int64_t n, const int64_t *rp, const int32_t *col, const double *val,
                      const int64_t *srp, const int32_t *scol, const int8_t *state, int32_t *agg);
int64_t orc_galerkin_nnz(int64_t n, const int64_t *rp, const int32_t *col, const int32_t *agg,
                         int64_t n_agg);
void orc_galerkin(int64_t n, const int64_t *rp, const int32_t *col, const double *val,
                  const int32_t *agg, int64_t n_agg, int64_t *crp, int32_t *ccol, double *cval);
double orc_gershgorin(int64_t n, const int64_t *rp, const int32_t *col, const double *val);
void orc_chebyshev(int64_t n, const int64_t *rp, const int32_t *col, const double *val,
                   double lam_max, int degree, const double *r, double *e, int zero_init);

void *orc_amg_setup(int64_t n, const int64_t *rp, const int32_t *col, const double *val,
                    double theta, int coarse_max, int max_levels, int cheb_degree, uint32_t seed,
                    int *status);
int orc_amg_levels(const void *h);
int64_t orc_amg_level_n(const void *h, int l);
int64_t orc_amg_level_nnz(const void *h, int l);
void orc_amg_level_copy(const void *h, int l, int64_t *rp, int32_t *col, double *val);
void orc_amg_level_agg(const void *h, int l, int32_t *agg);
double orc_amg_level_lambda(const void *h, int l);
void orc_amg_vcycle(const void *h, const double *r, double *e);
void orc_amg_free(void *h);

/* ---- dense LU with partial pivoting ---- */
int orc_dense_lu(int64_t n, double *a, int32_t *piv);
void orc_dense_lu_solve(int64_t n, const double *lu, const int32_t *piv, double *x);

/* ---- multicolouring and block ILU(0) ---- */
int orc_colour_jp(int64_t n, const int64_t *rp, const int32_t *col, uint32_t seed, int32_t *colour);
void *orc_bilu0_setup(int64_t n, int b, const int64_t *rp, const int32_t *col, const double *vt,
                      const int32_t *colour, int *status);
void orc_bilu0_solve(const void *h, const double *r, double *y);
void orc_bilu0_factors(const void *h, double *F);
void orc_bilu0_free(void *h);
/* Block ILU(1) (Sec. "Preconditioners": block ILU(k), k = 1 recommended):
 * the distance-2 order of a grid (cells (x + 2y + 3z) mod 7, other rows
 * first-fit from colour 7) and the factorisation on the level-1 pattern.
 * level 0 is orc_bilu0_setup.  The handle is freed by orc_bilu0_free; its
 * factors (orc_bilu0_factors) follow orc_bilu_pattern. */
int orc_colour_geo(int nx, int ny, int nz, int64_t n, const int64_t *rp, const int32_t *col,
                   int32_t *colour);
void *orc_biluk_setup(int64_t n, int b, const int64_t *rp, const int32_t *col, const double *vt,
                      const int32_t *colour, int level, int *status);
int64_t orc_bilu_nnz(const void *h);
void orc_bilu_pattern(const void *h, int64_t *rp, int32_t *col);
int orc_bilu_colours_independent(const void *h, const int32_t *colour);

/* ---- CPR-FPF preconditioner and FGMRES ---- */
#define ORC_CPR_FPF 0   /* F, P, F (Algorithm pc-fpf) */
#define ORC_CPR_FP 1    /* F, then P */
#define ORC_CPR_PF 2    /* P, then F */
typedef struct {
  double theta;      /* AMG strength threshold */
  int coarse_max;    /* stop coarsening at n <= coarse_max */
  int max_levels;
  int cheb_degree;
  uint32_t seed;
  int stages;        /* ORC_CPR_FPF / FP / PF */
  int decoupling;    /* ORC_DEC_* */
  int ilu_fill;      /* 0: block ILU(0), Jones-Plassmann colours; 1: block ILU(1), distance-2 order */
  int grid[3];       /* nx, ny, nz of the cells (rows 0 .. nx ny nz - 1), needed when ilu_fill = 1 */
} orc_cpr_opts;

void *orc_cpr_setup(int64_t n, int b, const int64_t *rp, const int32_t *col, const double *val,
                    const orc_cpr_opts *opts, int *status);
void orc_cpr_apply(const void *h, const double *v, double *z);
int orc_cpr_info(const void *h, int *n_levels, int *n_colours);
const void *orc_cpr_amg(const void *h);
void orc_cpr_colours(const void *h, int32_t *colour);
void orc_cpr_decoupled(const void *h, double *vt, double *dinv);
void orc_cpr_ilu_factors(const void *h, double *F);
const void *orc_cpr_ilu(const void *h);
void orc_cpr_free(void *h);

typedef struct {
  int iters;
  int restarts;
  int converged;
  double est_relres;
  double true_relres;
} orc_stats;

int orc_fgmres(int64_t n, int b, const int64_t *rp, const int32_t *col, const double *val,
               const void *cpr, const double *rhs, double *x, double rtol, int restart, int maxit,
               orc_stats *st, double *hist, int hist_cap);

/* Right-preconditioned BiCGSTAB (the Krylov solver of the paper's runs). */
int orc_bicgstab(int64_t n, int b, const int64_t *rp, const int32_t *col, const double *val,
                 const void *cpr, const double *rhs, double *x, double rtol, int maxit, orc_stats *st,
                 double *hist, int hist_cap);

/* ---- adjoint ---- */
void orc_outer_product(int64_t n, int b, const int64_t *rp, const int32_t *col,
                       const double *lambda, const double *x, double *dA);
int orc_chain_theta(int nx, int ny, int nz, int b, const double *k, double kvkh, double c_t,
                    const double *M, const int64_t *rp, const int32_t *col, const double *dA,
                    double *dtheta);

/* ---- thermal model: residual and Jacobian of one Newton step (trs_thermal.c) ----
 * One component set: water (water and gas phases) and one heavy-oil component
 * (oil phase).  Units: p kPa, T C, lengths m, time day, amounts gmol, energy kJ,
 * permeability mD, viscosity cP. */
typedef struct {
  double dx, dy, dz;          /* cell sizes */
  double depth_top;           /* depth of the top face of layer 0 (z grows downward) */
  double dt;                  /* time step */
  double kvkh;                /* vertical / horizontal permeability */
  double gravity;             /* m/s^2 */
  double phi_ref, cpor, ctpor, p_ref, T_ref;
  double cp1_r, cp2_r;        /* rock heat capacity, kJ/(m^3 C) and kJ/(m^3 C^2) */
  double kt_w, kt_o, kt_g, kt_r;  /* thermal conductivities, kJ/(m day C) */
  double rho_w_ref, cp_w, ct1_w, ct2_w, cpt_w, mw_w;
  double avisc_w, bvisc_w;    /* mu_w = avisc exp(bvisc / T_K) */
  double kv1, kv2, kv3, kv4, kv5, per_eps;
  double tc_w, pc_w;          /* critical temperature (C) and pressure (kPa) of water */
  double cpg[5];              /* gas heat-capacity polynomial of water, kJ/(gmol C^(k+1)) */
  double hvr, ev;             /* heat of vaporisation hvr (T_c - T)^ev */
  double rho_o_ref, cp_o, ct1_o, ct2_o, cpt_o, mw_o;
  double avisc_o, bvisc_o;
  double cpl1_o;              /* liquid heat capacity of the oil component, kJ/(gmol C) */
  double mug_a, mug_b;        /* mu_g = mug_a + mug_b T (T in C) */
  double h_inj;               /* enthalpy of injected steam, kJ/gmol */
  double R_gas;               /* gas constant, kJ/(gmol K) */
} orc_thermal_params;

/* Residual R(u) (n*4 doubles; cells then wells, wells' padding entries
 * R = u) and Jacobian dR/du on the pattern rp/col (that of orc_assemble for
 * the same grid and perforations), values in canonical BSR order.  rows:
 * NULL for every row, else the n_rows cell rows to compute (the well rows are
 * always computed; other entries are left as they are, zero them first).
 * swt: nswt x 3 (S_w, k_rw, k_row); slt: nslt x 3 (S_l, k_rg, k_rog).
 * well_type: 0 = injector at a fixed rate, 1 = producer at a fixed BHP. */
int orc_thermal_residual(int nx, int ny, int nz, int nw, int64_t np, const orc_thermal_params *P,
                         const double *swt, int nswt, const double *slt, int nslt, const double *k,
                         const int32_t *perf_well, const int32_t *perf_cell, const double *wi,
                         const int32_t *well_type, const double *well_target, const uint8_t *gas,
                         const double *u, const double *u_old, int64_t n_rows, const int64_t *rows, double *R);
int orc_thermal_jacobian(int nx, int ny, int nz, int nw, int64_t np, const orc_thermal_params *P,
                         const double *swt, int nswt, const double *slt, int nslt, const double *k,
                         const int32_t *perf_well, const int32_t *perf_cell, const double *wi,
                         const int32_t *well_type, const double *well_target, const uint8_t *gas,
                         const double *u, const double *u_old, int64_t n_rows, const int64_t *rows,
                         const int64_t *rp, const int32_t *col, double *val);
void orc_thermal_props(const orc_thermal_params *P, const double *swt, int nswt, const double *slt, int nslt,
                       const double *u, double *out);
double orc_rk_z(double A, double B);
void orc_thermal_totals(int nx, int ny, int nz, const orc_thermal_params *P, const double *swt, int nswt,
                        const double *slt, int nslt, const double *u, double *out);
void orc_thermal_well_sources(int nx, int ny, int nz, int nw, int64_t np, const orc_thermal_params *P,
                              const double *swt, int nswt, const double *slt, int nslt,
                              const int32_t *perf_well, const int32_t *perf_cell, const double *wi,
                              const int32_t *well_type, const double *u, double *out);

#ifdef __cplusplus
}
#endif
#endif
