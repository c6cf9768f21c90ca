/*
 * trs_thermal.c -- residual and Jacobian of the thermal reservoir model for
 * one Newton step (oracle).
 *
 * TEST INFRASTRUCTURE ONLY: used by tests, the smoke check and the CPU
 * baseline leg of the benchmark, never by the product path.  Shares no code,
 * header or table with the CUDA library.
 *
 * Model (Liu & Chen, arXiv 1812.03952, Sec. "Mathematical Model"), restricted
 * to one component set: a water component present in the water and gas
 * phases and one heavy-oil component present in the oil phase only (the
 * paper's component assumptions, with no light oil and no non-condensable
 * gas).  Unknowns per cell, natural variables (Sec. "Spatial
 * Discretization"): u = (p, S_w, S_g, T); S_o = 1 - S_w - S_g.  Equations
 * per cell:
 *   0  water moles   (Eq. eq4.2)   d/dt[phi(rho_w S_w + rho_g S_g)] + div(...) = q
 *   1  oil moles     (Eq. eq4.2)   d/dt[phi rho_o S_o] + div(...) = q
 *   2  energy        (Eq. eq4.3)   d/dt[phi sum rho S U + (1 - phi_ref) U_r] + ...
 *   3  gas constraint (Sec. "Spatial Discretization"): sum_i y_i - 1 = 0 when
 *      the gas phase exists, S_g = 0 when it does not.  The gas phase holds
 *      water only, so y_W = K*_W x_W with x_W = 1 (water phase is pure
 *      water): the constraint is K*_W(p, T, S_w) - 1 = 0.
 * Backward Euler in time (Sec. "Time Discretization"); two-point fluxes with
 * harmonic geometric transmissibility and upstream phase properties (Sec.
 * "Spatial Discretization"); Peaceman well terms (Sec. "Well Modeling",
 * Eq. well-model; unweighted mobility for injectors, fixed-rate and fixed-BHP
 * well equations).  Property correlations: Darcy (Eq. eq4.1), K-value with
 * the PER modification (Sec. "Phase Equilibrium Constraints"),
 * Redlich-Kwong Z factor (Sec. "Compressibility Factor of Real Gas"),
 * densities, viscosities, porosity, relative permeabilities by table with
 * Stone's model II, enthalpies and internal energies (Secs. "Density"
 * through "Energy").
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   - face gravity density: saturation-weighted mean of the two cells'
 *     gamma_a = rho_a * M_a * g, the plain mean when both saturations are 0;
 *   - face thermal conductivity: harmonic mean of the cells' bulk K_T
 *     (simple mixing rule of Sec. "Energy Conservation Equation");
 *   - relative-permeability tables: piecewise linear, constant beyond the
 *     ends; Stone II k_ro clipped at 0;
 *   - heat loss to the over/underburden (Vinsome) is left out;
 *   - producers: implicit cell mobilities, Q_a = WI c_u lambda_a (p_b - p);
 *     injectors: unweighted mobility Q = WI_u (p_b - p) of steam with a
 *     given enthalpy; well equations: injectors sum_m Q_m = q_target,
 *     producers p_b = p_target.
 *
 * The Jacobian is computed by complex-step differentiation of the residual
 * (Squire & Trapp, SIAM Review 40(1), 1998): dR/du_k = Im R(u + i h e_k) / h
 * with h = 1e-30, exact to rounding because no difference is taken.  So the
 * oracle states only the residual; every derivative follows from it.
 * Compiled with -ffp-contract=off like the rest of the oracle.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "trs_oracle.h"

typedef double complex cplx;

#define NV 4             /* unknowns per cell */
#define CS_H 1e-30       /* complex-step size */
#define C_UNIT 8.5270e-5 /* 86400 s/day * 9.869233e-16 m^2/mD * 1e3 Pa/kPa / 1e-3 Pa s/cP */

/* ---------------------------------------------------------------- helpers */
static double re(cplx z) { return creal(z); }

/* piecewise-linear interpolation of column c of an n x 3 table at s (by the
 * real part) on the closed interval of the table, constant beyond its ends:
 * at an end point the derivative is that of the end segment */
static cplx table(const double *tab, int n, int c, cplx s) {
  if (re(s) < tab[0]) return tab[c];
  if (re(s) > tab[(n - 1) * 3]) return tab[(n - 1) * 3 + c];
  int i = 0;
  while (i + 1 < n - 1 && re(s) >= tab[(i + 1) * 3]) i++;
  double x0 = tab[i * 3], x1 = tab[(i + 1) * 3], y0 = tab[i * 3 + c], y1 = tab[(i + 1) * 3 + c];
  return y0 + (y1 - y0) * (s - x0) / (x1 - x0);
}

/* ----------------------------------------------------------- properties */
/* Cell properties at state u (Sec. "Mathematical Model"). */
typedef struct {
  cplx phi;                 /* porosity */
  cplx S[3];                /* saturations w, o, g */
  cplx rho[3];              /* molar densities gmol/m^3 */
  cplx lam[3];              /* k_r rho / mu */
  cplx H[3];                /* phase enthalpies kJ/gmol */
  cplx U[3];                /* phase internal energies kJ/gmol */
  cplx gam[3];              /* gravity gradient rho * M * g, kPa/m */
  cplx Ur;                  /* rock internal energy kJ/m^3 */
  cplx KT;                  /* bulk thermal conductivity */
  cplx Kstar;               /* PER water K-value */
} orc_props;

/* Largest real root of Z^3 - Z^2 + (A - B - B^2) Z - A B = 0 (Redlich-Kwong),
 * by Newton's method from above the largest root, in complex arithmetic so
 * that the complex step carries through. */
static cplx rk_z(cplx A, cplx B) {
  cplx c1 = A - B - B * B, c0 = -A * B;
  /* Starting point.  Above the largest root f is increasing and convex, so
   * Newton's method from above converges to it -- unless f's local minimum
   * (the larger stationary point z_m) lies above zero.  Then the only real
   * root lies left of the local maximum, where f is increasing and concave,
   * and Newton's method from z = 0 (f(0) = -AB < 0) climbs to it. */
  double z0 = 1.0 + fabs(re(c1)) + fabs(re(c0));
  const double disc = 1.0 - 3.0 * re(c1);
  if (disc > 0.0) {
    const double zm = (1.0 + sqrt(disc)) / 3.0;
    if (((zm - 1.0) * zm + re(c1)) * zm + re(c0) > 0.0) z0 = 0.0;
  }
  cplx z = z0;
  for (int it = 0; it < 200; it++) {
    cplx f = ((z - 1.0) * z + c1) * z + c0;
    cplx fp = (3.0 * z - 2.0) * z + c1;
    cplx dz = f / fp;
    z = z - dz;
    if (fabs(re(dz)) <= 1e-16 * fabs(re(z))) break;
  }
  /* two more steps settle the complex part at the converged root */
  for (int it = 0; it < 2; it++) {
    cplx f = ((z - 1.0) * z + c1) * z + c0;
    cplx fp = (3.0 * z - 2.0) * z + c1;
    z = z - f / fp;
  }
  return z;
}

/* Water K-value K_W(p, T) = (kv1/p + kv2 p + kv3) exp(kv4 / (T - kv5)), Sec.
 * "Phase Equilibrium Constraints" (p in kPa, T in C). */
static cplx kvalue_w(const orc_thermal_params *P, cplx p, cplx T) {
  return (P->kv1 / p + P->kv2 * p + P->kv3) * cexp(P->kv4 / (T - P->kv5));
}

/* Gas-based water enthalpy H_gW(T) = integral from T_ref of the heat-capacity
 * polynomial (Sec. "Energy"), kJ/gmol. */
static cplx h_gas_w(const orc_thermal_params *P, cplx T) {
  cplx h = 0.0, tp = T, rp = P->T_ref;
  for (int k = 0; k < 5; k++) {
    h = h + P->cpg[k] * (tp - rp) / (double)(k + 1);
    tp = tp * T;
    rp = rp * P->T_ref;
  }
  return h;
}

/* Heat of vaporisation hvr (T_c - T)^ev below the critical temperature. */
static cplx h_vap_w(const orc_thermal_params *P, cplx T) {
  if (re(T) >= P->tc_w) return 0.0;
  return P->hvr * cexp(P->ev * clog(P->tc_w - T));
}

static void cell_props(const orc_thermal_params *P, const double *swt, int nswt, const double *slt,
                       int nslt, const cplx *u, orc_props *o) {
  const cplx p = u[0], Sw = u[1], Sg = u[2], T = u[3];
  const cplx So = 1.0 - Sw - Sg;
  const cplx TK = T + 273.15, dp = p - P->p_ref, dT = T - P->T_ref;
  o->S[0] = Sw;
  o->S[1] = So;
  o->S[2] = Sg;
  /* porosity, linear form (Sec. "Porosity") */
  o->phi = P->phi_ref * (1.0 + P->cpor * dp - P->ctpor * dT);
  /* densities (Sec. "Density") */
  o->rho[0] = P->rho_w_ref * cexp(P->cp_w * dp - P->ct1_w * dT - 0.5 * P->ct2_w * dT * dT + P->cpt_w * dp * dT);
  o->rho[1] = P->rho_o_ref * cexp(P->cp_o * dp - P->ct1_o * dT - 0.5 * P->ct2_o * dT * dT + P->cpt_o * dp * dT);
  {
    /* pure-water gas: the mixing rule gives T_crit = T_c and p_crit = p_c */
    const double TcK = P->tc_w + 273.15;
    cplx A = 0.427480 * (p / P->pc_w) * cpow(TcK / TK, 2.5);
    cplx B = 0.086640 * (p / P->pc_w) * (TcK / TK);
    cplx Z = rk_z(A, B);
    o->rho[2] = p / (Z * P->R_gas * TK);
  }
  /* viscosities (Sec. "Viscosity"), cP */
  cplx mu[3];
  mu[0] = P->avisc_w * cexp(P->bvisc_w / TK);
  mu[1] = P->avisc_o * cexp(P->bvisc_o / TK);
  mu[2] = P->mug_a + P->mug_b * T;
  /* relative permeabilities (Sec. "Relative Permeabilities"): swt (S_w, k_rw,
   * k_row), slt (S_l, k_rg, k_rog), Stone's model II for oil */
  cplx krw = table(swt, nswt, 1, Sw), krow = table(swt, nswt, 2, Sw);
  cplx Sl = 1.0 - Sg;
  cplx krg = table(slt, nslt, 1, Sl), krog = table(slt, nslt, 2, Sl);
  const double krocw = swt[2];
  cplx kro = krocw * ((krow / krocw + krw) * (krog / krocw + krg) - krw - krg);
  if (re(kro) < 0.0) kro = 0.0;
  o->lam[0] = krw * o->rho[0] / mu[0];
  o->lam[1] = kro * o->rho[1] / mu[1];
  o->lam[2] = krg * o->rho[2] / mu[2];
  /* enthalpies and internal energies (Sec. "Energy") */
  cplx Hg = h_gas_w(P, T);
  o->H[0] = Hg - h_vap_w(P, T);
  o->H[1] = P->cpl1_o * dT;
  o->H[2] = Hg;
  for (int a = 0; a < 3; a++) o->U[a] = o->H[a] - p / o->rho[a];
  o->Ur = P->cp1_r * dT + 0.5 * P->cp2_r * (T * T - P->T_ref * P->T_ref);
  /* gravity gradients, kPa/m */
  o->gam[0] = o->rho[0] * P->mw_w * P->gravity * 1e-3;
  o->gam[1] = o->rho[1] * P->mw_o * P->gravity * 1e-3;
  o->gam[2] = o->rho[2] * P->mw_w * P->gravity * 1e-3;
  /* bulk conductivity, simple mixing rule (Sec. "Energy Conservation Equation") */
  o->KT = o->phi * (Sw * P->kt_w + So * P->kt_o + Sg * P->kt_g) + (1.0 - o->phi) * P->kt_r;
  /* PER K-value of water (Sec. "Phase Equilibrium Constraints") */
  o->Kstar = Sw / (Sw + P->per_eps) * kvalue_w(P, p, T);
}

/* Accumulated amounts of water, oil and energy in a cell of volume V. */
static void amounts(const orc_thermal_params *P, const orc_props *o, double V, cplx *N) {
  N[0] = V * o->phi * (o->rho[0] * o->S[0] + o->rho[2] * o->S[2]);
  N[1] = V * o->phi * o->rho[1] * o->S[1];
  cplx e = 0.0;
  for (int a = 0; a < 3; a++) e = e + o->rho[a] * o->S[a] * o->U[a];
  N[2] = V * (o->phi * e + (1.0 - P->phi_ref) * o->Ur);
}

/* Water, oil and energy flowing out of cell i into cell j across one face:
 * T_geo lambda_up dPhi per phase (upstream by the sign of dPhi), enthalpy
 * carried at upstream, conduction T_cond (T_i - T_j). */
static void face_flux(const orc_props *oi, const orc_props *oj, cplx Ti_, cplx Tj_,
                      cplx pi, cplx pj, double zi, double zj, double Tgeo, double area_len, cplx *F) {
  F[0] = F[1] = F[2] = 0.0;
  for (int a = 0; a < 3; a++) {
    cplx ssum = oi->S[a] + oj->S[a];
    cplx g = (re(ssum) > 0.0) ? (oi->S[a] * oi->gam[a] + oj->S[a] * oj->gam[a]) / ssum
                              : 0.5 * (oi->gam[a] + oj->gam[a]);
    cplx dphi = (pi - pj) - g * (zi - zj);
    const orc_props *up = re(dphi) >= 0.0 ? oi : oj;
    cplx f = Tgeo * up->lam[a] * dphi;
    if (a == 1) F[1] = F[1] + f;
    else F[0] = F[0] + f;
    F[2] = F[2] + up->H[a] * f;
  }
  cplx kt = (re(oi->KT + oj->KT) > 0.0) ? 2.0 * oi->KT * oj->KT / (oi->KT + oj->KT) : 0.0;
  F[2] = F[2] + area_len * kt * (Ti_ - Tj_);
}

/* ------------------------------------------------------------ the model */
typedef struct {
  int nx, ny, nz, nw;
  int64_t n_c, np;
  const orc_thermal_params *P;
  const double *swt, *slt;
  int nswt, nslt;
  const double *k;
  const int32_t *perf_well, *perf_cell;
  const double *wi;
  const int32_t *well_type;   /* 0 injector (rate), 1 producer (BHP) */
  const double *well_target;  /* rate (gmol/day) or BHP (kPa) */
  const uint8_t *gas;
  const double *u_old;
} model;

static int64_t neighbour_of(const model *m, int64_t c, int d, int *dir_axis) {
  static const int D[6][3] = {{0, 0, -1}, {0, -1, 0}, {-1, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  int64_t x = c % m->nx, y = (c / m->nx) % m->ny, z = c / ((int64_t)m->nx * m->ny);
  x += D[d][0];
  y += D[d][1];
  z += D[d][2];
  *dir_axis = D[d][0] ? 0 : (D[d][1] ? 1 : 2);
  if (x < 0 || y < 0 || z < 0 || x >= m->nx || y >= m->ny || z >= m->nz) return -1;
  return x + (int64_t)m->nx * (y + (int64_t)m->ny * z);
}

static double depth_of(const model *m, int64_t c) {
  int64_t z = c / ((int64_t)m->nx * m->ny);
  return m->P->depth_top + ((double)z + 0.5) * m->P->dz;
}

/* geometric factors of the face of cell c in direction d toward cell j */
static void face_geometry(const model *m, int64_t c, int64_t j, int axis, double *Tgeo, double *area_len) {
  const orc_thermal_params *P = m->P;
  double al = axis == 0 ? P->dy * P->dz / P->dx : (axis == 1 ? P->dx * P->dz / P->dy : P->dx * P->dy / P->dz);
  double ki = m->k[c], kj = m->k[j];
  double kh = (ki + kj > 0.0) ? 2.0 * ki * kj / (ki + kj) : 0.0;
  if (axis == 2) kh = kh * P->kvkh;
  *Tgeo = C_UNIT * kh * al;
  *area_len = al;
}

/* Residual block of cell c's equations contributed by cell c itself and the
 * faces to its neighbours, with the states of c and its neighbours given
 * (complex); u_nb[d] is the state of the neighbour in direction d. */
static void cell_residual(const model *m, int64_t c, const cplx *uc, cplx uw_of_perf(const model *, int64_t, void *),
                          void *ctx, cplx (*u_nb)[NV], cplx *R) {
  const orc_thermal_params *P = m->P;
  const double V = P->dx * P->dy * P->dz;
  orc_props oc, oold, on;
  cell_props(P, m->swt, m->nswt, m->slt, m->nslt, uc, &oc);
  cplx uo[NV];
  for (int v = 0; v < NV; v++) uo[v] = m->u_old[c * NV + v];
  cell_props(P, m->swt, m->nswt, m->slt, m->nslt, uo, &oold);
  cplx N[3], No[3];
  amounts(P, &oc, V, N);
  amounts(P, &oold, V, No);
  for (int e = 0; e < 3; e++) R[e] = (N[e] - No[e]) / P->dt;
  for (int d = 0; d < 6; d++) {
    int axis;
    int64_t j = neighbour_of(m, c, d, &axis);
    if (j < 0) continue;
    double Tgeo, al;
    face_geometry(m, c, j, axis, &Tgeo, &al);
    cell_props(P, m->swt, m->nswt, m->slt, m->nslt, u_nb[d], &on);
    cplx F[3];
    face_flux(&oc, &on, uc[3], u_nb[d][3], uc[0], u_nb[d][0], depth_of(m, c), depth_of(m, j), Tgeo, al, F);
    for (int e = 0; e < 3; e++) R[e] = R[e] + F[e];
  }
  /* wells: Q > 0 flows into the cell */
  for (int64_t t = 0; t < m->np; t++) {
    if (m->perf_cell[t] != c) continue;
    int w = m->perf_well[t];
    cplx pb = uw_of_perf(m, w, ctx);
    if (m->well_type[w] == 0) {
      cplx Q = m->wi[t] * (pb - uc[0]);
      R[0] = R[0] - Q;
      R[2] = R[2] - Q * P->h_inj;
    } else {
      for (int a = 0; a < 3; a++) {
        cplx Q = m->wi[t] * C_UNIT * oc.lam[a] * (pb - uc[0]);
        if (a == 1) R[1] = R[1] - Q;
        else R[0] = R[0] - Q;
        R[2] = R[2] - oc.H[a] * Q;
      }
    }
  }
  /* gas constraint */
  R[3] = m->gas[c] ? oc.Kstar - 1.0 : uc[2];
}

/* the BHP of well w: the real state, or the perturbed one */
typedef struct {
  const double *u;
  int64_t n_c;
  int pert_well;
  cplx pert;
} bhp_ctx;

static cplx bhp_of(const model *m, int64_t w, void *ctx) {
  bhp_ctx *b = (bhp_ctx *)ctx;
  if (w == b->pert_well) return b->pert;
  return b->u[(m->n_c + w) * NV];
}

static void gather_neighbours(const model *m, int64_t c, const double *u, cplx (*u_nb)[NV]) {
  for (int d = 0; d < 6; d++) {
    int axis;
    int64_t j = neighbour_of(m, c, d, &axis);
    for (int v = 0; v < NV; v++) u_nb[d][v] = j >= 0 ? u[j * NV + v] : 0.0;
  }
}

/* well row residual: injectors sum_m WI_u (p_b - p_m) - q_target; producers
 * p_b - p_target */
static cplx well_residual(const model *m, int w, cplx pb, const cplx *p_perf_override, int64_t override_perf,
                          const double *u) {
  if (m->well_type[w] == 1) return pb - m->well_target[w];
  cplx q = 0.0;
  for (int64_t t = 0; t < m->np; t++) {
    if (m->perf_well[t] != w) continue;
    cplx pc = (t == override_perf) ? *p_perf_override : (cplx)u[(int64_t)m->perf_cell[t] * NV];
    q = q + m->wi[t] * (pb - pc);
  }
  return q - m->well_target[w];
}

static int64_t find_col(const int64_t *rp, const int32_t *col, int64_t i, int64_t j) {
  int64_t lo = rp[i], hi = rp[i + 1] - 1;
  while (lo <= hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (col[mid] == j) return mid;
    if (col[mid] < j) lo = mid + 1;
    else hi = mid - 1;
  }
  return -1;
}

static void init_model(model *m, int nx, int ny, int nz, int nw, int64_t np, const orc_thermal_params *P,
                       const double *swt, int nswt, const double *slt, int nslt, const double *k,
                       const int32_t *perf_well, const int32_t *perf_cell, const double *wi,
                       const int32_t *well_type, const double *well_target, const uint8_t *gas,
                       const double *u_old) {
  m->nx = nx;
  m->ny = ny;
  m->nz = nz;
  m->nw = nw;
  m->n_c = (int64_t)nx * ny * nz;
  m->np = np;
  m->P = P;
  m->swt = swt;
  m->slt = slt;
  m->nswt = nswt;
  m->nslt = nslt;
  m->k = k;
  m->perf_well = perf_well;
  m->perf_cell = perf_cell;
  m->wi = wi;
  m->well_type = well_type;
  m->well_target = well_target;
  m->gas = gas;
  m->u_old = u_old;
}

int orc_thermal_residual(int nx, int ny, int nz, int nw, int64_t np, const orc_thermal_params *P,
                         const double *swt, int nswt, const double *slt, int nslt, const double *k,
                         const int32_t *perf_well, const int32_t *perf_cell, const double *wi,
                         const int32_t *well_type, const double *well_target, const uint8_t *gas,
                         const double *u, const double *u_old, int64_t n_rows, const int64_t *rows, double *R) {
  if (nswt < 2 || nslt < 2 || P->dt <= 0.0) return -1;
  model m;
  init_model(&m, nx, ny, nz, nw, np, P, swt, nswt, slt, nslt, k, perf_well, perf_cell, wi, well_type, well_target,
             gas, u_old);
  bhp_ctx bc = {u, m.n_c, -1, 0.0};
  const int64_t count = rows ? n_rows : m.n_c;
  for (int64_t r = 0; r < count; r++) {
    const int64_t c = rows ? rows[r] : r;
    if (c >= m.n_c) continue;
    cplx uc[NV], u_nb[6][NV], Rc[NV];
    for (int v = 0; v < NV; v++) uc[v] = u[c * NV + v];
    gather_neighbours(&m, c, u, u_nb);
    cell_residual(&m, c, uc, bhp_of, &bc, u_nb, Rc);
    for (int v = 0; v < NV; v++) R[c * NV + v] = re(Rc[v]);
  }
  for (int w = 0; w < nw; w++) {
    int64_t row = m.n_c + w;
    R[row * NV] = re(well_residual(&m, w, u[row * NV], NULL, -1, u));
    for (int v = 1; v < NV; v++) R[row * NV + v] = u[row * NV + v];   /* padding rows: identity, zero target */
  }
  return 0;
}

int orc_thermal_jacobian(int nx, int ny, int nz, int nw, int64_t np, const orc_thermal_params *P,
                         const double *swt, int nswt, const double *slt, int nslt, const double *k,
                         const int32_t *perf_well, const int32_t *perf_cell, const double *wi,
                         const int32_t *well_type, const double *well_target, const uint8_t *gas,
                         const double *u, const double *u_old, int64_t n_rows, const int64_t *rows,
                         const int64_t *rp, const int32_t *col, double *val) {
  if (nswt < 2 || nslt < 2 || P->dt <= 0.0) return -1;
  model m;
  init_model(&m, nx, ny, nz, nw, np, P, swt, nswt, slt, nslt, k, perf_well, perf_cell, wi, well_type, well_target,
             gas, u_old);
  const int64_t n = m.n_c + nw, bb = NV * NV;
  if (!rows) memset(val, 0, sizeof(double) * (size_t)(rp[n] * bb));
  const int64_t count = rows ? n_rows : m.n_c;
  for (int64_t r = 0; r < count; r++) {
    const int64_t c = rows ? rows[r] : r;
    if (c >= m.n_c) continue;
    cplx uc[NV], u_nb[6][NV], Rc[NV];
    /* own columns */
    int64_t pd = find_col(rp, col, c, c);
    if (pd < 0) return -1;
    for (int v = 0; v < NV; v++) {
      bhp_ctx bc = {u, m.n_c, -1, 0.0};
      for (int q = 0; q < NV; q++) uc[q] = u[c * NV + q];
      uc[v] = uc[v] + I * CS_H;
      gather_neighbours(&m, c, u, u_nb);
      cell_residual(&m, c, uc, bhp_of, &bc, u_nb, Rc);
      for (int r = 0; r < NV; r++) val[pd * bb + r * NV + v] = cimag(Rc[r]) / CS_H;
    }
    /* neighbour columns */
    for (int d = 0; d < 6; d++) {
      int axis;
      int64_t j = neighbour_of(&m, c, d, &axis);
      if (j < 0) continue;
      int64_t pj = find_col(rp, col, c, j);
      if (pj < 0) return -1;
      for (int v = 0; v < NV; v++) {
        bhp_ctx bc = {u, m.n_c, -1, 0.0};
        for (int q = 0; q < NV; q++) uc[q] = u[c * NV + q];
        gather_neighbours(&m, c, u, u_nb);
        u_nb[d][v] = u_nb[d][v] + I * CS_H;
        cell_residual(&m, c, uc, bhp_of, &bc, u_nb, Rc);
        for (int r = 0; r < NV; r++) val[pj * bb + r * NV + v] = cimag(Rc[r]) / CS_H;
      }
    }
    /* well (BHP) columns: only slot 0 of a well block is a real unknown */
    for (int64_t t = 0; t < np; t++) {
      if (perf_cell[t] != c) continue;
      int w = perf_well[t];
      int64_t pw = find_col(rp, col, c, m.n_c + w);
      if (pw < 0) return -1;
      bhp_ctx bc = {u, m.n_c, w, u[(m.n_c + w) * NV] + I * CS_H};
      for (int q = 0; q < NV; q++) uc[q] = u[c * NV + q];
      gather_neighbours(&m, c, u, u_nb);
      cell_residual(&m, c, uc, bhp_of, &bc, u_nb, Rc);
      for (int r = 0; r < NV; r++) val[pw * bb + r * NV + 0] = cimag(Rc[r]) / CS_H;
    }
  }
  for (int w = 0; w < nw; w++) {
    int64_t row = m.n_c + w;
    int64_t pd = find_col(rp, col, row, row);
    if (pd < 0) return -1;
    cplx pb = u[row * NV] + I * CS_H;
    val[pd * bb] = cimag(well_residual(&m, w, pb, NULL, -1, u)) / CS_H;
    for (int s = 1; s < NV; s++) val[pd * bb + s * NV + s] = 1.0;
    for (int64_t t = 0; t < np; t++) {
      if (perf_well[t] != w) continue;
      int64_t pc = find_col(rp, col, row, perf_cell[t]);
      if (pc < 0) return -1;
      cplx pp = u[(int64_t)perf_cell[t] * NV] + I * CS_H;
      val[pc * bb] = cimag(well_residual(&m, w, u[row * NV], &pp, t, u)) / CS_H;
    }
  }
  return 0;
}

/* Cell properties at one real state, for the property pins: out[0..] =
 * phi, rho_w, rho_o, rho_g, lam_w, lam_o, lam_g, H_w, H_o, H_g, U_w, U_o,
 * U_g, U_r, K_T, K*_W (16 values). */
void orc_thermal_props(const orc_thermal_params *P, const double *swt, int nswt, const double *slt, int nslt,
                       const double *u, double *out) {
  cplx uc[NV];
  for (int v = 0; v < NV; v++) uc[v] = u[v];
  orc_props o;
  cell_props(P, swt, nswt, slt, nslt, uc, &o);
  double *q = out;
  *q++ = re(o.phi);
  for (int a = 0; a < 3; a++) *q++ = re(o.rho[a]);
  for (int a = 0; a < 3; a++) *q++ = re(o.lam[a]);
  for (int a = 0; a < 3; a++) *q++ = re(o.H[a]);
  for (int a = 0; a < 3; a++) *q++ = re(o.U[a]);
  *q++ = re(o.Ur);
  *q++ = re(o.KT);
  *q++ = re(o.Kstar);
}

/* Redlich-Kwong Z factor for given A, B (real), for the pins. */
double orc_rk_z(double A, double B) { return re(rk_z(A, B)); }

/* Total water, oil and energy in the cells at state u (for the conservation
 * pins): out[3]. */
void orc_thermal_totals(int nx, int ny, int nz, const orc_thermal_params *P, const double *swt, int nswt,
                        const double *slt, int nslt, const double *u, double *out) {
  const int64_t n_c = (int64_t)nx * ny * nz;
  const double V = P->dx * P->dy * P->dz;
  out[0] = out[1] = out[2] = 0.0;
  for (int64_t c = 0; c < n_c; c++) {
    cplx uc[NV], N[3];
    for (int v = 0; v < NV; v++) uc[v] = u[c * NV + v];
    orc_props o;
    cell_props(P, swt, nswt, slt, nslt, uc, &o);
    amounts(P, &o, V, N);
    for (int e = 0; e < 3; e++) out[e] += re(N[e]);
  }
}

/* Water, oil and energy that the wells put into the cells at state u
 * (out[3], positive = injected), for the conservation pins. */
void orc_thermal_well_sources(int nx, int ny, int nz, int nw, int64_t np, const orc_thermal_params *P,
                              const double *swt, int nswt, const double *slt, int nslt,
                              const int32_t *perf_well, const int32_t *perf_cell, const double *wi,
                              const int32_t *well_type, const double *u, double *out) {
  const int64_t n_c = (int64_t)nx * ny * nz;
  out[0] = out[1] = out[2] = 0.0;
  (void)nw;
  for (int64_t t = 0; t < np; t++) {
    int64_t c = perf_cell[t];
    int w = perf_well[t];
    double pb = u[(n_c + w) * NV], pc = u[c * NV];
    if (well_type[w] == 0) {
      double Q = wi[t] * (pb - pc);
      out[0] += Q;
      out[2] += Q * P->h_inj;
    } else {
      cplx uc[NV];
      for (int v = 0; v < NV; v++) uc[v] = u[c * NV + v];
      orc_props o;
      cell_props(P, swt, nswt, slt, nslt, uc, &o);
      for (int a = 0; a < 3; a++) {
        double Q = wi[t] * C_UNIT * re(o.lam[a]) * (pb - pc);
        if (a == 1) out[1] += Q;
        else out[0] += Q;
        out[2] += re(o.H[a]) * Q;
      }
    }
  }
}
