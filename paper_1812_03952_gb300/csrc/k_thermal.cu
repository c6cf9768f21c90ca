// Jacobian and residual of one Newton step of the thermal reservoir model
// (Liu & Chen, arXiv 1812.03952, Sec. "Mathematical Model" and Sec.
// "Numerical Methods"), for one component set: water in the water and gas
// phases, one heavy-oil component in the oil phase.  Unknowns per cell
// (p, S_w, S_g, T); equations: water moles, oil moles (Eq. eq4.2), energy
// (Eq. eq4.3), and the gas constraint (K*_W - 1 = 0 with gas, S_g = 0
// without; Sec. "Spatial Discretization").  Backward Euler (Sec. "Time
// Discretization"), two-point fluxes with harmonic geometric transmissibility
// and upstream phase properties (Sec. "Spatial Discretization"), Peaceman
// well terms (Sec. "Well Modeling").
//
// Derivatives are carried by forward-mode dual numbers (value and the four
// partial derivatives with respect to one cell's unknowns), so the Jacobian is
// the exact derivative of the residual this file computes.  Four kernels:
//   k_thermal_cells: per cell, the properties with their derivatives (kept
//     for the neighbours), the accumulation terms and the gas constraint;
//   k_thermal_faces: per face, once, the flux with its derivatives with
//     respect to both cells (a dual-number pass each), kept for the rows, and
//     the two off-diagonal blocks it gives;
//   k_thermal_rows:  per cell row, the six faces' terms and the
//     perforations, into the residual, the diagonal block and the tail;
//   k_thermal_wells: per well, the well equation.
#include <type_traits>

#include "trs_api_common.cuh"
#include "trs_kernels.cuh"

namespace trs {
namespace {

constexpr int kThreads = 128;
inline unsigned grid_of(int64_t n) { return (unsigned)((n + kThreads - 1) / kThreads); }

// 86400 s/day * 9.869233e-16 m^2/mD * 1e3 Pa/kPa / (1e-3 Pa s/cP)
constexpr double kUnit = 8.5270e-5;
constexpr int kNV = 4;

// ----------------------------------------------------------- dual numbers
struct D4 {
  double v;
  double d[kNV];
};

__device__ __forceinline__ D4 cst(double a) { return D4{a, {0.0, 0.0, 0.0, 0.0}}; }
__device__ __forceinline__ D4 var(double a, int k) {
  D4 r = cst(a);
  r.d[k] = 1.0;
  return r;
}
__device__ __forceinline__ D4 operator+(const D4 &a, const D4 &b) {
  D4 r;
  r.v = a.v + b.v;
#pragma unroll
  for (int k = 0; k < kNV; k++) r.d[k] = a.d[k] + b.d[k];
  return r;
}
__device__ __forceinline__ D4 operator-(const D4 &a, const D4 &b) {
  D4 r;
  r.v = a.v - b.v;
#pragma unroll
  for (int k = 0; k < kNV; k++) r.d[k] = a.d[k] - b.d[k];
  return r;
}
__device__ __forceinline__ D4 operator*(const D4 &a, const D4 &b) {
  D4 r;
  r.v = a.v * b.v;
#pragma unroll
  for (int k = 0; k < kNV; k++) r.d[k] = a.d[k] * b.v + a.v * b.d[k];
  return r;
}
__device__ __forceinline__ D4 operator/(const D4 &a, const D4 &b) {
  D4 r;
  const double ib = 1.0 / b.v;
  r.v = a.v * ib;
#pragma unroll
  for (int k = 0; k < kNV; k++) r.d[k] = (a.d[k] - r.v * b.d[k]) * ib;
  return r;
}
__device__ __forceinline__ D4 operator+(const D4 &a, double b) {
  D4 r = a;
  r.v += b;
  return r;
}
__device__ __forceinline__ D4 operator+(double b, const D4 &a) { return a + b; }
__device__ __forceinline__ D4 operator-(const D4 &a, double b) {
  D4 r = a;
  r.v -= b;
  return r;
}
__device__ __forceinline__ D4 operator-(double b, const D4 &a) {
  D4 r;
  r.v = b - a.v;
#pragma unroll
  for (int k = 0; k < kNV; k++) r.d[k] = -a.d[k];
  return r;
}
__device__ __forceinline__ D4 operator*(const D4 &a, double b) {
  D4 r;
  r.v = a.v * b;
#pragma unroll
  for (int k = 0; k < kNV; k++) r.d[k] = a.d[k] * b;
  return r;
}
__device__ __forceinline__ D4 operator*(double b, const D4 &a) { return a * b; }
__device__ __forceinline__ D4 operator/(const D4 &a, double b) {
  D4 r;
  r.v = a.v / b;
  const double ib = 1.0 / b;
#pragma unroll
  for (int k = 0; k < kNV; k++) r.d[k] = a.d[k] * ib;
  return r;
}
__device__ __forceinline__ D4 operator/(double a, const D4 &b) {
  D4 r;
  const double ib = 1.0 / b.v;
  r.v = a * ib;
#pragma unroll
  for (int k = 0; k < kNV; k++) r.d[k] = -r.v * b.d[k] * ib;
  return r;
}
__device__ __forceinline__ D4 dexp(const D4 &a) {
  D4 r;
  r.v = exp(a.v);
#pragma unroll
  for (int k = 0; k < kNV; k++) r.d[k] = r.v * a.d[k];
  return r;
}
__device__ __forceinline__ D4 dlog(const D4 &a) {
  D4 r;
  r.v = log(a.v);
#pragma unroll
  for (int k = 0; k < kNV; k++) r.d[k] = a.d[k] / a.v;
  return r;
}
// a^(5/2) = a^2 sqrt(a), d/da = (5/2) a sqrt(a) (a > 0)
__device__ __forceinline__ D4 dpow52(const D4 &a) {
  D4 r;
  const double q = sqrt(a.v);
  r.v = a.v * a.v * q;
  const double s = 2.5 * a.v * q;
#pragma unroll
  for (int k = 0; k < kNV; k++) r.d[k] = s * a.d[k];
  return r;
}

// the same operations on plain values (no derivative carried)
__device__ __forceinline__ double val(double x) { return x; }
__device__ __forceinline__ double val(const D4 &x) { return x.v; }
__device__ __forceinline__ double dexp(double a) { return exp(a); }
__device__ __forceinline__ double dlog(double a) { return log(a); }
__device__ __forceinline__ double dpow52(double a) { return a * a * sqrt(a); }
// the promotion of a value to a dual number with zero derivatives
__device__ __forceinline__ D4 dual(double a) { return cst(a); }
__device__ __forceinline__ D4 dual(const D4 &a) { return a; }

// ------------------------------------------------------------- properties
// piecewise-linear interpolation of column c of an n x 3 table on its closed
// interval, constant beyond the ends (the end segments' slopes at the ends);
// slope[2 i + c - 1] is the slope of column c on segment i (set on the host)
__device__ double table(const double *tab, const double *slope, int n, int c, double s) {
  if (s < tab[0]) return tab[c];
  if (s > tab[(n - 1) * 3]) return tab[(n - 1) * 3 + c];
  int i = 0;
  while (i + 1 < n - 1 && s >= tab[(i + 1) * 3]) i++;
  return tab[i * 3 + c] + slope[2 * i + c - 1] * (s - tab[i * 3]);
}

__device__ D4 table(const double *tab, const double *slope, int n, int c, const D4 &s) {
  if (s.v < tab[0]) return cst(tab[c]);
  if (s.v > tab[(n - 1) * 3]) return cst(tab[(n - 1) * 3 + c]);
  int i = 0;
  while (i + 1 < n - 1 && s.v >= tab[(i + 1) * 3]) i++;
  const double sl = slope[2 * i + c - 1];
  D4 r;
  r.v = tab[i * 3 + c] + sl * (s.v - tab[i * 3]);
#pragma unroll
  for (int k = 0; k < kNV; k++) r.d[k] = sl * s.d[k];
  return r;
}

// Largest real root of Z^3 - Z^2 + (A - B - B^2) Z - A B = 0 (Redlich-Kwong,
// Sec. "Compressibility Factor of Real Gas"): Newton's method on the values,
// then dZ = -(f_A dA + f_B dB) / f_Z.  Newton starts above the largest root,
// where f rises and is convex, unless f's local minimum (the larger
// stationary point) is above zero: the only real root is then left of the
// local maximum, where f rises and is concave, and Newton starts at z = 0
// (f(0) = -AB < 0).  The test is evaluated without contraction.
__device__ double rk_z(double a, double b) {
  const double c1 = a - b - b * b, c0 = -a * b;
  double z = 1.0 + fabs(c1) + fabs(c0);
  const double disc = 1.0 - 3.0 * c1;
  if (disc > 0.0) {
    const double zm = __ddiv_rn(__dadd_rn(1.0, sqrt(disc)), 3.0);
    const double fm = __dadd_rn(__dmul_rn(__dadd_rn(__dmul_rn(__dadd_rn(zm, -1.0), zm), c1), zm), c0);
    if (fm > 0.0) z = 0.0;
  }
  for (int it = 0; it < 200; it++) {
    const double f = ((z - 1.0) * z + c1) * z + c0;
    const double fp = (3.0 * z - 2.0) * z + c1;
    const double dz = f / fp;
    z = z - dz;
    if (fabs(dz) <= 1e-16 * fabs(z)) break;
  }
  return z;
}

__device__ D4 rk_z(const D4 &A, const D4 &B) {
  const double a = A.v, b = B.v;
  const double c1 = a - b - b * b;
  const double z = rk_z(a, b);
  const double fz = (3.0 * z - 2.0) * z + c1;
  const double fa = z - b, fb = -z - 2.0 * b * z - a, ifz = 1.0 / fz;
  D4 r;
  r.v = z;
#pragma unroll
  for (int k = 0; k < kNV; k++) r.d[k] = -(fa * A.d[k] + fb * B.d[k]) * ifz;
  return r;
}

template <class N>
struct CellProps {
  N phi, rho[3], lam[3], H[3], gam[3], KT, Kstar;
};

// N = D4: with the derivatives with respect to the cell's unknowns; N =
// double: values only (the old time level)
template <class N>
__device__ void cell_props(const trs_thermal_params &P, const ThermalTables &tb, const N &p, const N &Sw,
                           const N &Sg, const N &T, CellProps<N> &o) {
  const N So = 1.0 - Sw - Sg;
  const N TK = T + 273.15, dp = p - P.p_ref, dT = T - P.T_ref;
  o.phi = P.phi_ref * (1.0 + P.cpor * dp - P.ctpor * dT);
  o.rho[0] = P.rho_w_ref * dexp(P.cp_w * dp - P.ct1_w * dT - 0.5 * P.ct2_w * dT * dT + P.cpt_w * dp * dT);
  o.rho[1] = P.rho_o_ref * dexp(P.cp_o * dp - P.ct1_o * dT - 0.5 * P.ct2_o * dT * dT + P.cpt_o * dp * dT);
  {
    const double TcK = P.tc_w + 273.15;
    const N pr = p * (1.0 / P.pc_w), tr = TcK / TK;
    const N A = 0.427480 * pr * dpow52(tr);
    const N B = 0.086640 * pr * tr;
    const N Z = rk_z(A, B);
    o.rho[2] = p / (Z * P.R_gas * TK);
  }
  N mu[3];
  mu[0] = P.avisc_w * dexp(P.bvisc_w / TK);
  mu[1] = P.avisc_o * dexp(P.bvisc_o / TK);
  mu[2] = P.mug_a + P.mug_b * T;
  const N krw = table(tb.swt, tb.swt_slope, tb.nswt, 1, Sw), krow = table(tb.swt, tb.swt_slope, tb.nswt, 2, Sw);
  const N Sl = 1.0 - Sg;
  const N krg = table(tb.slt, tb.slt_slope, tb.nslt, 1, Sl), krog = table(tb.slt, tb.slt_slope, tb.nslt, 2, Sl);
  const double krocw = tb.swt[2];
  N kro = krocw * ((krow / krocw + krw) * (krog / krocw + krg) - krw - krg);
  if (val(kro) < 0.0) kro = kro * 0.0;
  o.lam[0] = krw * o.rho[0] / mu[0];
  o.lam[1] = kro * o.rho[1] / mu[1];
  o.lam[2] = krg * o.rho[2] / mu[2];
  // gas-based water enthalpy: integral of the heat-capacity polynomial from T_ref
  N hg = T * 0.0, tp = T;
  double rp = P.T_ref;
#pragma unroll
  for (int k = 0; k < 5; k++) {
    hg = hg + P.cpg[k] * (tp - rp) * (1.0 / (double)(k + 1));
    tp = tp * T;
    rp = rp * P.T_ref;
  }
  N hv = T * 0.0;
  if (val(T) < P.tc_w) hv = P.hvr * dexp(P.ev * dlog(P.tc_w - T));
  o.H[0] = hg - hv;
  o.H[1] = P.cpl1_o * dT;
  o.H[2] = hg;
  o.gam[0] = o.rho[0] * (P.mw_w * P.gravity * 1e-3);
  o.gam[1] = o.rho[1] * (P.mw_o * P.gravity * 1e-3);
  o.gam[2] = o.rho[2] * (P.mw_w * P.gravity * 1e-3);
  o.KT = o.phi * (Sw * P.kt_w + So * P.kt_o + Sg * P.kt_g) + (1.0 - o.phi) * P.kt_r;
  o.Kstar = Sw / (Sw + P.per_eps) * ((P.kv1 / p + P.kv2 * p + P.kv3) * dexp(P.kv4 / (T - P.kv5)));
}

// accumulated water and oil of a cell of volume V
template <class N>
__device__ void amounts(const CellProps<N> &o, const N &Sw, const N &Sg, double V, N (&Nm)[3]) {
  const N So = 1.0 - Sw - Sg;
  Nm[0] = V * o.phi * (o.rho[0] * Sw + o.rho[2] * Sg);
  Nm[1] = V * o.phi * o.rho[1] * So;
}

// accumulated energy: fluids' internal energy U = H - p / rho and the rock's
// (constant rock volume (1 - phi_ref) V, Sec. "Energy Conservation Equation")
template <class N>
__device__ N energy_amount(const trs_thermal_params &P, const CellProps<N> &o, const N &p, const N &Sw,
                           const N &Sg, const N &T, double V) {
  const N So = 1.0 - Sw - Sg;
  const N S[3] = {Sw, So, Sg};
  N e = T * 0.0;
#pragma unroll
  for (int a = 0; a < 3; a++) e = e + o.rho[a] * S[a] * (o.H[a] - p / o.rho[a]);
  const N dT = T - P.T_ref;
  const N Ur = P.cp1_r * dT + 0.5 * P.cp2_r * (T * T - P.T_ref * P.T_ref);
  return V * (o.phi * e + (1.0 - P.phi_ref) * Ur);
}

// Properties kept per cell for the flux kernel, structure of arrays:
// kProps dual numbers (lam[3], H[3], gam[3], K_T), each kNV + 1 doubles.
constexpr int kProps = 10;
constexpr int kPropDoubles = kProps * (kNV + 1);

__device__ __forceinline__ void store_d4(double *base, int64_t nc, int64_t c, int q, const D4 &x) {
  base[(int64_t)(q * (kNV + 1)) * nc + c] = x.v;
#pragma unroll
  for (int k = 0; k < kNV; k++) base[(int64_t)(q * (kNV + 1) + 1 + k) * nc + c] = x.d[k];
}
// the same property with its derivatives (wrt = true) or as a constant
__device__ __forceinline__ D4 load_d4(const double *base, int64_t nc, int64_t c, int q, bool wrt) {
  D4 x;
  x.v = base[(int64_t)(q * (kNV + 1)) * nc + c];
#pragma unroll
  for (int k = 0; k < kNV; k++) x.d[k] = wrt ? base[(int64_t)(q * (kNV + 1) + 1 + k) * nc + c] : 0.0;
  return x;
}

__device__ __forceinline__ double cell_depth(const trs_thermal_params &P, const Geom &g, int64_t c) {
  const int64_t z = c / ((int64_t)g.nx * g.ny);
  return P.depth_top + ((double)z + 0.5) * P.dz;
}

// ------------------------------------------------------------------ kernels
// Per cell: properties (kept for the neighbours), the accumulation terms
// (N(u) - N(u_old)) / dt with their derivatives and the gas constraint, into
// the residual and the diagonal block.
__global__ void __launch_bounds__(kThreads) k_thermal_cells(Geom g, trs_thermal_params P, ThermalTables tb,
                                                            const double *__restrict__ u,
                                                            const double *__restrict__ u_old,
                                                            const uint8_t *__restrict__ gas, double *props,
                                                            double *ell, double *R) {
  pdl_enter();
  const int64_t c = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  if (c >= g.nc) return;
  const int64_t nc = g.nc;
  const double V = P.dx * P.dy * P.dz;
  const D4 p = var(u[c * kNV + 0], 0), Sw = var(u[c * kNV + 1], 1), Sg = var(u[c * kNV + 2], 2),
           T = var(u[c * kNV + 3], 3);
  CellProps<D4> o;
  cell_props(P, tb, p, Sw, Sg, T, o);
#pragma unroll
  for (int a = 0; a < 3; a++) {
    store_d4(props, nc, c, a, o.lam[a]);
    store_d4(props, nc, c, 3 + a, o.H[a]);
    store_d4(props, nc, c, 6 + a, o.gam[a]);
  }
  store_d4(props, nc, c, 9, o.KT);
  D4 N[3];
  amounts(o, Sw, Sg, V, N);
  N[2] = energy_amount(P, o, p, Sw, Sg, T, V);
  // the old time level: values only
  double No[3];
  {
    const double po = u_old[c * kNV + 0], Swo = u_old[c * kNV + 1], Sgo = u_old[c * kNV + 2],
                 To = u_old[c * kNV + 3];
    CellProps<double> oo;
    cell_props(P, tb, po, Swo, Sgo, To, oo);
    amounts(oo, Swo, Sgo, V, No);
    No[2] = energy_amount(P, oo, po, Swo, Sgo, To, V);
  }
  const double idt = 1.0 / P.dt;
  double blk[kNV * kNV];
#pragma unroll
  for (int e = 0; e < 3; e++) {
    R[c * kNV + e] = (N[e].v - No[e]) * idt;
#pragma unroll
    for (int k = 0; k < kNV; k++) blk[e * kNV + k] = N[e].d[k] * idt;
  }
  const D4 g3 = gas[c] ? o.Kstar - 1.0 : Sg;
  R[c * kNV + 3] = g3.v;
#pragma unroll
  for (int k = 0; k < kNV; k++) blk[3 * kNV + k] = g3.d[k];
#pragma unroll
  for (int e = 0; e < kNV * kNV; e++) ell[((int64_t)kSelf * kNV * kNV + e) * nc + c] = blk[e];
}

// A cell's unknown k as a dual number (its derivative carried) or as a value.
template <class N>
__device__ __forceinline__ N unknown(double a, int k);
template <>
__device__ __forceinline__ D4 unknown<D4>(double a, int k) { return var(a, k); }
template <>
__device__ __forceinline__ double unknown<double>(double a, int) { return a; }
// A stored property with its derivatives (D4) or its value only (double).
template <class N>
__device__ __forceinline__ N prop(const double *base, int64_t nc, int64_t c, int q);
template <>
__device__ __forceinline__ D4 prop<D4>(const double *base, int64_t nc, int64_t c, int q) {
  return load_d4(base, nc, c, q, true);
}
template <>
__device__ __forceinline__ double prop<double>(const double *base, int64_t nc, int64_t c, int q) {
  return base[(int64_t)(q * (kNV + 1)) * nc + c];
}

// Water, oil and energy out of cell c through one face to cell j, with the
// derivatives with respect to c's unknowns (WC) or j's (!WC); the other
// cell's quantities enter as plain values.
template <bool WC>
__device__ void face_flux(const double *props, int64_t nc, int64_t c, int64_t j, const double *u, double Tgeo,
                          double al, double zc, double zj, D4 (&F)[3], bool *tie = nullptr) {
  using NC = typename std::conditional<WC, D4, double>::type;
  using NJ = typename std::conditional<WC, double, D4>::type;
  const NC pc = unknown<NC>(u[c * kNV], 0), Swc = unknown<NC>(u[c * kNV + 1], 1),
           Sgc = unknown<NC>(u[c * kNV + 2], 2), Tc = unknown<NC>(u[c * kNV + 3], 3);
  const NJ pj = unknown<NJ>(u[j * kNV], 0), Swj = unknown<NJ>(u[j * kNV + 1], 1),
           Sgj = unknown<NJ>(u[j * kNV + 2], 2), Tj = unknown<NJ>(u[j * kNV + 3], 3);
  const NC Sc[3] = {Swc, 1.0 - Swc - Sgc, Sgc};
  const NJ Sj[3] = {Swj, 1.0 - Swj - Sgj, Sgj};
  F[0] = F[1] = F[2] = cst(0.0);
#pragma unroll
  for (int a = 0; a < 3; a++) {
    const NC gc = prop<NC>(props, nc, c, 6 + a);
    const NJ gj = prop<NJ>(props, nc, j, 6 + a);
    const D4 ssum = dual(Sc[a] + Sj[a]);
    const D4 gbar = ssum.v > 0.0 ? (Sc[a] * gc + Sj[a] * gj) / ssum : 0.5 * (gc + gj);
    const D4 dphi = (pc - pj) - gbar * (zc - zj);
    if (tie && dphi.v == 0.0) *tie = true;
    D4 f, fH;
    if (dphi.v >= 0.0) {   // c upstream
      const NC lam = prop<NC>(props, nc, c, a), H = prop<NC>(props, nc, c, 3 + a);
      f = (Tgeo * lam) * dphi;
      fH = H * f;
    } else {
      const NJ lam = prop<NJ>(props, nc, j, a), H = prop<NJ>(props, nc, j, 3 + a);
      f = (Tgeo * lam) * dphi;
      fH = H * f;
    }
    if (a == 1) F[1] = F[1] + f;
    else F[0] = F[0] + f;
    F[2] = F[2] + fH;
  }
  const NC kc = prop<NC>(props, nc, c, 9);
  const NJ kj = prop<NJ>(props, nc, j, 9);
  const D4 ks = dual(kc + kj);
  const D4 kt = ks.v > 0.0 ? (2.0 * kc * kj) / ks : cst(0.0);
  F[2] = F[2] + al * kt * (Tc - Tj);
}

// Geometric factors of the face between c and j along axis (0 x, 1 y, 2 z):
// T_geo = c_u k_h A / L with the harmonic mean of the permeabilities (vertical
// ones times kv/kh), and A / L for conduction.
__device__ __forceinline__ double face_tgeo(const trs_thermal_params &P, const double *perm, int64_t c, int64_t j,
                                           int axis, double &al) {
  al = axis == 0 ? P.dy * P.dz / P.dx : (axis == 1 ? P.dx * P.dz / P.dy : P.dx * P.dy / P.dz);
  const double ki = perm[c], kj = perm[j];
  double kh = (ki + kj > 0.0) ? 2.0 * ki * kj / (ki + kj) : 0.0;
  if (axis == 2) kh = kh * P.kvkh;
  return kUnit * kh * al;
}

// Face terms kept for the row kernel, per cell c and positive axis (the face
// to c + e_x, c + e_y, c + e_z), structure of arrays: the flux F out of c (3),
// dF/du_c (12), dF/du_j (12), and 1.0 when a phase potential difference is
// exactly zero (then each side takes itself as upstream and the two rows'
// fluxes are not negatives of each other).
constexpr int kFaceDoubles = 28;

// Per face, once: the flux out of c and its derivatives with respect to both
// cells.  Row j sees the flux -F, so the off-diagonal blocks of both rows are
// written here: row c's column j is dF/du_j, row j's column c is -dF/du_c.
// Thread (c, axis): blockIdx.y is the axis.
__global__ void __launch_bounds__(kThreads) k_thermal_faces(Geom g, trs_thermal_params P,
                                                            const uint8_t *__restrict__ emask,
                                                            const double *__restrict__ perm,
                                                            const double *__restrict__ u, const double *props,
                                                            double *__restrict__ faces, double *ell) {
  pdl_enter();
  constexpr int BB = kNV * kNV;
  const int64_t c = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  if (c >= g.nc) return;
  const int axis = blockIdx.y;
  const int s = 4 + axis;                 // slots 4, 5, 6: x+, y+, z+
  if (!((emask[c] >> s) & 1u)) return;
  const int so = kSlots - 1 - s;          // the same face seen from j
  const int64_t nc = g.nc, j = c + g.off[s];
  double al;
  const double Tgeo = face_tgeo(P, perm, c, j, axis, al);
  D4 Fc[3], Fj[3];
  bool tie = false;
  face_flux<true>(props, nc, c, j, u, Tgeo, al, cell_depth(P, g, c), cell_depth(P, g, j), Fc, &tie);
  face_flux<false>(props, nc, c, j, u, Tgeo, al, cell_depth(P, g, c), cell_depth(P, g, j), Fj);
  double *fb = faces + (int64_t)axis * kFaceDoubles * nc + c;
#pragma unroll
  for (int e = 0; e < 3; e++) {
    fb[(int64_t)e * nc] = Fc[e].v;
#pragma unroll
    for (int k = 0; k < kNV; k++) {
      fb[(int64_t)(3 + e * kNV + k) * nc] = Fc[e].d[k];
      fb[(int64_t)(15 + e * kNV + k) * nc] = Fj[e].d[k];
      ell[((int64_t)s * BB + e * kNV + k) * nc + c] = Fj[e].d[k];
      ell[((int64_t)so * BB + e * kNV + k) * nc + j] = -Fc[e].d[k];
    }
  }
  fb[(int64_t)27 * nc] = tie ? 1.0 : 0.0;
#pragma unroll
  for (int k = 0; k < kNV; k++) {
    ell[((int64_t)s * BB + 3 * kNV + k) * nc + c] = 0.0;
    ell[((int64_t)so * BB + 3 * kNV + k) * nc + j] = 0.0;
  }
}

// Per cell row: the six faces' terms (kept by k_thermal_faces), added to the
// accumulation part k_thermal_cells left in the residual and the diagonal
// block.
__global__ void __launch_bounds__(kThreads) k_thermal_rows(Geom g, const uint8_t *__restrict__ emask,
                                                           const double *__restrict__ faces, double *ell, double *R) {
  pdl_enter();
  constexpr int BB = kNV * kNV;
  const int64_t c = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  if (c >= g.nc) return;
  const int64_t nc = g.nc;
  double dg[BB], rc[kNV];
#pragma unroll
  for (int e = 0; e < BB; e++) dg[e] = ell[((int64_t)kSelf * BB + e) * nc + c];
#pragma unroll
  for (int e = 0; e < kNV; e++) rc[e] = R[c * kNV + e];
  const unsigned m = emask[c];
  for (int d = 0; d < 6; d++) {
    const int s = d < 3 ? d : d + 1;
    if (!((m >> s) & 1u)) continue;
    const int64_t j = c + g.off[s];
    if (d >= 3) {
      // c's own face: F out of c and dF/du_c
      const double *fb = faces + (int64_t)(d - 3) * kFaceDoubles * nc + c;
#pragma unroll
      for (int e = 0; e < 3; e++) {
        rc[e] = rc[e] + fb[(int64_t)e * nc];
#pragma unroll
        for (int k = 0; k < kNV; k++) dg[e * kNV + k] = dg[e * kNV + k] + fb[(int64_t)(3 + e * kNV + k) * nc];
      }
      continue;
    }
    // the face kept by j (d = 0, 1, 2: z-, y-, x-, axis 2 - d): the flux out of
    // c is -F and its derivative with respect to c is -dF/du_j; a face with a
    // tie is left to k_thermal_ties
    const double *fb = faces + (int64_t)(2 - d) * kFaceDoubles * nc + j;
    if (fb[(int64_t)27 * nc] != 0.0) continue;
#pragma unroll
    for (int e = 0; e < 3; e++) {
      rc[e] = rc[e] - fb[(int64_t)e * nc];
#pragma unroll
      for (int k = 0; k < kNV; k++) dg[e * kNV + k] = dg[e * kNV + k] - fb[(int64_t)(15 + e * kNV + k) * nc];
    }
  }
#pragma unroll
  for (int e = 0; e < BB; e++) ell[((int64_t)kSelf * BB + e) * nc + c] = dg[e];
#pragma unroll
  for (int e = 0; e < kNV; e++) R[c * kNV + e] = rc[e];
}

// Per perforated cell: the perforations' terms, Q > 0 flowing into the cell,
// added to the residual and the diagonal block; the well-column tail blocks
// are written.
__global__ void __launch_bounds__(kThreads) k_thermal_perfs(
    Geom g, trs_thermal_params P, const double *__restrict__ u, const double *props,
    const int64_t *__restrict__ cperf_ptr, const int64_t *__restrict__ cperf_idx, const int64_t *__restrict__ perf_cw,
    const int32_t *__restrict__ perf_well, const double *__restrict__ wi, const int32_t *__restrict__ well_type,
    double *ell, double *tval, double *R) {
  pdl_enter();
  constexpr int BB = kNV * kNV;
  const int64_t c = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  if (c >= g.nc || cperf_ptr[c] == cperf_ptr[c + 1]) return;
  const int64_t nc = g.nc;
  double dg[BB], rc[kNV];
#pragma unroll
  for (int e = 0; e < BB; e++) dg[e] = ell[((int64_t)kSelf * BB + e) * nc + c];
#pragma unroll
  for (int e = 0; e < kNV; e++) rc[e] = R[c * kNV + e];
  {
    const double pcv = u[c * kNV];
    const int64_t wrow0 = g.nc;
    for (int64_t t = cperf_ptr[c]; t < cperf_ptr[c + 1]; t++) {
      const int64_t mm = cperf_idx[t];
      const int w = perf_well[mm];
      const double pb = u[(wrow0 + w) * kNV];
      double *blk = tval + perf_cw[mm] * BB;
#pragma unroll
      for (int e = 0; e < BB; e++) blk[e] = 0.0;
      if (well_type[w] == 0) {   // injector, unweighted mobility: Q = WI_u (p_b - p) of steam
        const double Q = wi[mm] * (pb - pcv);
        rc[0] -= Q;
        rc[2] -= Q * P.h_inj;
        dg[0 * kNV] += wi[mm];
        dg[2 * kNV] += wi[mm] * P.h_inj;
        blk[0 * kNV] = -wi[mm];
        blk[2 * kNV] = -wi[mm] * P.h_inj;
      } else {                   // producer, cell mobilities: Q_a = WI c_u lam_a (p_b - p)
#pragma unroll
        for (int a = 0; a < 3; a++) {
          const D4 lam = load_d4(props, nc, c, a, true), H = load_d4(props, nc, c, 3 + a, true);
          const D4 Q = (wi[mm] * kUnit) * lam * (pb - var(pcv, 0));
          const D4 QH = H * Q;
          const int eq = a == 1 ? 1 : 0;
          const double dQdpb = wi[mm] * kUnit * lam.v;
          rc[eq] -= Q.v;
          rc[2] -= QH.v;
#pragma unroll
          for (int k = 0; k < kNV; k++) {
            dg[eq * kNV + k] -= Q.d[k];
            dg[2 * kNV + k] -= QH.d[k];
          }
          blk[eq * kNV] -= dQdpb;
          blk[2 * kNV] -= H.v * dQdpb;
        }
      }
    }
  }
#pragma unroll
  for (int e = 0; e < BB; e++) ell[((int64_t)kSelf * BB + e) * nc + c] = dg[e];
#pragma unroll
  for (int e = 0; e < kNV; e++) R[c * kNV + e] = rc[e];
}

// The faces with a tie seen from the cell that does not keep them (its z-,
// y- or x- face): that side takes itself as upstream, so its flux and
// derivatives come from its own pair of one-sided passes, added to what
// k_thermal_rows left in the residual and the diagonal block.
__global__ void __launch_bounds__(kThreads) k_thermal_ties(Geom g, trs_thermal_params P,
                                                           const uint8_t *__restrict__ emask,
                                                           const double *__restrict__ perm,
                                                           const double *__restrict__ u, const double *props,
                                                           const double *__restrict__ faces, double *ell, double *R) {
  pdl_enter();
  constexpr int BB = kNV * kNV;
  const int64_t c = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  if (c >= g.nc) return;
  const int64_t nc = g.nc;
  const unsigned m = emask[c];
  for (int d = 0; d < 3; d++) {
    if (!((m >> d) & 1u)) continue;
    const int64_t j = c + g.off[d];
    const int axis = 2 - d;
    if (faces[((int64_t)axis * kFaceDoubles + 27) * nc + j] == 0.0) continue;
    double al;
    const double Tgeo = face_tgeo(P, perm, c, j, axis, al);
    D4 Fc[3], Fj[3];
    face_flux<true>(props, nc, c, j, u, Tgeo, al, cell_depth(P, g, c), cell_depth(P, g, j), Fc);
    face_flux<false>(props, nc, c, j, u, Tgeo, al, cell_depth(P, g, c), cell_depth(P, g, j), Fj);
#pragma unroll
    for (int e = 0; e < 3; e++) {
      R[c * kNV + e] += Fc[e].v;
#pragma unroll
      for (int k = 0; k < kNV; k++) {
        ell[((int64_t)kSelf * BB + e * kNV + k) * nc + c] += Fc[e].d[k];
        ell[((int64_t)d * BB + e * kNV + k) * nc + c] = Fj[e].d[k];
      }
    }
  }
}

// Per well: injectors sum_m WI_u (p_b - p_m) - q_target; producers
// p_b - p_target; the padding entries of the well block are an identity with
// residual u (zero for a padded state).
__global__ void __launch_bounds__(kThreads) k_thermal_wells(int nw, int64_t nc, const double *__restrict__ u,
                                                            const int64_t *__restrict__ wperf_ptr,
                                                            const int64_t *__restrict__ wperf_idx,
                                                            const int32_t *__restrict__ perf_cell,
                                                            const int64_t *__restrict__ perf_wc,
                                                            const int64_t *__restrict__ wdiag,
                                                            const double *__restrict__ wi,
                                                            const int32_t *__restrict__ well_type,
                                                            const double *__restrict__ well_target, double *tval,
                                                            double *R) {
  pdl_enter();
  constexpr int BB = kNV * kNV;
  const int w = blockIdx.x * kThreads + threadIdx.x;
  if (w >= nw) return;
  const int64_t row = nc + w;
  const double pb = u[row * kNV];
  double *dgb = tval + wdiag[w] * BB;
#pragma unroll
  for (int e = 0; e < BB; e++) dgb[e] = 0.0;
#pragma unroll
  for (int s = 1; s < kNV; s++) {
    dgb[s * kNV + s] = 1.0;
    R[row * kNV + s] = u[row * kNV + s];
  }
  if (well_type[w] == 0) {
    double q = 0.0, sum = 0.0;
    for (int64_t t = wperf_ptr[w]; t < wperf_ptr[w + 1]; t++) {
      const int64_t mm = wperf_idx[t];
      const double pcv = u[(int64_t)perf_cell[mm] * kNV];
      q = q + wi[mm] * (pb - pcv);
      sum = sum + wi[mm];
      double *blk = tval + perf_wc[mm] * BB;
#pragma unroll
      for (int e = 0; e < BB; e++) blk[e] = 0.0;
      blk[0] = -wi[mm];
    }
    dgb[0] = sum;
    R[row * kNV] = q - well_target[w];
  } else {
    for (int64_t t = wperf_ptr[w]; t < wperf_ptr[w + 1]; t++) {
      double *blk = tval + perf_wc[wperf_idx[t]] * BB;
#pragma unroll
      for (int e = 0; e < BB; e++) blk[e] = 0.0;
    }
    dgb[0] = 1.0;
    R[row * kNV] = pb - well_target[w];
  }
}

}  // namespace

void launch_thermal(trs_bsr *A, const trs_thermal_params &P, const ThermalTables &tb, const double *perm,
                    const double *u, const double *u_old, const uint8_t *gas, const double *wi,
                    const int32_t *well_type, const double *well_target, double *R, cudaStream_t s) {
  const int64_t nc = A->g.nc;
  const int64_t scratch = (int64_t)(kPropDoubles + 3 * kFaceDoubles) * nc;
  if ((int64_t)A->thermal_props.n < scratch) A->thermal_props.alloc((size_t)scratch);
  double *faces = A->thermal_props.p + (int64_t)kPropDoubles * nc;
  if (nc) {
    launch_pdl(k_thermal_cells, grid_of(nc), kThreads, 0, s, A->g, P, tb, u, u_old, gas, A->thermal_props.p,
               A->ell.p, R);
    TRS_LAUNCHED();
    launch_pdl(k_thermal_faces, dim3(grid_of(nc), 3), dim3(kThreads), 0, s, A->g, P, (const uint8_t *)A->emask.p,
               perm, u, (const double *)A->thermal_props.p, faces, A->ell.p);
    TRS_LAUNCHED();
    launch_pdl(k_thermal_rows, grid_of(nc), kThreads, 0, s, A->g, (const uint8_t *)A->emask.p, (const double *)faces,
               A->ell.p, R);
    TRS_LAUNCHED();
    if (A->n_perf) {
      launch_pdl(k_thermal_perfs, grid_of(nc), kThreads, 0, s, A->g, P, u, (const double *)A->thermal_props.p,
                 (const int64_t *)A->cperf_ptr.p, (const int64_t *)A->cperf_idx.p, (const int64_t *)A->perf_cw.p,
                 (const int32_t *)A->perf_well.p, wi, well_type, A->ell.p, A->tval.p, R);
      TRS_LAUNCHED();
    }
    launch_pdl(k_thermal_ties, grid_of(nc), kThreads, 0, s, A->g, P, (const uint8_t *)A->emask.p, perm, u,
               (const double *)A->thermal_props.p, (const double *)faces, A->ell.p, R);
    TRS_LAUNCHED();
  }
  if (A->n_wells) {
    launch_pdl(k_thermal_wells, grid_of(A->n_wells), kThreads, 0, s, A->n_wells, nc, u,
               (const int64_t *)A->wperf_ptr.p, (const int64_t *)A->wperf_idx.p, (const int32_t *)A->perf_cell.p,
               (const int64_t *)A->perf_wc.p, (const int64_t *)A->wdiag.p, wi, well_type, well_target, A->tval.p,
               R);
    TRS_LAUNCHED();
  }
}

}  // namespace trs

extern "C" trs_status trs_thermal_assemble(trs_bsr *A, const trs_thermal_params *prm, const double *swt,
                                           int32_t nswt, const double *slt, int32_t nslt, const double *perm,
                                           const double *u, const double *u_old, const uint8_t *gas,
                                           const double *wi, const int32_t *well_type,
                                           const double *well_target, double *residual, void *stream) {
  using namespace trs;
  return guarded([&] {
    TRS_REQUIRE(A && prm && swt && slt && perm && u && u_old && gas && residual, TRS_ERR_INVALID,
                "NULL argument");
    TRS_REQUIRE(A->synthetic, TRS_ERR_INVALID, "matrix was not made by trs_bsr_create_synthetic");
    TRS_REQUIRE(A->b == 4, TRS_ERR_UNSUPPORTED, "the thermal model has 4 unknowns per cell (b = 4)");
    TRS_REQUIRE(A->n_perf == 0 || (wi && well_type && well_target), TRS_ERR_INVALID, "NULL well array");
    TRS_REQUIRE(A->n_perf == 0 || (A->perf_cell.p && A->perf_well.p && A->cperf_ptr.p && A->wperf_ptr.p),
                TRS_ERR_INVALID, "matrix holds no perforation lists");
    TRS_REQUIRE(nswt >= 2 && nswt <= kThermalTableMax && nslt >= 2 && nslt <= kThermalTableMax, TRS_ERR_INVALID,
                "relative-permeability tables need 2..32 rows");
    TRS_REQUIRE(prm->dt > 0.0 && prm->dx > 0.0 && prm->dy > 0.0 && prm->dz > 0.0, TRS_ERR_INVALID,
                "dt and the cell sizes must be positive");
    ThermalTables tb{};
    tb.nswt = nswt;
    tb.nslt = nslt;
    for (int r = 0; r < 3 * nswt; r++) tb.swt[r] = swt[r];
    for (int r = 0; r < 3 * nslt; r++) tb.slt[r] = slt[r];
    for (int i = 0; i + 1 < nswt; i++)
      for (int c = 1; c <= 2; c++)
        tb.swt_slope[2 * i + c - 1] = (swt[3 * (i + 1) + c] - swt[3 * i + c]) / (swt[3 * (i + 1)] - swt[3 * i]);
    for (int i = 0; i + 1 < nslt; i++)
      for (int c = 1; c <= 2; c++)
        tb.slt_slope[2 * i + c - 1] = (slt[3 * (i + 1) + c] - slt[3 * i + c]) / (slt[3 * (i + 1)] - slt[3 * i]);
    for (int r = 1; r < nswt; r++)
      TRS_REQUIRE(swt[3 * r] > swt[3 * (r - 1)], TRS_ERR_INVALID, "table saturations must increase");
    for (int r = 1; r < nslt; r++)
      TRS_REQUIRE(slt[3 * r] > slt[3 * (r - 1)], TRS_ERR_INVALID, "table saturations must increase");
    TRS_REQUIRE(swt[2] > 0.0, TRS_ERR_INVALID, "k_row at connate water must be positive");
    launch_thermal(A, *prm, tb, perm, u, u_old, gas, wi, well_type, well_target, residual, (cudaStream_t)stream);
  });
}
