"""ctypes wrapper of the plain FP64 CPU oracle (trs_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by
the CPU-baseline leg of the benchmark.  The product path never imports it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liboracle.so")
SOURCES = [os.path.join(HERE, "trs_oracle.c"), os.path.join(HERE, "trs_thermal.c")]

i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
i8p = np.ctypeslib.ndpointer(np.int8, flags="C_CONTIGUOUS")
f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (plain C, no FMA contraction)."""
    newest = max(os.path.getmtime(s) for s in SOURCES + [os.path.join(HERE, "trs_oracle.h")])
    if not force and os.path.exists(LIB_PATH) and os.path.getmtime(LIB_PATH) >= newest:
        return LIB_PATH
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-Wall", "-o", tmp] + SOURCES + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


class _Stats(C.Structure):
    _fields_ = [("iters", C.c_int), ("restarts", C.c_int), ("converged", C.c_int),
                ("est_relres", C.c_double), ("true_relres", C.c_double)]


class _ThermalParams(C.Structure):
    _fields_ = [(f, C.c_double) for f in (
        "dx", "dy", "dz", "depth_top", "dt", "kvkh", "gravity",
        "phi_ref", "cpor", "ctpor", "p_ref", "T_ref", "cp1_r", "cp2_r",
        "kt_w", "kt_o", "kt_g", "kt_r",
        "rho_w_ref", "cp_w", "ct1_w", "ct2_w", "cpt_w", "mw_w", "avisc_w", "bvisc_w",
        "kv1", "kv2", "kv3", "kv4", "kv5", "per_eps", "tc_w", "pc_w")] + [
        ("cpg", C.c_double * 5)] + [(f, C.c_double) for f in (
            "hvr", "ev", "rho_o_ref", "cp_o", "ct1_o", "ct2_o", "cpt_o", "mw_o", "avisc_o", "bvisc_o",
            "cpl1_o", "mug_a", "mug_b", "h_inj", "R_gas")]


def thermal_params(d: dict) -> _ThermalParams:
    """The parameter struct of trs_thermal.c from a dict of named values."""
    P = _ThermalParams()
    for name, _ in _ThermalParams._fields_:
        if name == "cpg":
            P.cpg = (C.c_double * 5)(*[d[f"cpg{k}"] for k in range(1, 6)])
        else:
            setattr(P, name, float(d[name]))
    return P


class _CprOpts(C.Structure):
    _fields_ = [("theta", C.c_double), ("coarse_max", C.c_int), ("max_levels", C.c_int),
                ("cheb_degree", C.c_int), ("seed", C.c_uint32), ("stages", C.c_int),
                ("decoupling", C.c_int), ("ilu_fill", C.c_int), ("grid", C.c_int * 3)]


#: CPR stage orderings and decoupling methods (Sec. "Preconditioners",
#: Sec. "Decoupling Methods")
STAGES = {"fpf": 0, "fp": 1, "pf": 2}
DECOUPLINGS = {"abf": 0, "none": 1, "frs": 2, "frs+abf": 3}


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        L.orc_assembly_nnzb.restype = C.c_int64
        L.orc_assembly_nnzb.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int64, i32p, i32p]
        L.orc_assemble.restype = C.c_int
        L.orc_assemble.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, f64p, C.c_double, C.c_double,
                                   f64p, f64p, C.c_int, C.c_int64, i32p, i32p, f64p, f64p,
                                   i64p, i32p, f64p]
        for name in ("orc_bsr_spmv", "orc_bsr_spmv_t"):
            f = getattr(L, name)
            f.restype = None
            f.argtypes = [C.c_int64, C.c_int, i64p, i32p, f64p, f64p, f64p, C.c_double, C.c_double]
        L.orc_bsr_transpose.restype = C.c_int
        L.orc_bsr_transpose.argtypes = [C.c_int64, C.c_int, i64p, i32p, f64p, i64p, i32p, f64p]
        L.orc_pattern_symmetric.restype = C.c_int
        L.orc_pattern_symmetric.argtypes = [C.c_int64, i64p, i32p]
        L.orc_gj_inverse.restype = C.c_int
        L.orc_gj_inverse.argtypes = [C.c_int, f64p, f64p]
        L.orc_decouple_mode.restype = C.c_int
        L.orc_decouple_mode.argtypes = [C.c_int64, C.c_int, i64p, i32p, f64p, C.c_int, f64p, f64p]
        L.orc_decouple.restype = C.c_int
        L.orc_decouple.argtypes = [C.c_int64, C.c_int, i64p, i32p, f64p, f64p, f64p]
        L.orc_pressure_matrix.restype = None
        L.orc_pressure_matrix.argtypes = [C.c_int64, C.c_int, i64p, i32p, f64p, f64p]
        L.orc_strength.restype = C.c_int64
        L.orc_strength.argtypes = [C.c_int64, i64p, i32p, f64p, C.c_double, i64p, i32p]
        L.orc_mis2.restype = C.c_int
        L.orc_mis2.argtypes = [C.c_int64, i64p, i32p, C.c_uint32, i8p]
        L.orc_aggregate.restype = C.c_int64
        L.orc_aggregate.argtypes = [C.c_int64, i64p, i32p, f64p, i64p, i32p, i8p, i32p]
        L.orc_galerkin_nnz.restype = C.c_int64
        L.orc_galerkin_nnz.argtypes = [C.c_int64, i64p, i32p, i32p, C.c_int64]
        L.orc_galerkin.restype = None
        L.orc_galerkin.argtypes = [C.c_int64, i64p, i32p, f64p, i32p, C.c_int64, i64p, i32p, f64p]
        L.orc_gershgorin.restype = C.c_double
        L.orc_gershgorin.argtypes = [C.c_int64, i64p, i32p, f64p]
        L.orc_chebyshev.restype = None
        L.orc_chebyshev.argtypes = [C.c_int64, i64p, i32p, f64p, C.c_double, C.c_int, f64p, f64p,
                                    C.c_int]
        L.orc_amg_setup.restype = C.c_void_p
        L.orc_amg_setup.argtypes = [C.c_int64, i64p, i32p, f64p, C.c_double, C.c_int, C.c_int,
                                    C.c_int, C.c_uint32, C.POINTER(C.c_int)]
        L.orc_amg_levels.restype = C.c_int
        L.orc_amg_levels.argtypes = [C.c_void_p]
        L.orc_amg_level_n.restype = C.c_int64
        L.orc_amg_level_n.argtypes = [C.c_void_p, C.c_int]
        L.orc_amg_level_nnz.restype = C.c_int64
        L.orc_amg_level_nnz.argtypes = [C.c_void_p, C.c_int]
        L.orc_amg_level_copy.restype = None
        L.orc_amg_level_copy.argtypes = [C.c_void_p, C.c_int, i64p, i32p, f64p]
        L.orc_amg_level_agg.restype = None
        L.orc_amg_level_agg.argtypes = [C.c_void_p, C.c_int, i32p]
        L.orc_amg_level_lambda.restype = C.c_double
        L.orc_amg_level_lambda.argtypes = [C.c_void_p, C.c_int]
        L.orc_amg_vcycle.restype = None
        L.orc_amg_vcycle.argtypes = [C.c_void_p, f64p, f64p]
        L.orc_amg_free.restype = None
        L.orc_amg_free.argtypes = [C.c_void_p]
        L.orc_dense_lu.restype = C.c_int
        L.orc_dense_lu.argtypes = [C.c_int64, f64p, i32p]
        L.orc_dense_lu_solve.restype = None
        L.orc_dense_lu_solve.argtypes = [C.c_int64, f64p, i32p, f64p]
        L.orc_colour_jp.restype = C.c_int
        L.orc_colour_jp.argtypes = [C.c_int64, i64p, i32p, C.c_uint32, i32p]
        L.orc_bilu0_setup.restype = C.c_void_p
        L.orc_bilu0_setup.argtypes = [C.c_int64, C.c_int, i64p, i32p, f64p, i32p, C.POINTER(C.c_int)]
        L.orc_bilu0_solve.restype = None
        L.orc_bilu0_solve.argtypes = [C.c_void_p, f64p, f64p]
        L.orc_bilu0_factors.restype = None
        L.orc_bilu0_factors.argtypes = [C.c_void_p, f64p]
        L.orc_bilu0_free.restype = None
        L.orc_bilu0_free.argtypes = [C.c_void_p]
        L.orc_colour_geo.restype = C.c_int
        L.orc_colour_geo.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int64, i64p, i32p, i32p]
        L.orc_biluk_setup.restype = C.c_void_p
        L.orc_biluk_setup.argtypes = [C.c_int64, C.c_int, i64p, i32p, f64p, i32p, C.c_int,
                                      C.POINTER(C.c_int)]
        L.orc_bilu_nnz.restype = C.c_int64
        L.orc_bilu_nnz.argtypes = [C.c_void_p]
        L.orc_bilu_pattern.restype = None
        L.orc_bilu_pattern.argtypes = [C.c_void_p, i64p, i32p]
        L.orc_bilu_colours_independent.restype = C.c_int
        L.orc_bilu_colours_independent.argtypes = [C.c_void_p, i32p]
        L.orc_cpr_ilu.restype = C.c_void_p
        L.orc_cpr_ilu.argtypes = [C.c_void_p]
        L.orc_cpr_setup.restype = C.c_void_p
        L.orc_cpr_setup.argtypes = [C.c_int64, C.c_int, i64p, i32p, f64p, C.POINTER(_CprOpts),
                                    C.POINTER(C.c_int)]
        L.orc_cpr_apply.restype = None
        L.orc_cpr_apply.argtypes = [C.c_void_p, f64p, f64p]
        L.orc_cpr_info.restype = C.c_int
        L.orc_cpr_info.argtypes = [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.orc_cpr_amg.restype = C.c_void_p
        L.orc_cpr_amg.argtypes = [C.c_void_p]
        L.orc_cpr_colours.restype = None
        L.orc_cpr_colours.argtypes = [C.c_void_p, i32p]
        L.orc_cpr_decoupled.restype = None
        L.orc_cpr_decoupled.argtypes = [C.c_void_p, f64p, f64p]
        L.orc_cpr_ilu_factors.restype = None
        L.orc_cpr_ilu_factors.argtypes = [C.c_void_p, f64p]
        L.orc_cpr_free.restype = None
        L.orc_cpr_free.argtypes = [C.c_void_p]
        L.orc_fgmres.restype = C.c_int
        L.orc_fgmres.argtypes = [C.c_int64, C.c_int, i64p, i32p, f64p, C.c_void_p, f64p, f64p,
                                 C.c_double, C.c_int, C.c_int, C.POINTER(_Stats), f64p, C.c_int]
        L.orc_bicgstab.restype = C.c_int
        L.orc_bicgstab.argtypes = [C.c_int64, C.c_int, i64p, i32p, f64p, C.c_void_p, f64p, f64p,
                                   C.c_double, C.c_int, C.POINTER(_Stats), f64p, C.c_int]
        L.orc_outer_product.restype = None
        L.orc_outer_product.argtypes = [C.c_int64, C.c_int, i64p, i32p, f64p, f64p, f64p]
        L.orc_chain_theta.restype = C.c_int
        L.orc_chain_theta.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, f64p, C.c_double,
                                      C.c_double, f64p, i64p, i32p, f64p, f64p]
        u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")
        tp = C.POINTER(_ThermalParams)
        common = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int64, tp, f64p, C.c_int, f64p, C.c_int, f64p,
                  i32p, i32p, f64p, i32p, f64p, u8p, f64p, f64p]
        rowsp = C.c_void_p
        L.orc_thermal_residual.restype = C.c_int
        L.orc_thermal_residual.argtypes = common + [C.c_int64, rowsp, f64p]
        L.orc_thermal_jacobian.restype = C.c_int
        L.orc_thermal_jacobian.argtypes = common + [C.c_int64, rowsp, i64p, i32p, f64p]
        L.orc_thermal_props.restype = None
        L.orc_thermal_props.argtypes = [tp, f64p, C.c_int, f64p, C.c_int, f64p, f64p]
        L.orc_rk_z.restype = C.c_double
        L.orc_rk_z.argtypes = [C.c_double, C.c_double]
        L.orc_thermal_totals.restype = None
        L.orc_thermal_totals.argtypes = [C.c_int, C.c_int, C.c_int, tp, f64p, C.c_int, f64p, C.c_int, f64p,
                                         f64p]
        L.orc_thermal_well_sources.restype = None
        L.orc_thermal_well_sources.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int64, tp, f64p,
                                               C.c_int, f64p, C.c_int, i32p, i32p, f64p, i32p, f64p, f64p]
        _lib = L
    return _lib


class OracleError(RuntimeError):
    pass


def _check(st, what):
    if st < 0:
        raise OracleError(f"{what} failed with status {st}")
    return st


@dataclass
class BSR:
    """General block CSR: rp int64[n+1], col int32[nnzb], val float64[nnzb, b, b]."""
    n: int
    b: int
    rp: np.ndarray
    col: np.ndarray
    val: np.ndarray

    @property
    def nnzb(self):
        return int(self.rp[-1])

    def row_of_block(self):
        return np.repeat(np.arange(self.n, dtype=np.int64), np.diff(self.rp))

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.bsr_matrix((self.val.reshape(-1, self.b, self.b), self.col, self.rp),
                             shape=(self.n * self.b, self.n * self.b))

    def to_dense(self):
        return self.to_scipy().toarray()


def assemble(sysm) -> BSR:
    """Synthetic Jacobian of a :class:`SyntheticSystem`."""
    L = lib()
    n_c = sysm.nx * sysm.ny * sysm.nz
    nnzb = L.orc_assembly_nnzb(sysm.nx, sysm.ny, sysm.nz, sysm.n_wells, len(sysm.perf_cell),
                               sysm.perf_well, sysm.perf_cell)
    n = n_c + sysm.n_wells
    b = sysm.b
    rp = np.zeros(n + 1, np.int64)
    col = np.zeros(nnzb, np.int32)
    val = np.zeros(nnzb * b * b, np.float64)
    _check(L.orc_assemble(sysm.nx, sysm.ny, sysm.nz, b, sysm.k, sysm.kvkh, sysm.c_t,
                          sysm.M.reshape(-1), sysm.acc.reshape(-1), sysm.n_wells,
                          len(sysm.perf_cell), sysm.perf_well, sysm.perf_cell, sysm.wi,
                          sysm.lam.reshape(-1), rp, col, val), "assemble")
    return BSR(n, b, rp, col, val.reshape(nnzb, b, b))


def spmv(A: BSR, x, alpha=1.0, beta=0.0, y=None, transpose=False):
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.zeros(A.n * A.b) if y is None else np.array(y, dtype=np.float64)
    f = lib().orc_bsr_spmv_t if transpose else lib().orc_bsr_spmv
    f(A.n, A.b, A.rp, A.col, A.val.reshape(-1), x, y, alpha, beta)
    return y


def transpose(A: BSR) -> BSR:
    rpT = np.zeros_like(A.rp)
    colT = np.zeros_like(A.col)
    valT = np.zeros_like(A.val)
    _check(lib().orc_bsr_transpose(A.n, A.b, A.rp, A.col, A.val.reshape(-1), rpT, colT,
                                   valT.reshape(-1)), "transpose")
    return BSR(A.n, A.b, rpT, colT, valT)


def pattern_symmetric(A: BSR) -> bool:
    return bool(lib().orc_pattern_symmetric(A.n, A.rp, A.col))


def gj_inverse(D):
    D = np.ascontiguousarray(D, dtype=np.float64)
    b = D.shape[0]
    inv = np.zeros(b * b)
    _check(lib().orc_gj_inverse(b, D.reshape(-1), inv), "gj_inverse")
    return inv.reshape(b, b)


def decouple(A: BSR, mode="abf"):
    vt = np.zeros_like(A.val)
    dinv = np.zeros((A.n, A.b, A.b))
    _check(lib().orc_decouple_mode(A.n, A.b, A.rp, A.col, A.val.reshape(-1), DECOUPLINGS[mode],
                                   vt.reshape(-1), dinv.reshape(-1)), "decouple")
    return vt, dinv


def pressure_matrix(A: BSR, vt):
    ap = np.zeros(A.nnzb)
    lib().orc_pressure_matrix(A.n, A.b, A.rp, A.col, np.ascontiguousarray(vt).reshape(-1), ap)
    return ap


def strength(n, rp, col, val, theta):
    srp = np.zeros(n + 1, np.int64)
    scol = np.zeros(max(1, len(col)), np.int32)
    q = lib().orc_strength(n, rp, col, val, theta, srp, scol)
    return srp, scol[:q].copy()


def mis2(n, srp, scol, seed):
    state = np.zeros(n, np.int8)
    scol = np.ascontiguousarray(scol if len(scol) else np.zeros(1, np.int32), dtype=np.int32)
    rounds = lib().orc_mis2(n, srp, scol, seed, state)
    return state, rounds


def aggregate(n, rp, col, val, srp, scol, state):
    agg = np.zeros(n, np.int32)
    scol = np.ascontiguousarray(scol if len(scol) else np.zeros(1, np.int32), dtype=np.int32)
    n_agg = lib().orc_aggregate(n, rp, col, val, srp, scol, state, agg)
    return agg, int(n_agg)


def galerkin(n, rp, col, val, agg, n_agg):
    L = lib()
    nnz = L.orc_galerkin_nnz(n, rp, col, agg, n_agg)
    crp = np.zeros(n_agg + 1, np.int64)
    ccol = np.zeros(max(1, nnz), np.int32)
    cval = np.zeros(max(1, nnz))
    L.orc_galerkin(n, rp, col, val, agg, n_agg, crp, ccol, cval)
    return crp, ccol[:nnz].copy(), cval[:nnz].copy()


def gershgorin(n, rp, col, val):
    return lib().orc_gershgorin(n, rp, col, val)


def chebyshev(n, rp, col, val, lam, degree, r, e=None):
    r = np.ascontiguousarray(r, dtype=np.float64)
    zero = e is None
    e = np.zeros(n) if zero else np.array(e, dtype=np.float64)
    lib().orc_chebyshev(n, rp, col, val, lam, degree, r, e, int(zero))
    return e


def dense_lu_solve(A, rhs):
    A = np.array(A, dtype=np.float64)
    n = A.shape[0]
    piv = np.zeros(n, np.int32)
    _check(lib().orc_dense_lu(n, A.reshape(-1), piv), "dense_lu")
    x = np.array(rhs, dtype=np.float64)
    lib().orc_dense_lu_solve(n, A.reshape(-1), piv, x)
    return x


class AMG:
    def __init__(self, n, rp, col, val, theta=0.08, coarse_max=64, max_levels=12,
                 cheb_degree=2, seed=12345):
        st = C.c_int(0)
        self.h = lib().orc_amg_setup(n, rp, col, np.ascontiguousarray(val, dtype=np.float64),
                                     theta, coarse_max, max_levels, cheb_degree, seed,
                                     C.byref(st))
        if not self.h:
            raise OracleError(f"amg setup failed with status {st.value}")
        self.owned = True

    @classmethod
    def borrowed(cls, h):
        o = cls.__new__(cls)
        o.h = h
        o.owned = False
        return o

    @property
    def n_levels(self):
        return lib().orc_amg_levels(self.h)

    def level(self, l):
        L = lib()
        n = L.orc_amg_level_n(self.h, l)
        nnz = L.orc_amg_level_nnz(self.h, l)
        rp = np.zeros(n + 1, np.int64)
        col = np.zeros(max(1, nnz), np.int32)
        val = np.zeros(max(1, nnz))
        L.orc_amg_level_copy(self.h, l, rp, col, val)
        return rp, col[:nnz].copy(), val[:nnz].copy()

    def agg(self, l):
        n = lib().orc_amg_level_n(self.h, l)
        a = np.full(n, -1, np.int32)
        lib().orc_amg_level_agg(self.h, l, a)
        return a

    def lam(self, l):
        return lib().orc_amg_level_lambda(self.h, l)

    def sizes(self):
        return [int(lib().orc_amg_level_n(self.h, l)) for l in range(self.n_levels)]

    def vcycle(self, r):
        r = np.ascontiguousarray(r, dtype=np.float64)
        e = np.zeros_like(r)
        lib().orc_amg_vcycle(self.h, r, e)
        return e

    def __del__(self):
        if getattr(self, "owned", False) and self.h:
            lib().orc_amg_free(self.h)
            self.h = None


def colour_jp(A: BSR, seed):
    colour = np.zeros(A.n, np.int32)
    nc = lib().orc_colour_jp(A.n, A.rp, A.col, seed, colour)
    _check(nc, "colour")
    return colour, nc


def colour_geo(A: BSR, grid):
    """Distance-2 order of block ILU(1): cells (x + 2y + 3z) mod 7, the other
    rows first-fit from colour 7 (Sec. "Preconditioners", block ILU(k))."""
    colour = np.zeros(A.n, np.int32)
    nc = lib().orc_colour_geo(int(grid[0]), int(grid[1]), int(grid[2]), A.n, A.rp, A.col, colour)
    _check(nc, "colour_geo")
    return colour, nc


def _ilu_pattern(h, n):
    nnz = lib().orc_bilu_nnz(h)
    rp = np.zeros(n + 1, np.int64)
    col = np.zeros(max(nnz, 1), np.int32)
    lib().orc_bilu_pattern(h, rp, col)
    return rp, col[:nnz]


class BILU0:
    """Block ILU(level) in colour-major order; level 0 on the block pattern,
    level 1 on the level-1 fill pattern (:meth:`pattern`)."""

    def __init__(self, A: BSR, vt, colour, level=0):
        st = C.c_int(0)
        self.A = A
        self.h = lib().orc_biluk_setup(A.n, A.b, A.rp, A.col,
                                       np.ascontiguousarray(vt, dtype=np.float64).reshape(-1),
                                       np.ascontiguousarray(colour, dtype=np.int32), level,
                                       C.byref(st))
        if not self.h:
            raise OracleError(f"bilu setup failed with status {st.value}")

    def solve(self, r):
        y = np.zeros(self.A.n * self.A.b)
        lib().orc_bilu0_solve(self.h, np.ascontiguousarray(r, dtype=np.float64), y)
        return y

    def pattern(self):
        return _ilu_pattern(self.h, self.A.n)

    def factors(self):
        F = np.zeros((max(lib().orc_bilu_nnz(self.h), 1), self.A.b, self.A.b))
        lib().orc_bilu0_factors(self.h, F.reshape(-1))
        return F[:lib().orc_bilu_nnz(self.h)]

    def colours_independent(self, colour):
        return bool(lib().orc_bilu_colours_independent(self.h, np.ascontiguousarray(colour, dtype=np.int32)))

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_bilu0_free(self.h)
            self.h = None


#: default CPR options (the same defaults as the CUDA library)
CPR_DEFAULTS = dict(theta=0.08, coarse_max=64, max_levels=12, cheb_degree=2, seed=0x5EED1812,
                    stages="fpf", decoupling="abf", ilu_fill=0, grid=(0, 0, 0))


class CPR:
    def __init__(self, A: BSR, **kw):
        o = dict(CPR_DEFAULTS)
        o.update(kw)
        self.opts = _CprOpts(o["theta"], o["coarse_max"], o["max_levels"], o["cheb_degree"],
                             o["seed"], STAGES[o["stages"]], DECOUPLINGS[o["decoupling"]],
                             int(o["ilu_fill"]), (C.c_int * 3)(*[int(v) for v in o["grid"]]))
        st = C.c_int(0)
        self.A = A
        self.h = lib().orc_cpr_setup(A.n, A.b, A.rp, A.col, A.val.reshape(-1),
                                     C.byref(self.opts), C.byref(st))
        if not self.h:
            raise OracleError(f"cpr setup failed with status {st.value}")

    def apply(self, v):
        z = np.zeros(self.A.n * self.A.b)
        lib().orc_cpr_apply(self.h, np.ascontiguousarray(v, dtype=np.float64), z)
        return z

    def info(self):
        nl, nc = C.c_int(0), C.c_int(0)
        lib().orc_cpr_info(self.h, C.byref(nl), C.byref(nc))
        return nl.value, nc.value

    @property
    def amg(self):
        return AMG.borrowed(lib().orc_cpr_amg(self.h))

    def colours(self):
        c = np.zeros(self.A.n, np.int32)
        lib().orc_cpr_colours(self.h, c)
        return c

    def decoupled(self):
        vt = np.zeros_like(self.A.val)
        dinv = np.zeros((self.A.n, self.A.b, self.A.b))
        lib().orc_cpr_decoupled(self.h, vt.reshape(-1), dinv.reshape(-1))
        return vt, dinv

    def ilu_pattern(self):
        return _ilu_pattern(lib().orc_cpr_ilu(self.h), self.A.n)

    def ilu_factors(self):
        nnz = lib().orc_bilu_nnz(lib().orc_cpr_ilu(self.h))
        F = np.zeros((max(nnz, 1), self.A.b, self.A.b))
        lib().orc_cpr_ilu_factors(self.h, F.reshape(-1))
        return F[:nnz]

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_cpr_free(self.h)
            self.h = None


@dataclass
class SolveResult:
    x: np.ndarray
    status: int
    iters: int
    restarts: int
    converged: bool
    est_relres: float
    true_relres: float
    history: np.ndarray


def fgmres(A: BSR, cpr: CPR, rhs, rtol=1e-10, restart=30, maxit=1000, x0=None, hist_cap=4096):
    x = np.zeros(A.n * A.b) if x0 is None else np.array(x0, dtype=np.float64)
    st = _Stats()
    hist = np.zeros(hist_cap)
    status = lib().orc_fgmres(A.n, A.b, A.rp, A.col, A.val.reshape(-1), cpr.h,
                              np.ascontiguousarray(rhs, dtype=np.float64), x, rtol, restart,
                              maxit, C.byref(st), hist, hist_cap)
    _check(status, "fgmres")
    nh = min(hist_cap, st.iters + 1)
    return SolveResult(x, status, st.iters, st.restarts, bool(st.converged), st.est_relres,
                       st.true_relres, hist[:nh].copy())


def bicgstab(A: BSR, cpr: CPR, rhs, rtol=1e-10, maxit=1000, x0=None, hist_cap=4096):
    x = np.zeros(A.n * A.b) if x0 is None else np.array(x0, dtype=np.float64)
    st = _Stats()
    hist = np.zeros(hist_cap)
    status = lib().orc_bicgstab(A.n, A.b, A.rp, A.col, A.val.reshape(-1), cpr.h,
                                np.ascontiguousarray(rhs, dtype=np.float64), x, rtol, maxit,
                                C.byref(st), hist, hist_cap)
    _check(status, "bicgstab")
    nh = min(hist_cap, st.iters + 1)
    return SolveResult(x, status, st.iters, st.restarts, bool(st.converged), st.est_relres,
                       st.true_relres, hist[:nh].copy())


def outer_product(A: BSR, lam, x):
    dA = np.zeros_like(A.val)
    lib().orc_outer_product(A.n, A.b, A.rp, A.col, np.ascontiguousarray(lam, dtype=np.float64),
                            np.ascontiguousarray(x, dtype=np.float64), dA.reshape(-1))
    return dA


def chain_theta(sysm, A: BSR, dA):
    dth = np.zeros(sysm.nx * sysm.ny * sysm.nz)
    _check(lib().orc_chain_theta(sysm.nx, sysm.ny, sysm.nz, sysm.b, sysm.k, sysm.kvkh, sysm.c_t,
                                 sysm.M.reshape(-1), A.rp, A.col,
                                 np.ascontiguousarray(dA).reshape(-1), dth), "chain")
    return dth


def adjoint(A: BSR, g, x, rtol=1e-10, restart=30, maxit=1000, **cpr_kw):
    """Solve A^T lambda = g with CPR built on A^T; returns (lambda, dL/dA, result)."""
    AT = transpose(A)
    cpr = CPR(AT, **cpr_kw)
    res = fgmres(AT, cpr, g, rtol=rtol, restart=restart, maxit=maxit)
    return res.x, outer_product(A, res.x, x), res


def well_cell_indicator(sysm):
    """g = dL/dx for L = sum over perforated cells (each once) of the cell
    pressure (entry 0 of the cell block)."""
    g = np.zeros(sysm.n_unknowns)
    cells = np.unique(sysm.perf_cell)
    g[cells.astype(np.int64) * sysm.b] = 1.0
    return g


# ------------------------------------------------------------- thermal model
class Thermal:
    """Residual and Jacobian of the water + heavy-oil thermal model on a
    synthetic system's grid and wells (trs_thermal.c), for a ThermalState."""

    def __init__(self, sysm, state, swt, slt):
        self.s = sysm
        self.t = state
        self.P = thermal_params(state.params)
        self.swt = np.ascontiguousarray(swt, dtype=np.float64)
        self.slt = np.ascontiguousarray(slt, dtype=np.float64)

    def _args(self, u):
        s, t = self.s, self.t
        return (s.nx, s.ny, s.nz, s.n_wells, len(s.perf_cell), C.byref(self.P), self.swt.reshape(-1),
                len(self.swt), self.slt.reshape(-1), len(self.slt), s.k, s.perf_well, s.perf_cell, t.wi,
                t.well_type, t.well_target, t.gas, np.ascontiguousarray(u, dtype=np.float64), t.u_old)

    @staticmethod
    def _rows(rows):
        if rows is None:
            return 0, None, None
        r = np.ascontiguousarray(rows, dtype=np.int64)
        return len(r), r.ctypes.data_as(C.c_void_p), r

    def residual(self, u=None, rows=None):
        """R(u); with rows, only those cell rows (and the well rows) are filled."""
        R = np.zeros(self.s.n_unknowns)
        nr, rp_, keep = self._rows(rows)
        _check(lib().orc_thermal_residual(*self._args(self.t.u if u is None else u), nr, rp_, R),
               "thermal residual")
        return R

    def jacobian(self, u=None, rows=None, pattern=None) -> BSR:
        """dR/du in BSR on the pattern of the synthetic assembly (7-point +
        wells); with rows, only those cell rows (and the well rows) are filled."""
        A0 = pattern if pattern is not None else assemble(self.s)
        val = np.zeros_like(A0.val)
        nr, rp_, keep = self._rows(rows)
        _check(lib().orc_thermal_jacobian(*self._args(self.t.u if u is None else u), nr, rp_, A0.rp, A0.col,
                                          val.reshape(-1)), "thermal jacobian")
        return BSR(A0.n, A0.b, A0.rp, A0.col, val)

    def props(self, u_cell):
        out = np.zeros(16)
        lib().orc_thermal_props(C.byref(self.P), self.swt.reshape(-1), len(self.swt), self.slt.reshape(-1),
                                len(self.slt), np.ascontiguousarray(u_cell, dtype=np.float64), out)
        keys = ("phi", "rho_w", "rho_o", "rho_g", "lam_w", "lam_o", "lam_g", "H_w", "H_o", "H_g", "U_w", "U_o",
                "U_g", "U_r", "K_T", "K_star")
        return dict(zip(keys, out))

    def totals(self, u):
        out = np.zeros(3)
        s = self.s
        lib().orc_thermal_totals(s.nx, s.ny, s.nz, C.byref(self.P), self.swt.reshape(-1), len(self.swt),
                                 self.slt.reshape(-1), len(self.slt), np.ascontiguousarray(u, dtype=np.float64),
                                 out)
        return out

    def well_sources(self, u=None):
        out = np.zeros(3)
        s, t = self.s, self.t
        lib().orc_thermal_well_sources(s.nx, s.ny, s.nz, s.n_wells, len(s.perf_cell), C.byref(self.P),
                                       self.swt.reshape(-1), len(self.swt), self.slt.reshape(-1), len(self.slt),
                                       s.perf_well, s.perf_cell, t.wi, t.well_type,
                                       np.ascontiguousarray(t.u if u is None else u, dtype=np.float64), out)
        return out


def rk_z(A, B):
    return lib().orc_rk_z(float(A), float(B))
