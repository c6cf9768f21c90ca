"""ctypes binding of libtrs (C ABI in include/trs.h).

Argument marshalling only: every step of the solve runs in the CUDA library.
Device arrays are torch CUDA tensors (float64, contiguous) passed by their
data pointers on torch's current stream; host arrays are numpy arrays.  A
missing library or a missing GPU is an error, never a fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtrs.so")

TRS_OK = 0
TRS_ERR_INVALID = -1
TRS_ERR_OOM = -2
TRS_ERR_CUDA = -3
TRS_ERR_SINGULAR_BLOCK = -4
TRS_ERR_NAN = -5
TRS_ERR_NOT_CONVERGED = -6
TRS_ERR_BREAKDOWN = -7
TRS_ERR_COARSENING = -8
TRS_ERR_UNSUPPORTED = -9

TRS_FP64 = 0
TRS_FP32_PREC = 1
TRS_FGMRES = 0
TRS_BICGSTAB = 1
METHODS = {"fgmres": TRS_FGMRES, "bicgstab": TRS_BICGSTAB}
#: CPR stage orderings and decoupling methods by name
STAGES = {"fpf": 0, "fp": 1, "pf": 2}
DECOUPLINGS = {"abf": 0, "none": 1, "frs": 2, "frs+abf": 3}

#: every entry point declared in include/trs.h
EXPORTS = (
    "trs_bsr_create", "trs_bsr_create_synthetic", "trs_bsr_assemble", "trs_bsr_assemble_host",
    "trs_bsr_update_values",
    "trs_bsr_get_values", "trs_bsr_scale_diagonal", "trs_bsr_pattern", "trs_bsr_get_info",
    "trs_bsr_spmv", "trs_bsr_transpose", "trs_bsr_transpose_values", "trs_bsr_destroy", "trs_cpr_default_opts", "trs_cpr_setup",
    "trs_cpr_update", "trs_cpr_apply", "trs_cpr_get_info", "trs_cpr_get_aggregates",
    "trs_cpr_get_colours", "trs_cpr_get_decoupled", "trs_cpr_get_level", "trs_cpr_vcycle",
    "trs_cpr_destroy", "trs_solve_default_opts", "trs_fgmres_solve", "trs_fgmres_solve_host",
    "trs_bicgstab_solve", "trs_bicgstab_solve_host", "trs_solve_adjoint", "trs_outer_product", "trs_chain_theta", "trs_last_error", "trs_version",
    "trs_kernel_launches", "trs_residual_norm_noalloc", "trs_profile_spmv", "trs_thermal_assemble",
    "trs_test_stall_staged_copies",
)


class TrsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{msg} (status {code})")
        self.code = code


class CprOpts(C.Structure):
    _fields_ = [("precision", C.c_int32), ("theta", C.c_double), ("coarse_max", C.c_int32),
                ("max_levels", C.c_int32), ("cheb_degree", C.c_int32), ("seed", C.c_uint32),
                ("stages", C.c_int32), ("decoupling", C.c_int32), ("ilu_fill", C.c_int32)]


class SolveOpts(C.Structure):
    _fields_ = [("rtol", C.c_double), ("restart", C.c_int32), ("maxit", C.c_int32),
                ("use_x0", C.c_int32), ("method", C.c_int32), ("time_phases", C.c_int32)]


class SolveStats(C.Structure):
    _fields_ = [("iters", C.c_int32), ("restarts", C.c_int32), ("converged", C.c_int32),
                ("amg_levels", C.c_int32), ("n_colours", C.c_int32), ("est_relres", C.c_double),
                ("true_relres", C.c_double), ("ms_setup", C.c_double), ("ms_solve", C.c_double),
                ("ms_precond", C.c_double), ("ms_spmv", C.c_double), ("ms_orth", C.c_double),
                ("spmv_launches", C.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


#: field order of trs_thermal_params (include/trs.h)
THERMAL_FIELDS = (
    "dx", "dy", "dz", "depth_top", "dt", "kvkh", "gravity",
    "phi_ref", "cpor", "ctpor", "p_ref", "T_ref", "cp1_r", "cp2_r",
    "kt_w", "kt_o", "kt_g", "kt_r",
    "rho_w_ref", "cp_w", "ct1_w", "ct2_w", "cpt_w", "mw_w", "avisc_w", "bvisc_w",
    "kv1", "kv2", "kv3", "kv4", "kv5", "per_eps", "tc_w", "pc_w")
THERMAL_FIELDS_2 = ("hvr", "ev", "rho_o_ref", "cp_o", "ct1_o", "ct2_o", "cpt_o", "mw_o", "avisc_o", "bvisc_o",
                    "cpl1_o", "mug_a", "mug_b", "h_inj", "R_gas")


class ThermalParams(C.Structure):
    _fields_ = ([(f, C.c_double) for f in THERMAL_FIELDS] + [("cpg", C.c_double * 5)]
                + [(f, C.c_double) for f in THERMAL_FIELDS_2])

    @classmethod
    def from_dict(cls, d):
        P = cls()
        for f in THERMAL_FIELDS + THERMAL_FIELDS_2:
            setattr(P, f, float(d[f]))
        P.cpg = (C.c_double * 5)(*[float(d[f"cpg{k}"]) for k in range(1, 6)])
        return P


class BsrInfo(C.Structure):
    _fields_ = [("n_block_rows", C.c_int64), ("b", C.c_int32), ("nnzb", C.c_int64),
                ("n_cells", C.c_int64), ("grid", C.c_int32 * 3)]


class CprInfo(C.Structure):
    _fields_ = [("n_levels", C.c_int32), ("n_colours", C.c_int32), ("precision", C.c_int32),
                ("level_rows", C.c_int64 * 16), ("level_nnz", C.c_int64 * 16),
                ("level_lambda", C.c_double * 16)]


_lib = None
vp = C.c_void_p


def load(path: str = LIB_PATH):
    """Loads libtrs.so; raises if it is missing (build it first)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libtrs.so not found at {path}: run __graft_entry__.build()")
    L = C.CDLL(path)
    i32, i64, f64, u32 = C.c_int32, C.c_int64, C.c_double, C.c_uint32
    sig = {
        "trs_bsr_create": (i32, [i64, i32, vp, vp, vp, vp, vp, C.POINTER(vp)]),
        "trs_bsr_create_synthetic": (i32, [i32, i32, i32, i32, i32, i64, vp, vp, vp, C.POINTER(vp)]),
        "trs_bsr_assemble": (i32, [vp, vp, i32, f64, f64, vp, vp, vp, vp, vp]),
        "trs_bsr_assemble_host": (i32, [vp, vp, i32, f64, f64, vp, vp, vp, vp, vp]),
        "trs_bsr_update_values": (i32, [vp, vp, i32, vp]),
        "trs_bsr_get_values": (i32, [vp, vp, i32, vp]),
        "trs_bsr_scale_diagonal": (i32, [vp, vp, vp]),
        "trs_bsr_pattern": (i32, [vp, vp, vp]),
        "trs_bsr_get_info": (i32, [vp, C.POINTER(BsrInfo)]),
        "trs_bsr_spmv": (i32, [vp, f64, vp, f64, vp, i32, vp]),
        "trs_bsr_transpose": (i32, [vp, vp, C.POINTER(vp)]),
        "trs_bsr_transpose_values": (i32, [vp, vp, vp]),
        "trs_bsr_destroy": (None, [vp]),
        "trs_cpr_default_opts": (None, [C.POINTER(CprOpts)]),
        "trs_cpr_setup": (i32, [vp, C.POINTER(CprOpts), vp, C.POINTER(vp)]),
        "trs_cpr_update": (i32, [vp, vp, i32, vp]),
        "trs_cpr_apply": (i32, [vp, vp, vp, vp]),
        "trs_cpr_get_info": (i32, [vp, C.POINTER(CprInfo)]),
        "trs_cpr_get_aggregates": (i32, [vp, i32, vp]),
        "trs_cpr_get_colours": (i32, [vp, vp]),
        "trs_cpr_get_decoupled": (i32, [vp, vp, vp]),
        "trs_cpr_get_level": (i32, [vp, i32, vp, vp, vp]),
        "trs_cpr_vcycle": (i32, [vp, vp, vp, vp]),
        "trs_cpr_destroy": (None, [vp]),
        "trs_solve_default_opts": (None, [C.POINTER(SolveOpts)]),
        "trs_fgmres_solve": (i32, [vp, vp, vp, vp, C.POINTER(SolveOpts), vp, C.POINTER(SolveStats)]),
        "trs_fgmres_solve_host": (i32, [vp, vp, vp, vp, C.POINTER(SolveOpts), vp,
                                        C.POINTER(SolveStats)]),
        "trs_bicgstab_solve": (i32, [vp, vp, vp, vp, C.POINTER(SolveOpts), vp, C.POINTER(SolveStats)]),
        "trs_bicgstab_solve_host": (i32, [vp, vp, vp, vp, C.POINTER(SolveOpts), vp,
                                          C.POINTER(SolveStats)]),
        "trs_solve_adjoint": (i32, [vp, vp, vp, vp, vp, vp, vp, C.POINTER(SolveOpts), vp,
                                    C.POINTER(SolveStats)]),
        "trs_outer_product": (i32, [vp, vp, vp, vp, vp]),
        "trs_chain_theta": (i32, [vp, vp, i32, f64, f64, vp, vp, vp, vp, vp]),
        "trs_last_error": (C.c_char_p, []),
        "trs_version": (C.c_char_p, []),
        "trs_kernel_launches": (C.c_uint64, []),
        "trs_residual_norm_noalloc": (i32, [vp, vp, vp, vp, C.POINTER(C.c_double), vp]),
        "trs_profile_spmv": (i32, [i32, C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
        "trs_thermal_assemble": (i32, [vp, C.POINTER(ThermalParams), vp, i32, vp, i32, vp, vp, vp, vp, vp, vp,
                                       vp, vp, vp]),
        "trs_test_stall_staged_copies": (i32, [i32]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def kernel_launches() -> int:
    return int(load().trs_kernel_launches())


def profile_spmv(enable: bool):
    """Starts (enable) or stops timing of the FGMRES operator SpMV launches;
    returns (total_ms, launches) accumulated before this call."""
    ms, n = C.c_double(0.0), C.c_int64(0)
    _check(load().trs_profile_spmv(int(enable), C.byref(ms), C.byref(n)))
    return ms.value, n.value


def test_stall_staged_copies(extra_bytes: int):
    """Testing only: the staged Gram-Schmidt waits expect extra_bytes more
    than their copies deliver, so they run out (0 restores normal operation)."""
    _check(load().trs_test_stall_staged_copies(int(extra_bytes)))


def _check(code, allow=()):
    if code != TRS_OK and code not in allow:
        raise TrsError(code, load().trs_last_error().decode())
    return code


def _stream():
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dptr(t):
    """Device pointer of a contiguous CUDA float64/int tensor (or None)."""
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return C.c_void_p(t.data_ptr())


def _hptr(a):
    """Host pointer of a contiguous numpy array or CPU torch tensor (or None)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("expected a contiguous host array")
        return a.ctypes.data_as(C.c_void_p)
    if a.is_cuda or not a.is_contiguous():
        raise ValueError("expected a contiguous CPU tensor")
    return C.c_void_p(a.data_ptr())


def _empty(n, dtype=None, device="cuda"):
    import torch
    return torch.empty(n, dtype=dtype or torch.float64, device=device)


class Matrix:
    """Device block matrix (trs_bsr)."""

    def __init__(self, handle, keep=None):
        self.h = handle
        self._keep = keep
        info = BsrInfo()
        _check(load().trs_bsr_get_info(self.h, C.byref(info)))
        self.n = info.n_block_rows
        self.b = info.b
        self.nnzb = info.nnzb
        self.n_cells = info.n_cells
        self.grid = tuple(info.grid)

    @property
    def N(self):
        return self.n * self.b

    @classmethod
    def from_bsr(cls, rp, col, values, b, grid=None):
        rp = np.ascontiguousarray(rp, dtype=np.int64)
        col = np.ascontiguousarray(col, dtype=np.int32)
        vals = None if values is None else np.ascontiguousarray(values, dtype=np.float64)
        g = None if grid is None else np.ascontiguousarray(grid, dtype=np.int32)
        out = C.c_void_p()
        _check(load().trs_bsr_create(len(rp) - 1, b, _hptr(rp), _hptr(col),
                                     None if vals is None else _hptr(vals),
                                     None if g is None else _hptr(g), _stream(), C.byref(out)))
        return cls(out)

    @classmethod
    def synthetic_pattern(cls, nx, ny, nz, b, n_wells, perf_well, perf_cell):
        pw = np.ascontiguousarray(perf_well, dtype=np.int32)
        pc = np.ascontiguousarray(perf_cell, dtype=np.int32)
        out = C.c_void_p()
        _check(load().trs_bsr_create_synthetic(nx, ny, nz, b, n_wells, len(pc), _hptr(pw), _hptr(pc),
                                               _stream(), C.byref(out)))
        return cls(out)

    def assemble(self, perm, M, acc, wi, lam, kvkh, c_t, perm_is_log=False):
        _check(load().trs_bsr_assemble(self.h, _dptr(perm), int(perm_is_log), kvkh, c_t, _dptr(M),
                                       _dptr(acc), _dptr(wi), _dptr(lam), _stream()))

    def assemble_host(self, perm, M, acc, wi, lam, kvkh, c_t, perm_is_log=False):
        """trs_bsr_assemble from host buffers (float64 numpy arrays or CPU
        tensors, pinned for asynchronous copies); the copies are part of the call."""
        _check(load().trs_bsr_assemble_host(self.h, _hptr(perm), int(perm_is_log), kvkh, c_t, _hptr(M),
                                            _hptr(acc), _hptr(wi), _hptr(lam), _stream()))

    def update_values(self, values):
        if isinstance(values, np.ndarray):
            v = np.ascontiguousarray(values, dtype=np.float64)
            _check(load().trs_bsr_update_values(self.h, _hptr(v), 0, _stream()))
        else:
            _check(load().trs_bsr_update_values(self.h, _dptr(values), 1, _stream()))

    def values(self):
        out = np.zeros(self.nnzb * self.b * self.b)
        _check(load().trs_bsr_get_values(self.h, _hptr(out), 0, _stream()))
        return out.reshape(self.nnzb, self.b, self.b)

    def scale_diagonal(self, s):
        _check(load().trs_bsr_scale_diagonal(self.h, _dptr(s), _stream()))

    def pattern(self):
        rp = np.zeros(self.n + 1, np.int64)
        col = np.zeros(max(1, self.nnzb), np.int32)
        _check(load().trs_bsr_pattern(self.h, _hptr(rp), _hptr(col)))
        return rp, col[: self.nnzb]

    def spmv(self, x, y=None, alpha=1.0, beta=0.0, transpose=False):
        if y is None:
            y = _empty(self.N, device=x.device)
            beta = 0.0
        _check(load().trs_bsr_spmv(self.h, alpha, _dptr(x), beta, _dptr(y), int(transpose), _stream()))
        return y

    def transpose(self, into=None):
        """A^T as a new matrix, or refreshed in place into an earlier transpose."""
        if into is not None:
            _check(load().trs_bsr_transpose_values(self.h, into.h, _stream()))
            return into
        out = C.c_void_p()
        _check(load().trs_bsr_transpose(self.h, _stream(), C.byref(out)))
        return Matrix(out)

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.trs_bsr_destroy(self.h)
            self.h = None


def default_cpr_opts(**kw):
    o = CprOpts()
    load().trs_cpr_default_opts(C.byref(o))
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = {"fp64": TRS_FP64, "fp32": TRS_FP32_PREC}[v]
        elif k == "stages" and isinstance(v, str):
            v = STAGES[v]
        elif k == "decoupling" and isinstance(v, str):
            v = DECOUPLINGS[v]
        setattr(o, k, v)
    return o


def default_solve_opts(**kw):
    o = SolveOpts()
    load().trs_solve_default_opts(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class CPR:
    """CPR-FPF preconditioner handle (trs_cpr)."""

    def __init__(self, A: Matrix, **opts):
        self.opts = default_cpr_opts(**opts)
        out = C.c_void_p()
        _check(load().trs_cpr_setup(A.h, C.byref(self.opts), _stream(), C.byref(out)))
        self.h = out
        self.n, self.b = A.n, A.b

    def update(self, A: Matrix, reuse_amg=True):
        _check(load().trs_cpr_update(self.h, A.h, int(reuse_amg), _stream()))

    def apply(self, v):
        z = _empty(self.n * self.b, device=v.device)
        _check(load().trs_cpr_apply(self.h, _dptr(v), _dptr(z), _stream()))
        return z

    def vcycle(self, r):
        e = _empty(r.numel(), device=r.device)
        _check(load().trs_cpr_vcycle(self.h, _dptr(r), _dptr(e), _stream()))
        return e

    def info(self):
        i = CprInfo()
        _check(load().trs_cpr_get_info(self.h, C.byref(i)))
        L = i.n_levels
        return {"n_levels": L, "n_colours": i.n_colours, "precision": i.precision,
                "level_rows": list(i.level_rows[:L]), "level_nnz": list(i.level_nnz[:L]),
                "level_lambda": list(i.level_lambda[:L])}

    def aggregates(self, level):
        n = self.info()["level_rows"][level]
        a = np.zeros(n, np.int32)
        _check(load().trs_cpr_get_aggregates(self.h, level, _hptr(a)))
        return a

    def colours(self):
        c = np.zeros(self.n, np.int32)
        _check(load().trs_cpr_get_colours(self.h, _hptr(c)))
        return c

    def decoupled(self, nnzb):
        vt = np.zeros(nnzb * self.b * self.b)
        dinv = np.zeros(self.n * self.b * self.b)
        _check(load().trs_cpr_get_decoupled(self.h, _hptr(vt), _hptr(dinv)))
        return vt.reshape(nnzb, self.b, self.b), dinv.reshape(self.n, self.b, self.b)

    def level(self, l):
        inf = self.info()
        n, nnz = inf["level_rows"][l], inf["level_nnz"][l]
        rp = np.zeros(n + 1, np.int64)
        col = np.zeros(max(1, nnz), np.int32)
        val = np.zeros(max(1, nnz))
        _check(load().trs_cpr_get_level(self.h, l, _hptr(rp), _hptr(col), _hptr(val)))
        return rp, col[:nnz], val[:nnz]

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.trs_cpr_destroy(self.h)
            self.h = None


@dataclass
class Result:
    status: int
    stats: dict


def _device_solve(fn, A: Matrix, M: CPR, b, x, rtol, restart, maxit, use_x0, time_phases=False):
    if x is None:
        x = _empty(A.N, device=b.device)
        use_x0 = False
    o = default_solve_opts(rtol=rtol, restart=restart, maxit=maxit, use_x0=int(use_x0),
                           time_phases=int(time_phases))
    st = SolveStats()
    code = fn(A.h, M.h, _dptr(b), _dptr(x), C.byref(o), _stream(), C.byref(st))
    _check(code, allow=(TRS_ERR_NOT_CONVERGED,))
    return x, Result(code, st.as_dict())


def _host_solve(fn, A: Matrix, M: CPR, b, rtol, restart, maxit, x=None):
    bb = np.ascontiguousarray(b, dtype=np.float64) if isinstance(b, np.ndarray) else b
    if x is None:
        x = np.zeros(A.N)
    o = default_solve_opts(rtol=rtol, restart=restart, maxit=maxit, use_x0=0)
    st = SolveStats()
    code = fn(A.h, M.h, _hptr(bb), _hptr(x), C.byref(o), _stream(), C.byref(st))
    _check(code, allow=(TRS_ERR_NOT_CONVERGED,))
    return x, Result(code, st.as_dict())


def fgmres_solve(A: Matrix, M: CPR, b, x=None, rtol=1e-6, restart=30, maxit=1000, use_x0=False,
                 time_phases=False):
    """Solves A x = b by FGMRES (device tensors); returns (x, Result).
    time_phases: fill the per-phase device times of the stats."""
    return _device_solve(load().trs_fgmres_solve, A, M, b, x, rtol, restart, maxit, use_x0, time_phases)


def fgmres_solve_host(A: Matrix, M: CPR, b, rtol=1e-6, restart=30, maxit=1000, x=None):
    """The same solve with host vectors (numpy arrays or CPU tensors, x
    optional and overwritten); the copies are part of the call."""
    return _host_solve(load().trs_fgmres_solve_host, A, M, b, rtol, restart, maxit, x)


def bicgstab_solve(A: Matrix, M: CPR, b, x=None, rtol=1e-6, maxit=1000, use_x0=False, time_phases=False):
    """Solves A x = b by BiCGSTAB (device tensors); returns (x, Result)."""
    return _device_solve(load().trs_bicgstab_solve, A, M, b, x, rtol, 30, maxit, use_x0, time_phases)


def bicgstab_solve_host(A: Matrix, M: CPR, b, rtol=1e-6, maxit=1000, x=None):
    """BiCGSTAB with host vectors; the copies are part of the call."""
    return _host_solve(load().trs_bicgstab_solve_host, A, M, b, rtol, 30, maxit, x)


def krylov_solve(method: str, A: Matrix, M: CPR, b, x=None, rtol=1e-6, restart=30, maxit=1000,
                 use_x0=False, time_phases=False):
    """FGMRES or BiCGSTAB by name ("fgmres" | "bicgstab")."""
    if method == "fgmres":
        return fgmres_solve(A, M, b, x, rtol=rtol, restart=restart, maxit=maxit, use_x0=use_x0,
                            time_phases=time_phases)
    if method == "bicgstab":
        return bicgstab_solve(A, M, b, x, rtol=rtol, maxit=maxit, use_x0=use_x0, time_phases=time_phases)
    raise ValueError(f"unknown Krylov method {method!r}")


def solve_adjoint(A: Matrix, AT: Matrix, MT: CPR, g, x=None, want_dA=False, rtol=1e-6, restart=30,
                  maxit=1000, method="fgmres"):
    lam = _empty(A.N, device=g.device)
    dA = _empty(A.nnzb * A.b * A.b, device=g.device) if want_dA else None
    o = default_solve_opts(rtol=rtol, restart=restart, maxit=maxit, use_x0=0)
    o.method = METHODS[method]
    st = SolveStats()
    code = load().trs_solve_adjoint(A.h, AT.h, MT.h, _dptr(g), _dptr(x), _dptr(lam), _dptr(dA),
                                    C.byref(o), _stream(), C.byref(st))
    _check(code, allow=(TRS_ERR_NOT_CONVERGED,))
    return lam, dA, Result(code, st.as_dict())


def residual_norm_noalloc(A: Matrix, x, b, r):
    """r = b - A x (written into the caller's r) and ||r||_2, computed without
    any device allocation (static scratch inside the library)."""
    nrm = C.c_double(0.0)
    _check(load().trs_residual_norm_noalloc(A.h, _dptr(x), _dptr(b), _dptr(r), C.byref(nrm), _stream()))
    return nrm.value


def outer_product(A: Matrix, lam, x):
    dA = _empty(A.nnzb * A.b * A.b, device=lam.device)
    _check(load().trs_outer_product(A.h, _dptr(lam), _dptr(x), _dptr(dA), _stream()))
    return dA


def chain_theta(A: Matrix, perm, M, lam, x, kvkh, c_t, perm_is_log=False):
    dth = _empty(A.n_cells, device=lam.device)
    _check(load().trs_chain_theta(A.h, _dptr(perm), int(perm_is_log), kvkh, c_t, _dptr(M), _dptr(lam),
                                  _dptr(x), _dptr(dth), _stream()))
    return dth


class ThermalSystem:
    """The thermal model on a synthetic system's grid and wells, resident on
    the GPU: permeability, state, previous state, gas flags and well data;
    assemble() fills A (made by trs_bsr_create_synthetic, b = 4) with the
    Jacobian dR/du and returns the residual R(u) as a device tensor."""

    def __init__(self, sysm, state, swt, slt, device="cuda"):
        import torch
        if sysm.b != 4:
            raise ValueError("the thermal model has b = 4")
        self.sysm = sysm
        self.state = state
        self.P = ThermalParams.from_dict(state.params)
        self.swt = np.ascontiguousarray(swt, dtype=np.float64)
        self.slt = np.ascontiguousarray(slt, dtype=np.float64)
        t = lambda a, dt=None: torch.from_numpy(np.ascontiguousarray(a)).to(device)
        self.A = Matrix.synthetic_pattern(sysm.nx, sysm.ny, sysm.nz, sysm.b, sysm.n_wells,
                                          sysm.perf_well, sysm.perf_cell)
        self.k = t(sysm.k)
        self.u = t(state.u)
        self.u_old = t(state.u_old)
        self.gas = t(state.gas)
        one = lambda a, dtype: t(a) if len(a) else torch.zeros(1, dtype=dtype, device=device)
        self.wi = one(state.wi, torch.float64)
        self.well_type = one(state.well_type, torch.int32)
        self.well_target = one(state.well_target, torch.float64)
        self.R = _empty(sysm.n_unknowns, device=device)

    def assemble(self, u=None):
        uu = self.u if u is None else u
        _check(load().trs_thermal_assemble(self.A.h, C.byref(self.P), _hptr(self.swt), len(self.swt),
                                           _hptr(self.slt), len(self.slt), _dptr(self.k), _dptr(uu),
                                           _dptr(self.u_old), _dptr(self.gas), _dptr(self.wi),
                                           _dptr(self.well_type), _dptr(self.well_target), _dptr(self.R),
                                           _stream()))
        return self.R


class DeviceSystem:
    """A synthetic system resident on the GPU: pattern, assembly inputs, RHS."""

    def __init__(self, sysm, device="cuda"):
        import torch
        self.sysm = sysm
        self.A = Matrix.synthetic_pattern(sysm.nx, sysm.ny, sysm.nz, sysm.b, sysm.n_wells,
                                          sysm.perf_well, sysm.perf_cell)
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device)
        self.k = t(sysm.k)
        self.M = t(sysm.M.reshape(-1))
        self.acc = t(sysm.acc.reshape(-1))
        self.wi = t(sysm.wi) if len(sysm.wi) else torch.zeros(1, dtype=torch.float64, device=device)
        self.lam = t(sysm.lam.reshape(-1)) if len(sysm.wi) else torch.zeros(1, dtype=torch.float64,
                                                                            device=device)
        self.rhs = t(sysm.rhs)

    def assemble(self, perm=None, perm_is_log=False):
        self.A.assemble(self.k if perm is None else perm, self.M, self.acc, self.wi, self.lam,
                        self.sysm.kvkh, self.sysm.c_t, perm_is_log)
        return self.A
