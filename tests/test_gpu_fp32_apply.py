"""The FP32-preconditioner form of CPR (Ã, the block ILU(0) factors, the
pressure levels and the preconditioner's vectors in FP32; the coarsest
inverse in FP64) against the FP64 oracle, element by element, for every
stage ordering (Sec. "Preconditioners": FPF, FP, PF) and decoupling (Sec.
"Decoupling Methods": ABF, NONE, FRS, FRS+ABF).

The setup objects that decide integers are built in FP64 on both sides, so
the aggregates and colours are the oracle's; what differs is the rounding of
every stored operator and every operation to binary32.  The tolerance is a
first-order count of those roundings along the longest chain of dependent
operations of one application, each contributing at most a unit roundoff
u = 2^-24 relative to the quantities it combines:

  K = n_F * 2 * C * (m + b + 1)      block ILU sweeps: n_F solves, forward and
                                     backward over C colours, rows of m terms
                                     plus the b x b diagonal inverse
    + n_R * (m + 1)                  residuals f - Ã y
    + sum_l (2 d + 2) * (m_l + 2)    Chebyshev(d) pre/post, restriction and
                                     prolongation on level l (rows of m_l terms)
    + (b + 1)                        input scaling D^-1 v and the cast

with n_F = n_R = 2 for FPF and 1 for FP and PF, and m the longest row of Ã in
scalar terms.  K u is the worst case, every rounding of one sign.  The test
asserts the probabilistic form of the same count (Higham & Mary, "A new
approach to probabilistic rounding error analysis", SIAM J. Sci. Comput.
41(5), 2019): with rounding errors independent and of mean zero, the
accumulated relative error stays below lambda sqrt(K) u with probability at
least 1 - 2 exp(-lambda^2 / 2); lambda = 8 (a failure probability below
3e-14 per case).  It applies as a relative 2-norm error of z and assumes the
stages do not amplify rounding, which holds for the diagonally dominant
decoupled systems here (measured errors at 128x128x64 are 2e-7 to 8e-7,
about 3 to 13 u, against bounds near 5e-5).  A wrong operator -- a stale
factor, a missing colour, a cast through a 16-bit type (relative error near
5e-4 for binary16, 4e-3 for bfloat16) -- fails it.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

from test_gpu_parity import CASES, _case_id, _gpu_system, _rel, _sys  # noqa: E402

U32 = 2.0 ** -24
DECOUPLINGS = ["abf", "none", "frs", "frs+abf"]
STAGES = ["fpf", "fp", "pf"]


@pytest.fixture(scope="module")
def trs():
    from paper_1812_03952_gb300 import build as B
    B.build()
    from paper_1812_03952_gb300 import trs as T
    T.load()
    return T


LAMBDA = 8.0


def rounding_count(Ao, Mo, stages, cheb_degree=2):
    """K of the module docstring for one application of the oracle's CPR Mo
    (its colour count and AMG levels) on the matrix Ao."""
    b = Ao.b
    m = int(np.max(np.diff(Ao.rp))) * b
    n_levels, n_colours = Mo.info()
    n_f = 2 if stages == "fpf" else 1
    k = n_f * 2 * n_colours * (m + b + 1) + n_f * (m + 1) + (b + 1)
    amg = Mo.amg
    for l in range(n_levels):
        rp = amg.level(l)[0]
        m_l = int(np.max(np.diff(rp))) if len(rp) > 1 else 1
        k += (2 * cheb_degree + 2) * (m_l + 2)
    return k


def fp32_apply_tolerance(Ao, Mo, stages, cheb_degree=2):
    """lambda sqrt(K) u: the probabilistic rounding bound of one FP32 application."""
    return LAMBDA * np.sqrt(rounding_count(Ao, Mo, stages, cheb_degree)) * U32


@pytest.mark.parametrize("decoupling", DECOUPLINGS)
@pytest.mark.parametrize("stages", STAGES)
@pytest.mark.parametrize("case", CASES, ids=_case_id)
def test_fp32_cpr_apply_matches_oracle(trs, oracle, synth, case, stages, decoupling):
    s = _sys(synth, **case)
    ds = _gpu_system(trs, s)
    Ao = oracle.assemble(s)
    kw = dict(coarse_max=40, stages=stages, decoupling=decoupling)
    Mo = oracle.CPR(Ao, **kw)
    M = trs.CPR(ds.A, precision="fp32", **kw)
    # the integer decisions are the oracle's
    np.testing.assert_array_equal(M.colours(), Mo.colours())
    assert M.info()["level_rows"] == Mo.amg.sizes()
    tol = fp32_apply_tolerance(Ao, Mo, stages)
    rng = np.random.default_rng(21)
    for _ in range(2):
        v = rng.standard_normal(Ao.n * Ao.b)
        z = M.apply(torch.from_numpy(v).cuda()).cpu().numpy()
        zo = Mo.apply(v)
        err = _rel(z, zo)
        assert err <= tol, f"FP32 application differs from the oracle by {err:.3e} > {tol:.3e}"
        # FP32 rounding is present: the FP32 path is not secretly the FP64 one
        assert err > 0.0


def test_fp32_vcycle_matches_oracle(trs, oracle, synth):
    """The pressure V-cycle alone in FP32 against the oracle's FP64 V-cycle."""
    case = CASES[5]
    s = _sys(synth, **case)
    ds = _gpu_system(trs, s)
    Ao = oracle.assemble(s)
    Mo = oracle.CPR(Ao, coarse_max=40)
    M = trs.CPR(ds.A, precision="fp32", coarse_max=40)
    n0 = Mo.amg.sizes()[0]
    r = np.random.default_rng(22).standard_normal(n0)
    e = M.vcycle(torch.from_numpy(r).cuda()).cpu().numpy()
    eo = Mo.amg.vcycle(r)
    n_levels = Mo.amg.n_levels
    k = 0
    for l in range(n_levels):
        rp = Mo.amg.level(l)[0]
        k += 6 * (int(np.max(np.diff(rp))) + 2)
    assert 0.0 < _rel(e, eo) <= LAMBDA * np.sqrt(k) * U32
