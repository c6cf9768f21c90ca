"""FGMRES solves whose Arnoldi steps go through every orthogonalisation path.

CGS2 at step j works on K = j + 1 basis vectors.  Up to K + 1 = 32 the basis
tiles are staged in shared memory by bulk copies in kernels sized for 8, 16
or 32 vectors, or, when N is odd (rows not 16-byte aligned), read by the
register kernels; beyond 32 vectors the multi-dot and update passes run.
Each solve here runs long enough to pass through the paths named in its id,
and is compared with the oracle's FGMRES on the same system and options:
the solution within 1e-8 at rtol 1e-12, the iteration count within
two, and the true residual recomputed on the host.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)


@pytest.fixture(scope="module")
def trs():
    from paper_1812_03952_gb300 import build as B
    B.build()
    from paper_1812_03952_gb300 import trs as T
    T.load()
    return T


# FRS decoupling with the FP ordering needs about 40 iterations on these
# high-contrast systems (shale lenses, sigma 2).
CASES = [
    # 39 iterations in one cycle of FGMRES(60): staged 8, 16, 32 vectors, then the multi-dot passes
    dict(id="restart60_staged_then_multidot", shape=(48, 32, 16), b=4, seed=12, restart=60, rtol=1e-12),
    # the same in FGMRES(30): the first cycle reaches 30 vectors, then a restart
    dict(id="restart30_staged", shape=(48, 32, 16), b=4, seed=12, restart=30, rtol=1e-12),
    # b = 5 on an odd row count, N odd: the register kernels up to 31 vectors, then (34 iterations)
    # the multi-dot and update passes
    dict(id="odd_n_register_then_multidot", shape=(45, 31, 15), b=5, seed=14, restart=60, rtol=1e-12),
]


@pytest.mark.parametrize("case", CASES, ids=[c["id"] for c in CASES])
def test_fgmres_orthogonalisation_paths(trs, oracle, synth, case):
    s = synth.small_system(*case["shape"], b=case["b"], seed=case["seed"], n_pairs=2, sigma=2.0, kvkh=0.1,
                           shale_frac=0.1)
    if case["id"].startswith("odd_n"):
        assert (s.n_rows * s.b) % 2 == 1
    else:
        assert (s.n_rows * s.b) % 2 == 0
    ds = trs.DeviceSystem(s)
    A = ds.assemble()
    Ao = oracle.assemble(s)
    opts = dict(decoupling="frs", stages="fp")
    M = trs.CPR(A, precision="fp64", **opts)
    x, res = trs.fgmres_solve(A, M, ds.rhs, rtol=case["rtol"], restart=case["restart"])
    ref = oracle.fgmres(Ao, oracle.CPR(Ao, **opts), s.rhs, rtol=case["rtol"], restart=case["restart"])
    assert res.status == trs.TRS_OK and ref.converged
    xg = x.cpu().numpy()
    assert np.linalg.norm(xg - ref.x) / np.linalg.norm(ref.x) <= 1e-8
    assert np.linalg.norm(s.rhs - oracle.spmv(Ao, xg)) / np.linalg.norm(s.rhs) <= 1.01 * case["rtol"]
    assert abs(res.stats["iters"] - ref.iters) <= 2
    if case["id"] != "restart30_staged":
        assert res.stats["iters"] > 32   # past 32 vectors: the multi-dot passes
