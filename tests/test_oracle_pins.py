"""Pins of the CPU oracle against what the paper and the mathematics fix.

Every check here is independent of the oracle's own code: closed forms,
invariants of the assembly, exact rational arithmetic, brute-force graph
searches, library routines (numpy / scipy) that compute the same quantity by a
different method, and special cases that reduce to a textbook result.  Each
is chosen so that a plausible slip (a dropped term, a wrong sign or index, a
transposed operand) fails at least one of them.
"""
from fractions import Fraction
from collections import deque

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spl


# ---------------------------------------------------------------- helpers
def tiny(synth, nx=4, ny=3, nz=2, b=3, seed=5, **kw):
    return synth.small_system(nx, ny, nz, b, seed=seed, **kw)


def uniform_state(sysm, u0):
    b = sysm.b
    u = np.zeros(sysm.n_unknowns)
    u[: sysm.n_cells * b] = np.tile(u0, sysm.n_cells)
    u[sysm.n_cells * b:: b] = u0[0]
    return u


def dense_of(A):
    return A.to_dense()


def laplacian_7pt(nx, ny, nz):
    n = nx * ny * nz
    rows, cols, vals = [], [], []
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                i = x + nx * (y + ny * z)
                for dx, dy, dz in ((0, 0, -1), (0, -1, 0), (-1, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1)):
                    X, Y, Z = x + dx, y + dy, z + dz
                    if 0 <= X < nx and 0 <= Y < ny and 0 <= Z < nz:
                        rows.append(i); cols.append(X + nx * (Y + ny * Z)); vals.append(-1.0)
                rows.append(i); cols.append(i); vals.append(6.0)
    A = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    A.sort_indices()
    return A


def csr_parts(A):
    A = sp.csr_matrix(A)
    A.sort_indices()
    return (A.shape[0], A.indptr.astype(np.int64), A.indices.astype(np.int32),
            A.data.astype(np.float64))


# ------------------------------------------------------------- assembly
def test_uniform_state_has_no_flux(oracle, synth):
    """(A u)_c = Acc_c u0 and (A u)_w = 0 for a uniform state: every face
    block is matched by its opposite on the diagonal (TPFA flux is a
    difference), and the well rate vanishes when p_bhp = p_cell."""
    for b in (1, 3, 4, 5):
        s = tiny(synth, 5, 4, 3, b, seed=b)
        A = oracle.assemble(s)
        u0 = np.random.default_rng(b).uniform(-1, 1, b)
        Au = oracle.spmv(A, uniform_state(s, u0))
        want = np.einsum("crs,s->cr", s.acc, u0).reshape(-1)
        np.testing.assert_allclose(Au[: s.n_cells * b], want, rtol=1e-12, atol=1e-12)
        wells = Au[s.n_cells * b:].reshape(-1, b)
        np.testing.assert_allclose(wells[:, 0], 0.0, atol=1e-12)


def test_homogeneous_transmissibility_is_k(oracle, synth):
    """Harmonic mean of equal permeabilities is the permeability itself:
    A_ij = -c_T k M_ij on x/y faces and -c_T (kv/kh) k M_ij on z faces."""
    s = tiny(synth, 3, 3, 3, 2, seed=1, n_pairs=0, kvkh=0.1)
    s.k[:] = 250.0
    A = oracle.assemble(s)
    rows = A.row_of_block()
    nx, ny = s.nx, s.ny
    for p in range(A.nnzb):
        i, j = rows[p], A.col[p]
        if i == j:
            continue
        d = {-nx * ny: 0, -nx: 1, -1: 2, 1: 3, nx: 4, nx * ny: 5}[j - i]
        scale = 0.1 if d in (0, 5) else 1.0
        np.testing.assert_allclose(A.val[p], -s.c_t * scale * 250.0 * s.M[i, d], rtol=1e-15)


def test_two_cell_harmonic_mean(oracle, synth):
    """Two cells along x: T = c_T * 2 k1 k2 / (k1 + k2), not the arithmetic mean."""
    s = synth.small_system(2, 1, 1, 2, seed=3, n_pairs=0)
    s.k[:] = [100.0, 400.0]
    A = oracle.assemble(s)
    T = 1e-3 * 2 * 100.0 * 400.0 / 500.0          # 0.16
    np.testing.assert_allclose(A.val[1], -T * s.M[0, 3], rtol=1e-15)  # row 0, col 1 (+x)
    np.testing.assert_allclose(A.val[2], -T * s.M[1, 2], rtol=1e-15)  # row 1, col 0 (-x)
    np.testing.assert_allclose(A.val[0], s.acc[0] + T * s.M[0, 3], rtol=1e-14)


def test_impermeable_faces_and_boundary(oracle, synth):
    """k = 0 on both sides gives T = 0; no block exists across the boundary
    (no-flow), so nnzb = n + 2 * (internal faces) + 2 * perforations."""
    s = tiny(synth, 4, 3, 2, 2, seed=2)
    s.k[:] = 0.0
    A = oracle.assemble(s)
    nx, ny, nz = s.nx, s.ny, s.nz
    faces = (nx - 1) * ny * nz + nx * (ny - 1) * nz + nx * ny * (nz - 1)
    assert A.nnzb == s.n_rows + 2 * faces + 2 * len(s.perf_cell)
    rows = A.row_of_block()
    cell_off = (rows < s.n_cells) & (A.col < s.n_cells) & (rows != A.col)
    assert np.all(A.val[cell_off] == 0.0)
    assert oracle.pattern_symmetric(A)


def test_well_rows(oracle, synth):
    """Fixed-rate well row: A_ww(0,0) = sum_m WI_m Lam_m, A_wc(0,0) = -WI_m Lam_m,
    identity on the padded entries; cell rows get -WI lam in the BHP column."""
    s = tiny(synth, 6, 4, 3, 4, seed=9, n_pairs=1)
    A = oracle.assemble(s)
    Ad = dense_of(A)
    b, nc = s.b, s.n_cells
    for w in range(s.n_wells):
        m = np.where(s.perf_well == w)[0]
        Lam = s.lam[m].sum(axis=1)
        r = (nc + w) * b
        np.testing.assert_allclose(Ad[r, r], np.sum(s.wi[m] * Lam), rtol=1e-14)
        np.testing.assert_allclose(Ad[r, s.perf_cell[m] * b], -s.wi[m] * Lam, rtol=1e-14)
        np.testing.assert_array_equal(Ad[r + 1: r + b, r + 1: r + b], np.eye(b - 1))
        for mm in m:
            c = s.perf_cell[mm]
            np.testing.assert_allclose(Ad[c * b: c * b + b, r], -s.wi[mm] * s.lam[mm], rtol=1e-14)


# ---------------------------------------------------------- Gauss-Jordan
def _frac_inverse(M):
    """Exact inverse by the adjugate (cofactor) formula in rationals."""
    n = len(M)

    def det(a):
        if len(a) == 1:
            return a[0][0]
        return sum((-1) ** j * a[0][j] * det([row[:j] + row[j + 1:] for row in a[1:]])
                   for j in range(len(a)))

    d = det(M)
    adj = [[(-1) ** (i + j) * det([r[:i] + r[i + 1:] for k, r in enumerate(M) if k != j])
            for j in range(n)] for i in range(n)]
    return [[adj[i][j] / d for j in range(n)] for i in range(n)]


def test_gj_inverse_exact_rational(oracle):
    """A 3x3 needing a row swap (zero leading entry), against the exact
    rational adjugate inverse."""
    M = [[Fraction(0), Fraction(2), Fraction(1)],
         [Fraction(3), Fraction(-1), Fraction(2)],
         [Fraction(1), Fraction(1), Fraction(4)]]
    exact = np.array([[float(v) for v in row] for row in _frac_inverse(M)])
    got = oracle.gj_inverse(np.array([[float(v) for v in row] for row in M]))
    np.testing.assert_allclose(got, exact, rtol=1e-15, atol=1e-16)


def test_gj_inverse_random_and_singular(oracle):
    rng = np.random.default_rng(0)
    for b in (1, 2, 4, 5, 8):
        D = rng.standard_normal((b, b)) + b * np.eye(b)
        np.testing.assert_allclose(oracle.gj_inverse(D) @ D, np.eye(b), atol=1e-13)
    with pytest.raises(oracle.OracleError):
        oracle.gj_inverse(np.array([[1.0, 2.0], [2.0, 4.0]]))


# ------------------------------------------------------------ decoupling
def test_abf_decoupling(oracle, synth):
    """Eq. decoupled-abf: D_i Ã_ij = A_ij, Ã_ii = I exactly, and the
    decoupled system has the same solution (D^-1 A) x = D^-1 b."""
    s = tiny(synth, 4, 4, 3, 4, seed=4)
    A = oracle.assemble(s)
    vt, dinv = oracle.decouple(A)
    rows = A.row_of_block()
    for p in range(A.nnzb):
        i = rows[p]
        if A.col[p] == i:
            np.testing.assert_array_equal(vt[p], np.eye(s.b))
        else:
            D = np.linalg.inv(dinv[i])
            scale = np.abs(A.val[p]).max() + 1e-300
            assert np.abs(D @ vt[p] - A.val[p]).max() <= 1e-12 * scale * np.linalg.cond(D)
    At = oracle.BSR(A.n, A.b, A.rp, A.col, vt).to_dense()
    x = np.linalg.solve(dense_of(A), s.rhs)
    f = np.concatenate([dinv[i] @ s.rhs[i * s.b:(i + 1) * s.b] for i in range(A.n)])
    np.testing.assert_allclose(At @ x, f, rtol=1e-9, atol=1e-9)


def test_frs_then_abf_equals_abf(oracle, synth):
    """Two-stage FRS+ABF (add all rows into the pressure row, then ABF)
    gives the same decoupled matrix as ABF alone in exact arithmetic
    (Sec. Decoupling Methods): (F A_ii)^-1 F A_ij = A_ii^-1 A_ij."""
    s = tiny(synth, 3, 3, 2, 3, seed=6)
    A = oracle.assemble(s)
    vt, _ = oracle.decouple(A)
    F = np.eye(s.b)
    F[0, :] = 1.0
    A2 = oracle.BSR(A.n, A.b, A.rp, A.col, np.einsum("rs,pst->prt", F, A.val).copy())
    vt2, _ = oracle.decouple(A2)
    np.testing.assert_allclose(vt2, vt, rtol=1e-9, atol=1e-11)


@pytest.mark.parametrize("mode", ["none", "frs", "frs+abf"])
def test_decoupling_modes(oracle, synth, mode):
    """Sec. Decoupling Methods: Ã_ij = D_i^-1 A_ij for every stored block with
    D_i^-1 = I (none), R = ones in the first row and on the diagonal (FRS,
    Eq. decoupled-frs: all rows added into the pressure row), or
    (R A_ii)^-1 R (FRS then ABF), which equals A_ii^-1 and leaves Ã_ii = I."""
    s = tiny(synth, 4, 3, 3, 4, seed=9)
    A = oracle.assemble(s)
    vt, dinv = oracle.decouple(A, mode)
    b = s.b
    R = np.eye(b)
    R[0, :] = 1.0
    rows = A.row_of_block()
    if mode == "none":
        np.testing.assert_array_equal(vt, A.val)
        np.testing.assert_array_equal(dinv, np.broadcast_to(np.eye(b), dinv.shape))
    elif mode == "frs":
        np.testing.assert_array_equal(dinv, np.broadcast_to(R, dinv.shape))
        # the pressure row is the column sum; the other rows are untouched
        np.testing.assert_array_equal(vt[:, 1:, :], A.val[:, 1:, :])
        np.testing.assert_allclose(vt[:, 0, :], A.val.sum(axis=1), rtol=1e-15,
                                   atol=1e-15 * np.abs(A.val).max())
    else:
        vt_abf, dinv_abf = oracle.decouple(A, "abf")
        diag = A.col == rows
        np.testing.assert_array_equal(vt[diag], np.broadcast_to(np.eye(b), vt[diag].shape))
        np.testing.assert_allclose(vt, vt_abf, rtol=1e-9, atol=1e-11)
        np.testing.assert_allclose(dinv, dinv_abf, rtol=1e-9, atol=1e-11 * np.abs(dinv_abf).max())
    if mode != "frs+abf":
        np.testing.assert_allclose(np.einsum("prs,pst->prt", dinv[rows], A.val), vt, rtol=1e-14,
                                   atol=1e-15 * np.abs(A.val).max())


def test_pressure_matrix_scalar_case(oracle, synth):
    """For b = 1 the pressure matrix is the Jacobi-scaled matrix D^-1 A."""
    s = tiny(synth, 4, 3, 3, 1, seed=8)
    A = oracle.assemble(s)
    vt, dinv = oracle.decouple(A)
    ap = oracle.pressure_matrix(A, vt)
    Ad = dense_of(A)
    Ap = sp.csr_matrix((ap, A.col, A.rp), shape=(A.n, A.n)).toarray()
    np.testing.assert_allclose(Ap, Ad / np.diag(Ad)[:, None], rtol=1e-15)


# --------------------------------------------------------------- AMG
def _strong_bruteforce(Ad, theta):
    n = Ad.shape[0]
    S = np.zeros((n, n), bool)
    for i in range(n):
        for j in range(n):
            if i == j or (Ad[i, j] == 0 and Ad[j, i] == 0 and True):
                continue
            s = max(abs(Ad[i, j]), abs(Ad[j, i]))
            S[i, j] = s > 0 and s >= theta * np.sqrt(abs(Ad[i, i] * Ad[j, j]))
    return S


def test_strength_graph(oracle):
    A = sp.csr_matrix(np.array([[4.0, -1.0, 0.0, -0.1],
                                [-1.0, 4.0, -2.0, 0.0],
                                [0.0, -0.2, 1.0, 0.0],
                                [-0.1, 0.0, 0.0, 4.0]]))
    A.eliminate_zeros()
    n, rp, col, val = csr_parts(A)
    srp, scol = oracle.strength(n, rp, col, val, 0.25)
    S = _strong_bruteforce(A.toarray(), 0.25)
    got = np.zeros_like(S)
    for i in range(n):
        got[i, scol[srp[i]:srp[i + 1]]] = True
    np.testing.assert_array_equal(got, S)
    # 1 -- 2: max(2, 0.2) = 2 >= 0.25 * sqrt(4) = 0.5 strong; 0 -- 3 weak
    assert got[1, 2] and got[2, 1] and not got[0, 3]


def _bfs_dist(adj, src, limit):
    dist = {src: 0}
    q = deque([src])
    while q:
        u = q.popleft()
        if dist[u] == limit:
            continue
        for v in adj[u]:
            if v not in dist:
                dist[v] = dist[u] + 1
                q.append(v)
    return dist


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_mis2_is_distance2_independent_and_maximal(oracle, seed):
    """No two IN nodes within distance 2; every OUT node with an edge is
    within distance 2 of an IN node (brute-force BFS)."""
    rng = np.random.default_rng(seed)
    n = 300
    R = sp.random(n, n, density=0.012, random_state=seed, format="csr")
    R = (R + R.T).tocsr()
    R.setdiag(0)
    R.eliminate_zeros()
    R.sort_indices()
    srp, scol = R.indptr.astype(np.int64), R.indices.astype(np.int32)
    state, rounds = oracle.mis2(n, srp, scol, int(rng.integers(1, 2**31)))
    adj = [scol[srp[i]:srp[i + 1]].tolist() for i in range(n)]
    IN = set(np.where(state == 2)[0].tolist())
    assert rounds >= 1 and len(IN) > 0
    for u in IN:
        d = _bfs_dist(adj, u, 2)
        assert not (set(d) - {u}) & IN
    for v in range(n):
        if adj[v] and v not in IN:
            assert set(_bfs_dist(adj, v, 2)) & IN
        if not adj[v]:
            assert state[v] == 0


def test_aggregation_partition_and_galerkin(oracle, synth):
    """Aggregates partition the nodes with strong neighbours, each root sits
    in its own aggregate numbered by root order, and A_c = P^T A P equals the
    scipy sparse triple product (row sums aggregate exactly)."""
    s = tiny(synth, 8, 7, 5, 4, seed=12)
    A = oracle.assemble(s)
    vt, _ = oracle.decouple(A)
    ap = oracle.pressure_matrix(A, vt)
    n = A.n
    srp, scol = oracle.strength(n, A.rp, A.col, ap, 0.25)
    state, _ = oracle.mis2(n, srp, scol, 77)
    agg, n_agg = oracle.aggregate(n, A.rp, A.col, ap, srp, scol, state)
    has_strong = np.diff(srp) > 0
    assert np.all(agg[has_strong] >= 0) and np.all(agg[~has_strong] == -1)
    roots = np.where(state == 2)[0]
    np.testing.assert_array_equal(agg[roots], np.arange(n_agg))
    assert set(np.unique(agg[agg >= 0]).tolist()) == set(range(n_agg))
    crp, ccol, cval = oracle.galerkin(n, A.rp, A.col, ap, agg, n_agg)
    sel = agg >= 0
    P = sp.csr_matrix((np.ones(sel.sum()), (np.where(sel)[0], agg[sel])), shape=(n, n_agg))
    Ap = sp.csr_matrix((ap, A.col, A.rp), shape=(n, n))
    Ac_ref = (P.T @ Ap @ P).toarray()
    Ac = sp.csr_matrix((cval, ccol, crp), shape=(n_agg, n_agg)).toarray()
    np.testing.assert_allclose(Ac, Ac_ref, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(Ac.sum(1), (P.T @ (Ap @ P)).toarray().sum(1), rtol=1e-12)


def test_gershgorin_bounds_laplacian_spectrum(oracle):
    """For the 7-point Dirichlet Laplacian, max_i sum_j |a_ij| / a_ii = 2 and
    it bounds the analytic lambda_max of D^-1 A = (1/6) sum_d 2(1 - cos(pi n_d/(n_d+1)))."""
    nx, ny, nz = 7, 6, 5
    n, rp, col, val = csr_parts(laplacian_7pt(nx, ny, nz))
    lam = oracle.gershgorin(n, rp, col, val)
    analytic = sum(2 * (1 - np.cos(np.pi * m / (m + 1))) for m in (nx, ny, nz)) / 6
    assert lam == 2.0 and lam >= analytic


def test_chebyshev_matches_polynomial_closed_form(oracle):
    """Degree-k Chebyshev smoothing from e = 0 leaves the error
    p_k(D^-1 A) (A^-1 r), p_k(t) = T_k((theta - t)/delta) / T_k(theta/delta),
    evaluated here on the eigen-decomposition of the 1-D Laplacian."""
    n = 40
    A = sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1]).tocsr()
    nn, rp, col, val = csr_parts(A)
    lam = 2.0                                     # Gershgorin bound of D^-1 A
    r = np.random.default_rng(3).standard_normal(n)
    Ad = A.toarray()
    w, Q = np.linalg.eigh(Ad / 2.0)               # D^-1 A = A / 2 is symmetric here
    x = np.linalg.solve(Ad, r)
    a, bnd = 0.3 * lam, lam
    th, de = (bnd + a) / 2, (bnd - a) / 2
    for k in (1, 2, 3, 4):
        e = oracle.chebyshev(nn, rp, col, val, lam, k, r)
        Tk = np.polynomial.chebyshev.Chebyshev.basis(k)
        p = Tk((th - w) / de) / Tk(th / de)
        want = x - Q @ (p * (Q.T @ x))
        np.testing.assert_allclose(e, want, rtol=1e-10, atol=1e-12)


def test_dense_lu(oracle):
    rng = np.random.default_rng(4)
    A = rng.standard_normal((50, 50))
    A[0, 0] = 0.0                                  # forces a pivot
    bvec = rng.standard_normal(50)
    np.testing.assert_allclose(oracle.dense_lu_solve(A, bvec), np.linalg.solve(A, bvec),
                               rtol=1e-10, atol=1e-12)


def test_amg_single_level_is_exact_and_vcycle_contracts(oracle):
    Lp = laplacian_7pt(12, 10, 8) + sp.eye(960) * 0.01
    n, rp, col, val = csr_parts(Lp)
    r = np.random.default_rng(1).standard_normal(n)
    one = oracle.AMG(n, rp, col, val, coarse_max=2000)
    assert one.n_levels == 1
    np.testing.assert_allclose(Lp @ one.vcycle(r), r, rtol=1e-11, atol=1e-11)
    multi = oracle.AMG(n, rp, col, val, coarse_max=50)
    assert multi.n_levels >= 2
    e = multi.vcycle(r)
    assert np.linalg.norm(r - Lp @ e) < 0.5 * np.linalg.norm(r)


# ------------------------------------------------------------ colouring / ILU
def test_colouring_valid(oracle, synth):
    s = tiny(synth, 9, 8, 4, 2, seed=13, n_pairs=2)
    A = oracle.assemble(s)
    colour, nc = oracle.colour_jp(A, 99)
    rows = A.row_of_block()
    off = rows != A.col
    assert np.all(colour[rows[off]] != colour[A.col[off]])
    assert colour.min() == 0 and colour.max() == nc - 1 and nc <= 12


def _ilu_dense_factors(A, F, colour):
    n, b = A.n, A.b
    order = np.lexsort((np.arange(n), colour))
    pos = np.empty(n, int)
    pos[order] = np.arange(n)
    N = n * b
    L, U = np.eye(N), np.zeros((N, N))
    rows = A.row_of_block()
    for p in range(A.nnzb):
        i, j = rows[p], A.col[p]
        blk = (slice(i * b, i * b + b), slice(j * b, j * b + b))
        if i == j:
            U[blk] = np.linalg.inv(F[p])
        elif pos[j] < pos[i]:
            L[blk] = F[p]
        else:
            U[blk] = F[p]
    return L, U


def test_bilu0_defining_identity(oracle, synth):
    """(L U)_ij = Ã_ij on every stored block (ILU(0) definition), and the
    triangular solves invert L U exactly."""
    s = tiny(synth, 6, 5, 4, 3, seed=14, n_pairs=2)
    A = oracle.assemble(s)
    vt, _ = oracle.decouple(A)
    colour, _ = oracle.colour_jp(A, 5)
    ilu = oracle.BILU0(A, vt, colour)
    L, U = _ilu_dense_factors(A, ilu.factors(), colour)
    LU = L @ U
    At = oracle.BSR(A.n, A.b, A.rp, A.col, vt).to_dense()
    pat = np.zeros_like(At, dtype=bool)
    rows = A.row_of_block()
    for p in range(A.nnzb):
        i, j = rows[p], A.col[p]
        pat[i * A.b:(i + 1) * A.b, j * A.b:(j + 1) * A.b] = True
    assert np.abs((LU - At)[pat]).max() < 1e-11
    r = np.random.default_rng(0).standard_normal(A.n * A.b)
    np.testing.assert_allclose(LU @ ilu.solve(r), r, rtol=1e-9, atol=1e-9)


def test_bilu0_block_diagonal_is_exact(oracle, synth):
    s = tiny(synth, 4, 3, 2, 3, seed=15, n_pairs=0)
    s.k[:] = 0.0                                   # no flux => block diagonal
    A = oracle.assemble(s)
    vt, _ = oracle.decouple(A)
    colour, _ = oracle.colour_jp(A, 1)
    r = np.random.default_rng(1).standard_normal(A.n * A.b)
    np.testing.assert_allclose(oracle.BILU0(A, vt, colour).solve(r), r, rtol=1e-15)


# ------------------------------------------------------------ block ILU(1)
def _graph(A):
    G = np.zeros((A.n, A.n), bool)
    G[A.row_of_block(), A.col] = True
    np.fill_diagonal(G, False)
    return G


def test_colour_geo_is_distance2(oracle, synth):
    """The order of block ILU(1): cells two or fewer cell-to-cell steps
    apart never share a colour (7 colours), the other rows (wells) take
    colours from 7 on and no two of them within two steps share one."""
    s = tiny(synth, 9, 8, 5, 4, seed=16, n_pairs=2)
    A = oracle.assemble(s)
    colour, ncol = oracle.colour_geo(A, (s.nx, s.ny, s.nz))
    nc = s.nx * s.ny * s.nz
    G = _graph(A)
    Gi = G.astype(int)
    Gc = Gi[:nc, :nc]
    d2 = (Gc + Gc @ Gc) > 0
    np.fill_diagonal(d2, False)
    a, c = np.nonzero(d2)
    assert np.all(colour[a] != colour[c])
    assert sorted(set(colour[:nc].tolist())) == list(range(7))
    w = np.arange(nc, A.n)
    assert len(w) == 4 and np.all(colour[w] >= 7)
    dw = ((Gi + Gi @ Gi) > 0)[np.ix_(w, w)]
    np.fill_diagonal(dw, False)
    a, c = np.nonzero(dw)
    assert np.all(colour[w][a] != colour[w][c])
    assert ncol == colour.max() + 1


def _level_of_fill(A, colour, p):
    """The symbolic phase of ILU(p) by Gaussian elimination on a dense level
    matrix in the colour-major order (Saad, Iterative Methods for Sparse
    Linear Systems, Sec. 10.3.3): lev = 0 on the pattern, infinite
    elsewhere; for every row i and earlier k with lev_ik <= p,
    lev_ij = min(lev_ij, lev_ik + lev_kj + 1); entries above p dropped."""
    n = A.n
    order = np.lexsort((np.arange(n), colour))
    P = np.zeros((n, n), bool)
    P[A.row_of_block(), A.col] = True
    lev = np.where(P[np.ix_(order, order)], 0.0, np.inf)
    for i in range(n):
        for k in range(i):
            if lev[i, k] <= p:
                lev[i, k + 1:] = np.minimum(lev[i, k + 1:], lev[i, k] + lev[k, k + 1:] + 1)
        lev[i, lev[i] > p] = np.inf
    out = np.zeros((n, n), bool)
    out[np.ix_(order, order)] = np.isfinite(lev)
    return out


def _pattern_dense(n, rp, col):
    P = np.zeros((n, n), bool)
    P[np.repeat(np.arange(n), np.diff(rp)), col] = True
    return P


def test_bilu1_pattern_is_level_of_fill_one(oracle, synth):
    s = tiny(synth, 7, 6, 4, 3, seed=19, n_pairs=2)
    A = oracle.assemble(s)
    vt, _ = oracle.decouple(A)
    colour, _ = oracle.colour_geo(A, (s.nx, s.ny, s.nz))
    ilu = oracle.BILU0(A, vt, colour, level=1)
    rp, col = ilu.pattern()
    P1 = _pattern_dense(A.n, rp, col)
    np.testing.assert_array_equal(P1, _level_of_fill(A, colour, 1))
    assert P1.sum() > 1.5 * A.nnzb                      # level-1 fill is present
    np.testing.assert_array_equal(_pattern_dense(A.n, A.rp, A.col), _level_of_fill(A, colour, 0))
    assert all(np.all(np.diff(col[rp[i]:rp[i + 1]]) > 0) for i in range(A.n))
    # rows of one colour stay uncoupled in the factor pattern
    a, c = np.nonzero(P1 & ~np.eye(A.n, dtype=bool))
    assert np.all(colour[a] != colour[c])


def _ilu_dense_from_pattern(n, b, rp, col, F, colour):
    order = np.lexsort((np.arange(n), colour))
    pos = np.empty(n, int)
    pos[order] = np.arange(n)
    L, U = np.eye(n * b), np.zeros((n * b, n * b))
    rows = np.repeat(np.arange(n), np.diff(rp))
    for p in range(len(col)):
        i, j = rows[p], col[p]
        blk = (slice(i * b, i * b + b), slice(j * b, j * b + b))
        if i == j:
            U[blk] = np.linalg.inv(F[p])
        elif pos[j] < pos[i]:
            L[blk] = F[p]
        else:
            U[blk] = F[p]
    return L, U


def test_bilu1_defining_identity(oracle, synth):
    """(L U)_ij = Ã_ij on every block of the level-1 pattern, Ã_ij = 0 on the
    fill blocks, which ILU(0) leaves wrong; the sweeps invert L U."""
    s = tiny(synth, 7, 5, 4, 3, seed=20, n_pairs=2)
    A = oracle.assemble(s)
    vt, _ = oracle.decouple(A)
    colour, _ = oracle.colour_geo(A, (s.nx, s.ny, s.nz))
    ilu = oracle.BILU0(A, vt, colour, level=1)
    rp, col = ilu.pattern()
    L, U = _ilu_dense_from_pattern(A.n, A.b, rp, col, ilu.factors(), colour)
    LU = L @ U
    At = oracle.BSR(A.n, A.b, A.rp, A.col, vt).to_dense()
    blk = np.ones((A.b, A.b), bool)
    P1 = np.kron(_pattern_dense(A.n, rp, col), blk)
    fill = P1 & ~np.kron(_pattern_dense(A.n, A.rp, A.col), blk)
    assert np.abs((LU - At)[P1]).max() < 1e-11
    ilu0 = oracle.BILU0(A, vt, colour, level=0)
    L0, U0 = _ilu_dense_from_pattern(A.n, A.b, A.rp, A.col, ilu0.factors(), colour)
    assert np.abs((L0 @ U0 - At)[fill]).max() > 1e-3
    r = np.random.default_rng(5).standard_normal(A.n * A.b)
    np.testing.assert_allclose(LU @ ilu.solve(r), r, rtol=1e-9, atol=1e-9)


def test_cpr_ilu1_options_and_convergence(oracle, synth):
    s = tiny(synth, 10, 9, 5, 4, seed=21, n_pairs=2)
    A = oracle.assemble(s)
    grid = (s.nx, s.ny, s.nz)
    c1 = oracle.CPR(A, ilu_fill=1, grid=grid)
    assert c1.info()[1] == 8                             # 7 cell colours + the wells
    np.testing.assert_array_equal(c1.colours(), oracle.colour_geo(A, grid)[0])
    r1 = oracle.fgmres(A, c1, s.rhs, rtol=1e-10)
    r0 = oracle.fgmres(A, oracle.CPR(A), s.rhs, rtol=1e-10)
    assert r1.converged and r1.true_relres <= 1e-10 and r1.iters < r0.iters
    x = np.linalg.solve(A.to_dense(), s.rhs)
    assert np.linalg.norm(r1.x - x) / np.linalg.norm(x) < 1e-8
    for bad in (dict(ilu_fill=2, grid=grid), dict(ilu_fill=1),
                dict(ilu_fill=1, grid=(s.nx * s.ny * s.nz, 1, 1))):
        with pytest.raises(oracle.OracleError):
            oracle.CPR(A, **bad)


def test_cpr_ilu1_error_propagation(oracle, synth):
    """CPR-FPF with F = ILU(1)(Ã)^-1: I - B Ã = (I - FÃ)(I - PÃ)(I - FÃ)."""
    s = tiny(synth, 7, 3, 3, 3, seed=22, n_pairs=1)
    A = oracle.assemble(s)
    cpr = oracle.CPR(A, coarse_max=8, ilu_fill=1, grid=(s.nx, s.ny, s.nz))
    vt, dinv = cpr.decoupled()
    n, b = A.n, A.b
    N = n * b
    At = oracle.BSR(n, b, A.rp, A.col, vt).to_dense()
    ilu = oracle.BILU0(A, vt, cpr.colours(), level=1)
    I = np.eye(N)
    Fm = np.column_stack([ilu.solve(I[:, k]) for k in range(N)])
    Pp = np.column_stack([cpr.amg.vcycle(np.eye(n)[:, k]) for k in range(n)])
    Pm = np.zeros((N, N))
    Pm[np.ix_(np.arange(n) * b, np.arange(n) * b)] = Pp
    EF, EP = I - Fm @ At, I - Pm @ At
    B = (I - EF @ EP @ EF) @ np.linalg.inv(At)
    v = np.random.default_rng(25).standard_normal(N)
    f = np.einsum("irs,is->ir", dinv, v.reshape(n, b)).reshape(-1)
    want = B @ f
    np.testing.assert_allclose(cpr.apply(v), want, rtol=0, atol=1e-9 * np.abs(want).max())


# ------------------------------------------------------------------ CPR
def test_cpr_identity_when_no_flux(oracle, synth):
    """With k = 0 and no wells, Ã = I and CPR(Ã)^-1 = I, so M^-1 v = D^-1 v."""
    s = tiny(synth, 4, 4, 2, 4, seed=16, n_pairs=0)
    s.k[:] = 0.0
    A = oracle.assemble(s)
    cpr = oracle.CPR(A)
    v = np.random.default_rng(2).standard_normal(A.n * A.b)
    _, dinv = cpr.decoupled()
    want = np.einsum("irs,is->ir", dinv, v.reshape(A.n, A.b)).reshape(-1)
    np.testing.assert_allclose(cpr.apply(v), want, rtol=1e-14)
    res = oracle.fgmres(A, cpr, s.rhs, rtol=1e-12)
    assert res.iters == 1 and res.converged


def test_cpr_right_preconditioner_identity(oracle, synth):
    """M^-1 (A w) = CPR(Ã)^-1 (Ã w), since D^-1 A = Ã (decoupling as a right
    factor)."""
    s = tiny(synth, 5, 4, 3, 3, seed=17)
    A = oracle.assemble(s)
    cpr = oracle.CPR(A)
    vt, dinv = cpr.decoupled()
    w = np.random.default_rng(3).standard_normal(A.n * A.b)
    Aw = oracle.spmv(A, w)
    Atw = oracle.spmv(oracle.BSR(A.n, A.b, A.rp, A.col, vt), w)
    # CPR(Ã)^-1 u with u = D^-1 (D u):
    Du = np.einsum("irs,is->ir", np.linalg.inv(dinv), Atw.reshape(A.n, A.b)).reshape(-1)
    np.testing.assert_allclose(cpr.apply(Aw), cpr.apply(Du), rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("decoupling", ["abf", "none", "frs"])
@pytest.mark.parametrize("stages", ["fpf", "fp", "pf"])
def test_cpr_stage_error_propagation(oracle, synth, stages, decoupling):
    """A multiplicative combination of stages has the product of the stage
    error operators as its error operator.  With F = ILU(0)(Ã)^-1 and
    P = Pi_p AMG(A_PP)^-1 Pi_r as dense operators, the preconditioner B of
    CPR(Ã) satisfies I - B Ã = (I - FÃ)(I - PÃ)(I - FÃ) for FPF,
    (I - PÃ)(I - FÃ) for FP (F first) and (I - FÃ)(I - PÃ) for PF."""
    s = tiny(synth, 4, 3, 3, 3, seed=23, n_pairs=1)
    A = oracle.assemble(s)
    cpr = oracle.CPR(A, stages=stages, decoupling=decoupling, coarse_max=8)
    vt, dinv = cpr.decoupled()
    n, b = A.n, A.b
    N = n * b
    At = oracle.BSR(n, b, A.rp, A.col, vt).to_dense()
    ilu = oracle.BILU0(A, vt, cpr.colours())
    I = np.eye(N)
    Fm = np.column_stack([ilu.solve(I[:, k]) for k in range(N)])
    Pp = np.column_stack([cpr.amg.vcycle(np.eye(n)[:, k]) for k in range(n)])
    Pm = np.zeros((N, N))
    Pm[np.ix_(np.arange(n) * b, np.arange(n) * b)] = Pp
    EF, EP = I - Fm @ At, I - Pm @ At
    E = {"fpf": EF @ EP @ EF, "fp": EP @ EF, "pf": EF @ EP}[stages]
    B = (I - E) @ np.linalg.inv(At)
    v = np.random.default_rng(24).standard_normal(N)
    f = np.einsum("irs,is->ir", dinv, v.reshape(n, b)).reshape(-1)
    want = B @ f
    np.testing.assert_allclose(cpr.apply(v), want, rtol=0, atol=1e-9 * np.abs(want).max())


def test_cpr_scalar_reduces_to_ilu_plus_amg(oracle, synth):
    """b = 1 and no wells: CPR-FPF is ILU(0), residual, AMG on D^-1 A, residual, ILU(0)."""
    s = tiny(synth, 6, 5, 4, 1, seed=18, n_pairs=0)
    A = oracle.assemble(s)
    cpr = oracle.CPR(A, coarse_max=30)
    vt, dinv = cpr.decoupled()
    At = oracle.BSR(A.n, 1, A.rp, A.col, vt)
    ilu = oracle.BILU0(A, vt, cpr.colours())
    amg = cpr.amg
    v = np.random.default_rng(4).standard_normal(A.n)
    f = dinv.reshape(-1) * v
    y = ilu.solve(f)
    y = y + amg.vcycle(f - oracle.spmv(At, y))
    z = y + ilu.solve(f - oracle.spmv(At, y))
    np.testing.assert_allclose(cpr.apply(v), z, rtol=1e-13, atol=1e-14)


# --------------------------------------------------------------- FGMRES
@pytest.mark.parametrize("shape", [(2, 2, 2, 4), (4, 3, 2, 4), (5, 4, 3, 5), (8, 8, 2, 4)])
def test_fgmres_matches_direct_solve(oracle, synth, shape):
    nx, ny, nz, b = shape
    s = synth.small_system(nx, ny, nz, b, seed=sum(shape), n_pairs=1 if nz > 1 else 0)
    A = oracle.assemble(s)
    res = oracle.fgmres(A, oracle.CPR(A), s.rhs, rtol=1e-10)
    As = A.to_scipy().tocsc()
    x = spl.spsolve(As, s.rhs)
    cond = np.linalg.cond(As.toarray())
    assert res.converged and res.true_relres <= 1e-10
    assert np.linalg.norm(res.x - x) / np.linalg.norm(x) <= max(1e-12, cond * 1e-10)
    h = res.history
    assert np.all(np.diff(h) <= 1e-12 * h[0])     # minimal-residual: never increases


def test_fgmres_small_system_exact_in_n_steps(oracle, synth):
    """N <= 30 unknowns: exact (to rounding) within N Arnoldi steps of one cycle."""
    s = synth.small_system(3, 2, 2, 2, seed=3, n_pairs=0)
    A = oracle.assemble(s)
    N = A.n * A.b
    assert N <= 30
    res = oracle.fgmres(A, oracle.CPR(A), s.rhs, rtol=1e-13, restart=30)
    assert res.converged and res.iters <= N


def test_fgmres_config0(oracle, synth):
    s = synth.config(0)
    A = oracle.assemble(s)
    res = oracle.fgmres(A, oracle.CPR(A), s.rhs, rtol=1e-10)
    x = spl.spsolve(A.to_scipy().tocsc(), s.rhs)
    assert res.converged
    assert np.linalg.norm(res.x - x) / np.linalg.norm(x) < 1e-8


# --------------------------------------------------------------- BiCGSTAB
@pytest.mark.parametrize("shape", [(2, 2, 2, 4), (5, 4, 3, 5), (8, 8, 2, 4)])
def test_bicgstab_matches_direct_solve(oracle, synth, shape):
    nx, ny, nz, b = shape
    s = synth.small_system(nx, ny, nz, b, seed=sum(shape) + 1, n_pairs=1 if nz > 1 else 0)
    A = oracle.assemble(s)
    res = oracle.bicgstab(A, oracle.CPR(A), s.rhs, rtol=1e-10)
    As = A.to_scipy().tocsc()
    x = spl.spsolve(As, s.rhs)
    cond = np.linalg.cond(As.toarray())
    assert res.converged and res.true_relres <= 1e-10
    assert np.linalg.norm(res.x - x) / np.linalg.norm(x) <= max(1e-12, cond * 1e-10)


def test_bicgstab_iterates_match_scipy(oracle, synth):
    """The k-th iterate equals that of scipy's right-preconditioned BiCGSTAB
    (same van der Vorst recurrences, shadow residual r0) with M = CPR."""
    s = synth.small_system(7, 6, 4, 4, seed=29, n_pairs=1)
    A = oracle.assemble(s)
    cpr = oracle.CPR(A)
    As = A.to_scipy().tocsr()
    N = A.n * A.b
    Mop = spl.LinearOperator((N, N), matvec=lambda v: cpr.apply(np.asarray(v).reshape(-1)))
    for k in (1, 2, 3, 5):
        mine = oracle.bicgstab(A, cpr, s.rhs, rtol=1e-15, maxit=k)
        assert mine.iters == k and not mine.converged
        ref, _ = spl.bicgstab(As, s.rhs, rtol=1e-30, atol=0.0, maxiter=k, M=Mop)
        np.testing.assert_allclose(mine.x, ref, rtol=0, atol=1e-9 * np.abs(ref).max())
        # the reported true residual is that of the returned iterate
        tr = np.linalg.norm(s.rhs - As @ mine.x) / np.linalg.norm(s.rhs)
        np.testing.assert_allclose(mine.true_relres, tr, rtol=1e-10)


def test_bicgstab_exact_preconditioner_one_step(oracle, synth):
    """With M = A^-1 (no flux: CPR^-1 D^-1 = A^-1) the first half step gives s = 0."""
    s = tiny(synth, 4, 4, 2, 4, seed=16, n_pairs=0)
    s.k[:] = 0.0
    A = oracle.assemble(s)
    res = oracle.bicgstab(A, oracle.CPR(A), s.rhs, rtol=1e-12)
    assert res.iters == 1 and res.converged
    x = spl.spsolve(A.to_scipy().tocsc(), s.rhs)
    np.testing.assert_allclose(res.x, x, rtol=1e-12, atol=1e-14)


def test_bicgstab_zero_rhs(oracle, synth):
    s = tiny(synth, 3, 3, 2, 4, seed=5)
    A = oracle.assemble(s)
    res = oracle.bicgstab(A, oracle.CPR(A), np.zeros(A.n * A.b))
    assert res.converged and res.iters == 0 and np.all(res.x == 0)


# --------------------------------------------------------------- adjoint
def test_transpose_dot_product(oracle, synth):
    s = tiny(synth, 5, 4, 3, 4, seed=19)
    A = oracle.assemble(s)
    rng = np.random.default_rng(5)
    x, y = rng.standard_normal(A.n * A.b), rng.standard_normal(A.n * A.b)
    lhs = oracle.spmv(A, x) @ y
    rhs = x @ oracle.spmv(A, y, transpose=True)
    assert abs(lhs - rhs) <= 1e-13 * (abs(lhs) + 1)
    AT = oracle.transpose(A)
    np.testing.assert_allclose(oracle.spmv(AT, y), oracle.spmv(A, y, transpose=True), rtol=1e-13,
                               atol=1e-14)
    np.testing.assert_array_equal(dense_of(AT), dense_of(A).T)


def _loss(oracle, s, k):
    s2 = s
    old = s.k.copy()
    s2.k[:] = k
    A = oracle.assemble(s2)
    s.k[:] = old
    return A


def test_adjoint_gradient_against_finite_differences(oracle, synth):
    """dL/dtheta from A^T lambda = g, the outer product and the chain through
    the harmonic transmissibility, against central differences along seeded
    directions (difference-solve form: L+ - L- = g^T A+^-1 (A- - A+) x-)."""
    s = tiny(synth, 6, 5, 3, 4, seed=20)
    A = oracle.assemble(s)
    x = oracle.fgmres(A, oracle.CPR(A), s.rhs, rtol=1e-12).x
    g = oracle.well_cell_indicator(s)
    lam, dA, res = oracle.adjoint(A, g, x, rtol=1e-12)
    assert np.linalg.norm(oracle.spmv(A, lam, transpose=True) - g) <= 1e-11 * np.linalg.norm(g)
    dth = oracle.chain_theta(s, A, dA)
    theta = np.log(s.k)
    h = 1e-6
    for d in synth.seeded_directions(s.n_cells, 6, 123):
        Ap = _loss(oracle, s, np.exp(theta + h * d))
        Am = _loss(oracle, s, np.exp(theta - h * d))
        xm = spl.spsolve(Am.to_scipy().tocsc(), s.rhs)
        rhs = oracle.spmv(Am, xm) - oracle.spmv(Ap, xm)
        delta = spl.spsolve(Ap.to_scipy().tocsc(), rhs)
        fd = (g @ delta) / (2 * h)
        an = dth @ d
        assert abs(fd - an) <= 1e-5 * max(abs(fd), 1e-3 * np.abs(dth).sum() * 1e-3)


def test_adjoint_rhs_gradient_is_lambda(oracle, synth):
    """L is linear in b: L(b + e) - L(b) = g^T A^-1 e = lambda^T e exactly."""
    s = tiny(synth, 4, 4, 3, 3, seed=21)
    A = oracle.assemble(s)
    g = oracle.well_cell_indicator(s)
    lam, _, _ = oracle.adjoint(A, g, np.zeros(A.n * A.b), rtol=1e-12)
    Ad = dense_of(A)
    e = np.random.default_rng(6).standard_normal(A.n * A.b)
    np.testing.assert_allclose(g @ np.linalg.solve(Ad, e), lam @ e, rtol=1e-9)
