"""Pins of the oracle's thermal model (oracle/trs_thermal.c): the residual of
one Newton step of the water + heavy-oil model (Sec. "Mathematical Model",
Sec. "Numerical Methods") and its complex-step Jacobian.

What pins it, none of which restates its formulas:
  * the Jacobian against central differences of the residual, every column;
  * conservation: the flux terms cancel in pairs, so the sum of every cell's
    water, oil and energy residual is the change of the totals over dt minus
    what the wells put in;
  * a uniform state without gravity and wells has no flow: every cell's
    residual is its own accumulation change, and each block row of the
    Jacobian sums to that cell's accumulation derivative;
  * physical values the correlations must reproduce: the saturation pressure
    of water at 100 C and 200 C (steam tables: 101.42 and 1554.9 kPa) from the
    paper's K-value constants, the latent heat of water at 100 C (40.65
    kJ/gmol) from its heat-of-vaporisation constants, the Redlich-Kwong cubic
    and its ideal-gas limit, reference densities and porosity;
  * the relative-permeability tables of the paper at their nodes, and
    Stone's model II reducing to k_row without gas and to k_rog at connate
    water;
  * Newton's method on a small system converges quadratically with this
    Jacobian (the system-level consistency of J with R).
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla


@pytest.fixture(scope="module")
def thermal(oracle, synth):
    def make(nx=5, ny=4, nz=4, n_pairs=1, seed=11, gravity=9.80665, dt=1.0):
        s = synth.small_system(nx, ny, nz, 4, seed=seed, n_pairs=n_pairs, sigma=1.0)
        t = synth.thermal_state(s, seed + 100, dt=dt, gravity=gravity)
        return s, t, oracle.Thermal(s, t, synth.SWT, synth.SLT)
    return make


def _difference_column(th, u0, k, gas_free_sg):
    """Column k of dR/du by central differences; where the variable is S_g of
    a cell without gas (S_g = 0, the end of the liquid-gas table, a kink) by
    a forward difference into S_g > 0, the side whose slope the Jacobian
    takes."""
    if gas_free_sg:
        h = 1e-8
        up = u0.copy()
        up[k] += h
        return (th.residual(up) - th.residual(u0)) / h, 1e-5
    h = 1e-6 * max(1.0, abs(u0[k]))
    up, um = u0.copy(), u0.copy()
    up[k] += h
    um[k] -= h
    return (th.residual(up) - th.residual(um)) / (2.0 * h), 1e-6


def test_jacobian_matches_central_differences(thermal):
    s, t, th = thermal()
    J = th.jacobian().to_dense()
    u0 = t.u.copy()
    n = len(u0)
    scale = np.max(np.abs(J), axis=1)
    for k in range(n):
        c, v = divmod(k, 4)
        fd, tol = _difference_column(th, u0, k, c < s.n_cells and v == 2 and not t.gas[c])
        err = np.abs(J[:, k] - fd) / np.maximum(scale, 1e-300)
        assert err.max() <= tol, (c, v, float(err.max()))


def test_jacobian_without_gravity_and_with_gas_everywhere_matches_differences(thermal, synth, oracle):
    s, t, _ = thermal(nx=4, ny=3, nz=3, seed=17, gravity=0.0)
    n_c = s.n_cells
    u = t.u.reshape(-1, 4)
    u[:n_c, 2] = 0.21      # away from the table nodes (kinks of the interpolation)
    u[:n_c, 1] = 0.52
    u[:n_c, 3] = 190.0 + 10.0 * np.random.default_rng(3).random(n_c)
    t.gas[:] = 1
    th = oracle.Thermal(s, t, synth.SWT, synth.SLT)
    J = th.jacobian().to_dense()
    u0 = t.u.copy()
    scale = np.max(np.abs(J), axis=1)
    for k in range(len(u0)):
        fd, tol = _difference_column(th, u0, k, False)
        assert np.all(np.abs(J[:, k] - fd) <= tol * np.maximum(scale, 1e-300)), k


def test_conservation(thermal):
    s, t, th = thermal(nx=6, ny=5, nz=4, seed=13)
    R = th.residual().reshape(-1, 4)[:s.n_cells]
    dt = t.params["dt"]
    change = (th.totals(t.u) - th.totals(t.u_old)) / dt
    src = th.well_sources()
    for e in range(3):
        lhs = R[:, e].sum()
        rhs = change[e] - src[e]
        mag = np.abs(R[:, e]).sum() + abs(change[e]) + abs(src[e])
        assert abs(lhs - rhs) <= 1e-12 * mag, (e, lhs, rhs)


def test_uniform_state_has_no_flow(thermal, synth, oracle):
    s, t, _ = thermal(nx=5, ny=4, nz=3, n_pairs=0, seed=19, gravity=0.0)
    n_c = s.n_cells
    u = t.u.reshape(-1, 4)
    u[:] = (1800.0, 0.6, 0.0, 60.0)
    uo = t.u_old.reshape(-1, 4)
    uo[:] = (1795.0, 0.61, 0.0, 59.5)
    t.gas[:] = 0
    th = oracle.Thermal(s, t, synth.SWT, synth.SLT)
    R = th.residual().reshape(-1, 4)
    per_cell = (th.totals(t.u) - th.totals(t.u_old)) / t.params["dt"] / n_c
    for e in range(3):
        np.testing.assert_allclose(R[:, e], per_cell[e], rtol=1e-12)
    np.testing.assert_array_equal(R[:, 3], 0.0)
    A = th.jacobian()
    rows = A.row_of_block()
    sums = np.zeros((A.n, 4, 4))
    np.add.at(sums, rows, A.val)
    # every block row sums to the same accumulation derivative
    for c in range(1, n_c):
        np.testing.assert_allclose(sums[c], sums[0], rtol=1e-10, atol=1e-9 * np.abs(sums[0]).max())
    # ... which is d(accumulation)/du: the own block minus the flux parts
    eps = 1e-6
    for k in range(3):
        up = t.u.copy().reshape(-1, 4)
        up[:, k] += eps * max(1.0, abs(up[0, k]))
        d = (th.totals(up.reshape(-1)) - th.totals(t.u)) / (eps * max(1.0, abs(u[0, k]))) / t.params["dt"] / n_c
        np.testing.assert_allclose(sums[0][:3, k], d, rtol=1e-5)


def test_gas_constraint_rows(thermal):
    s, t, th = thermal(seed=23)
    A = th.jacobian()
    rows = A.row_of_block()
    for p in range(A.nnzb):
        i, j = rows[p], A.col[p]
        if i >= s.n_cells:
            continue
        if not t.gas[i]:
            expect = np.array([0, 0, 1, 0]) if i == j else np.zeros(4)
            np.testing.assert_array_equal(A.val[p][3], expect)
        elif i != j:
            np.testing.assert_array_equal(A.val[p][3], 0.0)


def test_injector_columns_closed_form(thermal):
    """Cell rows of an injector perforation: dR/dp_b = -WI_u (water) and
    -WI_u h_inj (energy), nothing else."""
    s, t, th = thermal(seed=29)
    A = th.jacobian()
    rows = A.row_of_block()
    n_c = s.n_cells
    for m in range(len(s.perf_cell)):
        w = s.perf_well[m]
        if t.well_type[w] != 0:
            continue
        c = s.perf_cell[m]
        p = np.nonzero((rows == c) & (A.col == n_c + w))[0][0]
        np.testing.assert_allclose(A.val[p][:, 0], [-t.wi[m], 0.0, -t.wi[m] * t.params["h_inj"], 0.0],
                                   rtol=1e-15)
        np.testing.assert_array_equal(A.val[p][:, 1:], 0.0)


def test_saturation_pressure_and_latent_heat(thermal):
    """The paper's K-value constants give the steam-table saturation pressure
    (K_W = 1 with S_w = 1, where the PER factor is 1 / (1 + eps)), and its
    heat-of-vaporisation constants the latent heat at 100 C."""
    s, t, th = thermal()
    eps = t.params["per_eps"]
    for T, p_table in ((100.0, 101.42), (200.0, 1554.9)):
        # K* p is independent of p for kv2 = kv3 = 0: solve K* (1 + eps) = 1 for p
        ks = th.props([1000.0, 1.0, 0.0, T])["K_star"]
        p_sat = ks * (1.0 + eps) * 1000.0
        assert abs(p_sat - p_table) <= 0.005 * p_table, (T, p_sat)
    pr = th.props([101.325, 1.0, 0.0, 100.0])
    latent = pr["H_g"] - pr["H_w"]
    assert abs(latent - 40.65) <= 0.01 * 40.65, latent
    assert th.props([500.0, 0.7, 0.0, t.params["T_ref"]])["H_g"] == 0.0
    assert th.props([500.0, 0.7, 0.0, t.params["T_ref"]])["H_o"] == 0.0


def test_redlich_kwong(oracle, thermal):
    assert oracle.rk_z(0.0, 0.0) == 1.0
    for A, B in ((0.01, 0.002), (0.1, 0.02), (0.3, 0.05)):
        z = oracle.rk_z(A, B)
        f = z ** 3 - z ** 2 + (A - B - B * B) * z - A * B
        assert abs(f) <= 1e-14
        roots = np.roots([1.0, -1.0, A - B - B * B, -A * B])
        assert abs(z - max(r.real for r in roots if abs(r.imag) < 1e-9)) <= 1e-12
    # near-ideal at low pressure: Z -> 1
    assert abs(oracle.rk_z(1e-6, 1e-7) - 1.0) < 1e-6
    # the model's whole (p, T) range, cold compressed water included, where
    # the cubic has one real (liquid-like) root below a positive local
    # minimum: Z is a root, and no real root lies above it
    P = thermal()[1].params
    TcK = P["tc_w"] + 273.15
    for p in (200.0, 500.0, 1000.0, 1915.35, 2000.0, 5000.0, 10000.0, 20000.0):
        for T in (5.0, 12.43, 25.0, 50.0, 100.0, 150.0, 200.0, 250.0, 300.0, 350.0):
            TK = T + 273.15
            A = 0.427480 * (p / P["pc_w"]) * (TcK / TK) ** 2.5
            B = 0.086640 * (p / P["pc_w"]) * (TcK / TK)
            c1, c0 = A - B - B * B, -A * B
            z = oracle.rk_z(A, B)
            assert abs(((z - 1.0) * z + c1) * z + c0) <= 1e-15 * max(1.0, abs(c1), abs(c0)), (p, T)
            real = [r.real for r in np.roots([1.0, -1.0, c1, c0]) if abs(r.imag) <= 1e-7]
            assert z >= max(real) - 1e-9, (p, T, z, real)
    # states where Newton's method started above every root cycles near the
    # local minimum instead of reaching the liquid-like root
    for p, T in ((3000.0, 64.0), (3000.0, 69.0), (3800.0, 88.0), (4700.0, 129.0), (5800.0, 148.0)):
        TK = T + 273.15
        A = 0.427480 * (p / P["pc_w"]) * (TcK / TK) ** 2.5
        B = 0.086640 * (p / P["pc_w"]) * (TcK / TK)
        z = oracle.rk_z(A, B)
        real = [r.real for r in np.roots([1.0, -1.0, A - B - B * B, -A * B]) if abs(r.imag) <= 1e-7]
        assert len(real) == 1 and abs(z - real[0]) <= 1e-12 * max(1.0, abs(z)), (p, T, z, real)
    # the single-real-root case met at 1915 kPa and 12.4 C
    A, B = 0.2868008466275823, 0.01704208436092397
    assert abs(oracle.rk_z(A, B) - 0.0195254201115644) <= 1e-13
    # saturated steam at 200 C: Z about 0.91 (steam tables: v = 0.1272 m^3/kg)
    s, t, th = thermal()
    rho_g = th.props([1554.9, 0.5, 0.3, 200.0])["rho_g"]
    z = 1554.9 / (rho_g * t.params["R_gas"] * 473.15)
    assert 0.88 <= z <= 0.96, z


def test_reference_values(thermal):
    s, t, th = thermal()
    P = t.params
    pr = th.props([P["p_ref"], 0.6, 0.0, P["T_ref"]])
    assert pr["rho_w"] == P["rho_w_ref"] and pr["rho_o"] == P["rho_o_ref"]
    assert pr["phi"] == P["phi_ref"]
    one = th.props([P["p_ref"], 1.0, 0.0, P["T_ref"]])
    assert abs(one["K_T"] - (P["phi_ref"] * P["kt_w"] + (1 - P["phi_ref"]) * P["kt_r"])) <= 1e-12 * one["K_T"]


def test_relative_permeability_tables_and_stone(thermal, synth):
    """Ratios at one (p, T) cancel density and viscosity: table nodes of the
    paper (Figs. rela-swt, rela-slt) and Stone II's reductions."""
    s, t, th = thermal()
    pt = lambda sw, sg: th.props([1500.0, sw, sg, 120.0])
    swt, slt = synth.SWT, synth.SLT
    # k_rw and k_row (= k_ro without gas) at nodes S_w = 0.6 and 0.8
    a, b = pt(0.60, 0.0), pt(0.80, 0.0)
    assert abs(a["lam_w"] / b["lam_w"] - 0.00861 / 0.07162) <= 1e-12
    assert abs(a["lam_o"] / b["lam_o"] - 0.15625 / 0.00625) <= 1e-9
    # at connate water S_w = 0.45, Stone II gives k_rog(S_l): node S_l = 0.8 (S_g = 0.2)
    c, d = pt(0.45, 0.2), pt(0.45, 0.0)
    assert abs(c["lam_o"] / d["lam_o"] - 0.12346 / 0.4) <= 1e-9
    # k_rg at node S_l = 0.7 (S_g = 0.3) against S_l = 0.55 (S_g = 0.45)
    e, f = pt(0.45, 0.3), pt(0.45, 0.45)
    assert abs(e["lam_g"] / f["lam_g"] - 0.06856 / 0.14202) <= 1e-12
    # midpoint of two nodes: linear interpolation
    g = pt(0.625, 0.0)
    assert abs(g["lam_w"] / a["lam_w"] - 0.5 * (0.00861 + 0.01768) / 0.00861) <= 1e-12
    assert swt.shape == (12, 3) and slt.shape == (19, 3)


def test_newton_converges_quadratically(thermal):
    """Newton's method with this Jacobian (direct sparse solves) on a small
    system converges quadratically.  The state u* is made an exact root by
    solving R(u) - R(u*) = 0, and Newton starts from u* plus a small seeded
    perturbation (S_g only where gas exists, so that no step crosses the
    table end at S_g = 0)."""
    s, t, th = thermal(nx=5, ny=4, nz=4, seed=31, dt=0.5)
    ustar = t.u.copy()
    R0 = th.residual(ustar)
    rng = np.random.default_rng(5)
    du = np.zeros((len(ustar) // 4, 4))
    n_c = s.n_cells
    du[:n_c, 0] = rng.normal(0.0, 0.05, n_c)
    du[:n_c, 1] = rng.normal(0.0, 5e-5, n_c)
    du[:n_c, 2] = np.where(t.gas == 1, rng.normal(0.0, 5e-5, n_c), 0.0)
    du[:n_c, 3] = rng.normal(0.0, 0.005, n_c)
    du[n_c:, 0] = rng.normal(0.0, 0.05, s.n_wells)
    u = ustar + du.reshape(-1)
    errs = []
    for it in range(6):
        errs.append(np.linalg.norm(u - ustar) / np.linalg.norm(ustar))
        if errs[-1] <= 1e-14:
            break
        J = th.jacobian(u).to_scipy().tocsc()
        u = u - spla.spsolve(J, th.residual(u) - R0)
    e = np.array(errs)
    assert e[-1] <= 1e-13, e
    # quadratic: e_{k+1} <= C e_k^2 with one C for every step above rounding
    ks = [k for k in range(len(e) - 1) if e[k + 1] > 1e-13]
    assert ks and all(e[k + 1] <= 1e4 * e[k] ** 2 for k in ks), e
