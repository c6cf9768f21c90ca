"""Seeded synthetic inputs shaped like the paper's SAGD thermal models.

This module only draws random numbers and lays out index data.  It holds none
of the solver's arithmetic: transmissibilities, the Jacobian assembly, the
decoupling and everything after it are computed independently by the CUDA
library and by the CPU oracle from the arrays produced here.

Shapes follow the paper's workloads: b unknowns per cell (pressure, component
moles, energy; Sec. "Mathematical Model", natural variables with p and T always
unknown), a 7-point two-point flux stencil on a structured grid (Sec.
"Numerical Methods", transmissibility paragraph) and horizontal SAGD well pairs
along x with the producer a few layers below the injector (Examples num-sagd,
num-light, num-11m).  Permeability is lognormal or channelised.

Conventions shared by both consumers (layout only):
  * cell index c = x + nx*(y + ny*z);
  * the six face directions of a cell are ordered (-z, -y, -x, +x, +y, +z),
    which is ascending neighbour index;
  * wells are numbered after the cells; well w is injector if w is even and
    producer of the same pair if odd; perforations are listed well by well,
    each well's perforations in ascending x;
  * vectors hold (n_c + n_w) blocks of b entries; a well's BHP is entry 0 of
    its block, entries 1..b-1 of a well block are padding (zero RHS).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

#: face directions as (dx, dy, dz), ascending neighbour index
DIRECTIONS = ((0, 0, -1), (0, -1, 0), (-1, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1))

#: geometric transmissibility constant per mD for unit cells and unit faces
C_T = 1.0e-3

#: seed base of the named workloads
SEED_BASE = 1812_03952


@dataclass
class SyntheticSystem:
    nx: int
    ny: int
    nz: int
    b: int
    k: np.ndarray            # float64 [n_c] permeability in mD (0 = impermeable)
    kvkh: float              # vertical/horizontal permeability ratio
    c_t: float               # transmissibility constant
    M: np.ndarray            # float64 [n_c, 6, b, b] mobility block per directed face
    acc: np.ndarray          # float64 [n_c, b, b] accumulation block
    n_wells: int
    perf_well: np.ndarray    # int32 [n_perf]
    perf_cell: np.ndarray    # int32 [n_perf]
    wi: np.ndarray           # float64 [n_perf] well index
    lam: np.ndarray          # float64 [n_perf, b] perforation mobilities
    rhs: np.ndarray          # float64 [(n_c + n_w) * b]
    name: str = "custom"
    meta: dict = field(default_factory=dict)

    @property
    def n_cells(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def n_rows(self) -> int:
        return self.n_cells + self.n_wells

    @property
    def n_unknowns(self) -> int:
        """Padded vector length (n_c + n_w) * b."""
        return self.n_rows * self.b

    @property
    def theta(self) -> np.ndarray:
        """Log-permeability (only defined where k > 0)."""
        with np.errstate(divide="ignore"):
            return np.log(self.k)


def cell_index(nx, ny, x, y, z):
    return x + nx * (y + ny * z)


def lognormal_perm(rng, n, mean_md=500.0, sigma=1.0):
    """i.i.d. lognormal permeability with arithmetic mean ``mean_md``."""
    mu = np.log(mean_md) - 0.5 * sigma * sigma
    return np.exp(mu + sigma * rng.standard_normal(n))


def facies_perm(rng, nx, ny, nz, sand=2000.0, shale=50.0, shale_frac=0.30,
                corr=(8.0, 2.0, 1.0)):
    """Binary channelised field: smoothed Gaussian noise thresholded so that
    ``shale_frac`` of the cells are shale.  ``corr`` is the smoothing length in
    cells along (x, y, z)."""
    from scipy.ndimage import gaussian_filter
    noise = rng.standard_normal((nz, ny, nx))
    field_ = gaussian_filter(noise, sigma=(corr[2], corr[1], corr[0]), mode="wrap")
    cut = np.quantile(field_, shale_frac)
    k = np.where(field_ <= cut, shale, sand)
    return k.reshape(-1).astype(np.float64)


def shale_lenses(rng, nx, ny, nz, frac=0.10):
    """Boolean mask of one-cell-thick horizontal lenses of size U(8,64) x U(4,32)
    cells, added until at least ``frac`` of the cells are covered."""
    mask = np.zeros((nz, ny, nx), dtype=bool)
    target = frac * mask.size
    covered = 0
    while covered < target:
        lx = int(rng.integers(8, 65))
        ly = int(rng.integers(4, 33))
        x0 = int(rng.integers(0, max(1, nx - lx + 1)))
        y0 = int(rng.integers(0, max(1, ny - ly + 1)))
        z0 = int(rng.integers(0, nz))
        sub = mask[z0, y0:y0 + ly, x0:x0 + lx]
        covered += int(sub.size - sub.sum())
        sub[...] = True
    return mask.reshape(-1)


def horizontal_pairs(nx, ny, nz, ys, z_inj, z_prod, x0, x1):
    """SAGD well pairs along x: list of per-well cell lists (injector first)."""
    wells = []
    for y in ys:
        for zi, zp in zip(np.atleast_1d(z_inj), np.atleast_1d(z_prod)):
            wells.append([cell_index(nx, ny, x, y, zi) for x in range(x0, x1)])
            wells.append([cell_index(nx, ny, x, y, zp) for x in range(x0, x1)])
    return wells


def build_system(nx, ny, nz, b, k, wells, seed, kvkh=1.0, name="custom", meta=None):
    """Draw the mobility/accumulation blocks, the perforation data and the RHS.

    * M (one per directed face): column 0 (pressure, the phase mobilities)
      ~ U(1, 2), other columns (mobility derivatives times the potential
      difference) ~ U(0, 0.01): a dominant pressure column.
    * Acc = s * (diag(0.05 u_0, u_1, ..., u_{b-1}) + off-diagonal U(-0.05, 0.05)),
      u ~ U(0.5, 1.5), s = C_T * mean(k): over one day the transported
      unknowns accumulate on the scale of one face transmissibility (cell
      CFL number near one), while the pressure column only sees a small
      compressibility term, so the pressure sub-problem stays elliptic.
    * WI = 10 * C_T * mean(k) for every perforation; lam ~ U(0.5, 1.5)^b.
    * RHS ~ N(0, 1) on real unknowns, 0 on padded well entries.
    """
    rng = np.random.default_rng(seed)
    n_c = nx * ny * nz
    M = rng.uniform(0.0, 0.01, size=(n_c, 6, b, b))
    M[:, :, :, 0] = rng.uniform(1.0, 2.0, size=(n_c, 6, b))
    kmean = float(np.mean(k))
    s = C_T * kmean
    acc = rng.uniform(-0.05, 0.05, size=(n_c, b, b))
    idx = np.arange(b)
    acc[:, idx, idx] = rng.uniform(0.5, 1.5, size=(n_c, b))
    acc[:, 0, 0] *= 0.05
    acc *= s
    perf_well, perf_cell = [], []
    for w, cells in enumerate(wells):
        if len(set(cells)) != len(cells):
            raise ValueError("a well perforates a cell twice")
        perf_well.extend([w] * len(cells))
        perf_cell.extend(cells)
    n_perf = len(perf_cell)
    perf_well = np.asarray(perf_well, dtype=np.int32)
    perf_cell = np.asarray(perf_cell, dtype=np.int32)
    wi = np.full(n_perf, 10.0 * C_T * kmean)
    lam = rng.uniform(0.5, 1.5, size=(n_perf, b))
    n_w = len(wells)
    rhs = rng.standard_normal((n_c + n_w, b))
    rhs[n_c:, 1:] = 0.0
    return SyntheticSystem(nx=nx, ny=ny, nz=nz, b=b, k=np.ascontiguousarray(k, dtype=np.float64),
                           kvkh=float(kvkh), c_t=C_T, M=np.ascontiguousarray(M),
                           acc=np.ascontiguousarray(acc), n_wells=n_w, perf_well=perf_well,
                           perf_cell=perf_cell, wi=wi, lam=np.ascontiguousarray(lam),
                           rhs=rhs.reshape(-1).copy(), name=name, meta=dict(meta or {}))


def small_system(nx=6, ny=5, nz=3, b=4, seed=7, sigma=1.0, n_pairs=1, kvkh=1.0,
                 shale_frac=0.0, name=None):
    """A small system for tests: lognormal k, ``n_pairs`` horizontal pairs."""
    rng = np.random.default_rng(seed)
    n_c = nx * ny * nz
    k = lognormal_perm(rng, n_c, 500.0, sigma)
    if shale_frac > 0:
        k[rng.random(n_c) < shale_frac] = 0.0
    wells = []
    if n_pairs > 0 and nz >= 2:
        ys = [int(v) for v in np.linspace(0, ny - 1, n_pairs + 2)[1:-1].round()]
        zi, zp = max(0, nz // 2 - 1), min(nz - 1, nz // 2)
        x0, x1 = (1, nx - 1) if nx > 2 else (0, nx)
        wells = horizontal_pairs(nx, ny, nz, ys, zi, zp, x0, x1)
    return build_system(nx, ny, nz, b, k, wells, seed + 1, kvkh=kvkh,
                        name=name or f"small_{nx}x{ny}x{nz}_b{b}")


def config(index: int) -> SyntheticSystem:
    """The five named workloads (0-based index).

    0: 16x16x4, b=4, sigma 1.0, one vertical injector/producer pair.
    1: 128x128x64, b=4, sigma 1.5, kv/kh 0.1, 4 SAGD pairs of 100 perforations.
    2: 256x256x128, b=5, channelised sand/shale, 16 pairs of 200 perforations.
    3: 64x64x32, b=4, sigma 1.0, one pair of 48 perforations (adjoint check).
    4: 512x256x64, b=4, sigma 2.0 with 10% shale lenses, 200 pairs of 150.
    """
    seed = SEED_BASE + index + 1
    rng = np.random.default_rng(seed)
    if index == 0:
        nx, ny, nz, b = 16, 16, 4, 4
        k = lognormal_perm(rng, nx * ny * nz, 500.0, 1.0)
        wells = [[cell_index(nx, ny, 2, 2, z) for z in range(nz)],
                 [cell_index(nx, ny, 13, 13, z) for z in range(nz)]]
        return build_system(nx, ny, nz, b, k, wells, seed + 100, 1.0, "16x16x4_b4")
    if index == 1:
        nx, ny, nz, b = 128, 128, 64, 4
        k = lognormal_perm(rng, nx * ny * nz, 500.0, 1.5)
        wells = horizontal_pairs(nx, ny, nz, [16, 48, 80, 112], 29, 34, 14, 114)
        return build_system(nx, ny, nz, b, k, wells, seed + 100, 0.1, "128x128x64_b4")
    if index == 2:
        nx, ny, nz, b = 256, 256, 128, 5
        k = facies_perm(rng, nx, ny, nz)
        wells = horizontal_pairs(nx, ny, nz, [8 + 16 * m for m in range(16)], 60, 65, 28, 228)
        return build_system(nx, ny, nz, b, k, wells, seed + 100, 1.0, "256x256x128_b5")
    if index == 3:
        nx, ny, nz, b = 64, 64, 32, 4
        k = lognormal_perm(rng, nx * ny * nz, 500.0, 1.0)
        wells = horizontal_pairs(nx, ny, nz, [32], 13, 18, 8, 56)
        return build_system(nx, ny, nz, b, k, wells, seed + 100, 1.0, "64x64x32_b4")
    if index == 4:
        nx, ny, nz, b = 512, 256, 64, 4
        k = lognormal_perm(rng, nx * ny * nz, 500.0, 2.0)
        k[shale_lenses(rng, nx, ny, nz, 0.10)] = 0.0
        ys = [2 + 5 * m for m in range(50)]
        wells = horizontal_pairs(nx, ny, nz, ys, [8, 24, 40, 56], [13, 29, 45, 61], 181, 331)
        return build_system(nx, ny, nz, b, k, wells, seed + 100, 1.0, "512x256x64_b4")
    raise ValueError(f"no workload {index}")


def diagonal_scalings(n_rows: int, steps: int, seed: int, amplitude: float = 0.2):
    """Per-step, per-row factors (1 + amplitude*u), u ~ U(-1, 1), for a
    sequence of Newton-like systems (applied to the cells' accumulation
    blocks, or to whole diagonal blocks by trs_bsr_scale_diagonal)."""
    rng = np.random.default_rng(seed)
    return 1.0 + amplitude * rng.uniform(-1.0, 1.0, size=(steps, n_rows))


def seeded_directions(n: int, count: int, seed: int):
    """Unit directions for finite-difference checks."""
    rng = np.random.default_rng(seed)
    d = rng.standard_normal((count, n))
    return d / np.linalg.norm(d, axis=1, keepdims=True)


# ------------------------------------------------------------- thermal state
#: oil-water relative permeability table of the paper (Fig. rela-swt):
#: S_w, k_rw, k_row (capillary pressure zero)
SWT = np.array([
    [0.45, 0.0, 0.4], [0.47, 0.000056, 0.361], [0.50, 0.000552, 0.30625], [0.55, 0.00312, 0.225],
    [0.60, 0.00861, 0.15625], [0.65, 0.01768, 0.1], [0.70, 0.03088, 0.05625], [0.75, 0.04871, 0.025],
    [0.77, 0.05724, 0.016], [0.80, 0.07162, 0.00625], [0.82, 0.08229, 0.00225], [0.85, 0.1, 0.0]])

#: liquid-gas relative permeability table of the paper (Fig. rela-slt):
#: S_l = S_w + S_o, k_rg, k_rog
SLT = np.array([
    [0.45, 0.2, 0.0], [0.55, 0.14202, 0.0], [0.57, 0.13123, 0.00079], [0.60, 0.11560, 0.00494],
    [0.62, 0.10555, 0.00968], [0.65, 0.09106, 0.01975], [0.67, 0.08181, 0.02844], [0.70, 0.06856, 0.04444],
    [0.72, 0.06017, 0.05709], [0.75, 0.04829, 0.07901], [0.77, 0.04087, 0.09560], [0.80, 0.03054, 0.12346],
    [0.83, 0.02127, 0.15486], [0.85, 0.01574, 0.17778], [0.87, 0.01080, 0.20227], [0.90, 0.00467, 0.24198],
    [0.92, 0.00165, 0.27042], [0.94, 0.0, 0.30044], [1.0, 0.0, 0.4]])

#: parameter order of the thermal model (the layout both consumers read)
THERMAL_FIELDS = (
    "dx", "dy", "dz", "depth_top", "dt", "kvkh", "gravity",
    "phi_ref", "cpor", "ctpor", "p_ref", "T_ref", "cp1_r", "cp2_r",
    "kt_w", "kt_o", "kt_g", "kt_r",
    "rho_w_ref", "cp_w", "ct1_w", "ct2_w", "cpt_w", "mw_w", "avisc_w", "bvisc_w",
    "kv1", "kv2", "kv3", "kv4", "kv5", "per_eps", "tc_w", "pc_w",
    "cpg1", "cpg2", "cpg3", "cpg4", "cpg5", "hvr", "ev",
    "rho_o_ref", "cp_o", "ct1_o", "ct2_o", "cpt_o", "mw_o", "avisc_o", "bvisc_o", "cpl1_o",
    "mug_a", "mug_b", "h_inj", "R_gas")


def thermal_params(kvkh=1.0, dt=0.1, gravity=9.80665):
    """Parameters of the water + heavy-oil thermal model.  Units: p kPa, T C,
    lengths m, time day, amounts gmol, energy kJ, permeability mD, viscosity cP.

    Values the paper gives: the water K-value constants kv1 = 1.1705e5 atm,
    kv4 = -3816.44, kv5 = -227.02 C; the water gas heat-capacity polynomial
    (34.49885, -0.01426, 4.7356e-5, -3.56759e-8, 9.35531e-12 J/(gmol C^k))
    and hvr = 4820 J/(gmol C^0.38), ev = 0.38; the oil liquid heat capacity
    0.5 Btu/(lb F); the gas viscosity 0.0136 + 3.8e-5 T cP (Sec. "Phase
    Equilibrium Constraints", "Viscosity", "Energy").  The rest are typical
    values for a heavy-oil (bitumen) reservoir: oil viscosity about 1.6e6 cP
    at 15 C and 10 cP at 200 C, water 1.0 cP at 20 C and 0.135 cP at 200 C."""
    p = dict(
        dx=5.0, dy=2.0, dz=1.0, depth_top=300.0, dt=dt, kvkh=kvkh, gravity=gravity,
        phi_ref=0.3, cpor=1.0e-6, ctpor=0.0, p_ref=101.325, T_ref=15.0, cp1_r=2350.0, cp2_r=0.0,
        kt_w=53.5, kt_o=11.5, kt_g=4.0, kt_r=216.0,
        rho_w_ref=55500.0, cp_w=4.5e-7, ct1_w=2.0e-4, ct2_w=1.0e-6, cpt_w=0.0, mw_w=0.018015,
        avisc_w=5.17e-3, bvisc_w=1543.0,
        kv1=1.1705e5 * 101.325, kv2=0.0, kv3=0.0, kv4=-3816.44, kv5=-227.02, per_eps=1.0e-4,
        tc_w=373.946, pc_w=22064.0,
        cpg1=34.49885e-3, cpg2=-0.01426e-3, cpg3=4.7356e-5 * 1e-3, cpg4=-3.56759e-8 * 1e-3,
        cpg5=9.35531e-12 * 1e-3, hvr=4.820, ev=0.38,
        rho_o_ref=1600.0, cp_o=7.0e-7, ct1_o=6.5e-4, ct2_o=0.0, cpt_o=0.0, mw_o=0.6,
        avisc_o=7.2e-8, bvisc_o=8860.0, cpl1_o=0.5 * 4.1868 * 0.6,
        mug_a=0.0136, mug_b=3.8e-5, h_inj=8.3, R_gas=8.314462618e-3)
    assert tuple(p) == THERMAL_FIELDS
    return p


@dataclass
class ThermalState:
    """A Newton iterate of the thermal model and its data: u and u_old hold
    (n_c + n_w) blocks of (p, S_w, S_g, T) for cells and (p_b, 0, 0, 0) for
    wells; gas[c] = 1 where the gas phase exists."""
    u: np.ndarray
    u_old: np.ndarray
    gas: np.ndarray          # uint8 [n_c]
    wi: np.ndarray           # float64 [n_perf]: injectors gmol/(day kPa), producers mD m
    well_type: np.ndarray    # int32 [n_w]: 0 injector at a fixed rate, 1 producer at a fixed BHP
    well_target: np.ndarray  # float64 [n_w]: rate (gmol/day) or BHP (kPa)
    params: dict


def thermal_state(sysm: SyntheticSystem, seed: int, dt=0.1, gravity=9.80665) -> ThermalState:
    """A seeded SAGD-like state of the thermal model on sysm's grid and wells:
    near-hydrostatic pressure, a steam chamber (gas present, 185-205 C) around
    each injector, a warm ring around it and cold bitumen elsewhere; the
    previous time level slightly cooler, at lower pressure and with slightly
    different saturations.  The default time step, 0.1 day, keeps the cell
    throughput of the 1 m cells in the steam chamber on the scale of the
    cell's content over a step."""
    rng = np.random.default_rng(seed)
    prm = thermal_params(sysm.kvkh, dt, gravity)
    nx, ny, nz = sysm.nx, sysm.ny, sysm.nz
    n_c, n_w = sysm.n_cells, sysm.n_wells
    z = np.arange(n_c) // (nx * ny)
    y = (np.arange(n_c) // nx) % ny
    x = np.arange(n_c) % nx
    depth = prm["depth_top"] + (z + 0.5) * prm["dz"]
    p = 1500.0 + 9.8 * (depth - prm["depth_top"]) + rng.normal(0.0, 5.0, n_c)
    # distance to the nearest injector line (in cells, y-z plane) within its x range
    dist = np.full(n_c, np.inf)
    for w in range(0, n_w, 2):
        cells = sysm.perf_cell[sysm.perf_well == w]
        if len(cells) == 0:
            continue
        wx, wy, wz = cells % nx, (cells // nx) % ny, cells // (nx * ny)
        inside = (x >= wx.min()) & (x <= wx.max())
        d = np.sqrt((y - wy[0]) ** 2 + (z - wz[0]) ** 2)
        dist = np.where(inside, np.minimum(dist, d), dist)
    chamber = dist <= 2.0
    ring = (dist > 2.0) & (dist <= 4.0)
    T = rng.uniform(12.0, 20.0, n_c)
    T[ring] = rng.uniform(40.0, 150.0, int(ring.sum()))
    T[chamber] = rng.uniform(185.0, 205.0, int(chamber.sum()))
    Sw = rng.uniform(0.5, 0.75, n_c)
    Sg = np.zeros(n_c)
    Sw[chamber] = rng.uniform(0.46, 0.55, int(chamber.sum()))
    Sg[chamber] = rng.uniform(0.1, 0.35, int(chamber.sum()))
    gas = chamber.astype(np.uint8)
    u = np.zeros((n_c + n_w, 4))
    u[:n_c] = np.stack([p, Sw, Sg, T], axis=1)
    u_old = u.copy()
    u_old[:n_c, 0] -= rng.uniform(0.0, 3.0, n_c)
    u_old[:n_c, 3] -= rng.uniform(0.0, 0.5, n_c)
    u_old[:n_c, 1] += rng.uniform(-0.005, 0.005, n_c)
    u_old[:n_c, 2] = np.where(chamber, np.clip(Sg + rng.uniform(-0.005, 0.005, n_c), 0.0, None), 0.0)
    n_perf = len(sysm.perf_cell)
    wi = np.zeros(n_perf)
    well_type = (np.arange(n_w) % 2).astype(np.int32)
    well_target = np.zeros(n_w)
    for w in range(n_w):
        m = sysm.perf_well == w
        pc = p[sysm.perf_cell[m]] if m.any() else np.array([1500.0])
        if well_type[w] == 0:
            wi[m] = rng.uniform(200.0, 400.0, int(m.sum()))
            u[n_c + w, 0] = float(pc.mean()) + 300.0
            well_target[w] = float(wi[m].sum()) * 300.0 * rng.uniform(0.9, 1.1)
        else:
            wi[m] = rng.uniform(0.5e4, 1.5e4, int(m.sum()))
            well_target[w] = float(pc.mean()) - 200.0
            u[n_c + w, 0] = well_target[w] + rng.uniform(-5.0, 5.0)
    u_old[n_c:] = u[n_c:]
    return ThermalState(u=u.reshape(-1).copy(), u_old=u_old.reshape(-1).copy(), gas=gas, wi=wi,
                        well_type=well_type, well_target=well_target, params=prm)
