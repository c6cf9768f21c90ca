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
