"""Seeded synthetic workloads shaped like the paper's shear-flow runs (Sec. 6).

Each builder returns plain numpy arrays and numbers; it does none of the
method's arithmetic. Lattice nodes sit at integer coordinates ``0..n-1``;
the moving walls sit half a spacing outside the first and last y rows.

Readings of the paper that fix these shapes:

* Sec. 6.1 drives linear shear by moving the x-z planes in -x (bottom) and
  +x (top) with ``u_wall = H * gamma_dot / 2``; periodic in x and z.
* Sec. 6.1 defines ``Ca = eta * gamma_dot / mu``. In lattice units
  ``eta = rho * c_s^2 * (tau - 1/2)`` with ``rho = 1`` and ``gamma_dot =
  2 u_wall / ny``.
* Sec. 2 sets ``mu_1 = w mu`` and ``mu_2 = (1 - w) mu``.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np

from .mesh import perturb, sphere_tet_mesh

NOISE_SEED = 20030313


@dataclass
class Cell:
    x_ref: np.ndarray  # [V,3] float64, absolute lattice coordinates
    tets: np.ndarray  # [T,4] int32
    y0: np.ndarray  # [V,3] float64, current positions at t = 0
    mu: float
    kappa: float
    w: float
    # optional materials per tet: region index [T] and one (mu, kappa, w) per region
    regions: Optional[np.ndarray] = None
    region_materials: Optional[list] = None


@dataclass
class Workload:
    name: str
    nx: int
    ny: int
    nz: int
    tau: float
    u_wall_lo: float  # x velocity of the wall at y = -1/2
    u_wall_hi: float  # x velocity of the wall at y = ny - 1/2
    body_force: tuple = (0.0, 0.0, 0.0)
    cells: list = field(default_factory=list)
    steps: int = 100
    delta: int = 2  # immersed-boundary delta kernel: support width 2 (trilinear) or 4 (Peskin four-point)

    @property
    def n_nodes(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def n_tets(self) -> int:
        return sum(len(c.tets) for c in self.cells)

    @property
    def n_verts(self) -> int:
        return sum(len(c.x_ref) for c in self.cells)


def lattice_viscosity(tau: float) -> float:
    """Kinematic viscosity of the BGK lattice fluid, c_s^2 (tau - 1/2)."""
    return (tau - 0.5) / 3.0


def shear_modulus_for_ca(ca: float, tau: float, u_wall: float, ny: int) -> float:
    """mu from Ca = eta gamma_dot / mu (Sec. 6.1), rho = 1."""
    gamma_dot = 2.0 * u_wall / ny
    return lattice_viscosity(tau) * gamma_dot / ca


def sphere_cell(R, h, centre, mu, kappa, w, noise=0.0, seed=NOISE_SEED) -> Cell:
    x, tets = sphere_tet_mesh(R, h)
    x = x + np.asarray(centre, np.float64)[None, :]
    y0 = perturb(x, noise, seed) if noise > 0 else x.copy()
    return Cell(x_ref=x, tets=tets, y0=y0, mu=mu, kappa=kappa, w=w)


def small_shear(steps: int = 100) -> Workload:
    """32^3 box, R = 8 sphere (~1k vertices, ~4.3k tets), mu = 1e-3,
    kappa = 0.1, w = 0.5, current positions perturbed by 1 % of R, tau = 1,
    walls at -/+0.01. Sized for the FP64 oracle."""
    cell = sphere_cell(8.0, 1.4, (15.5, 15.5, 15.5), 1e-3, 0.1, 0.5, noise=0.08)
    return Workload("shear_32^3_R8", 32, 32, 32, 1.0, -0.01, 0.01, cells=[cell], steps=steps)


def production_shear(ca: float = 0.2, w: float = 1.0, steps: int = 10000, n: int = 128) -> Workload:
    """128^3 box, R = 16 sphere (~4.2k vertices, ~20k tets) at the centre,
    walls at -/+0.05, tau = 1; mu from Ca, kappa = 50 mu."""
    u_wall = 0.05
    mu = shear_modulus_for_ca(ca, 1.0, u_wall, n)
    c = (n - 1) / 2.0
    cell = sphere_cell(16.0, 1.72, (c, c, c), mu, 50.0 * mu, w)
    return Workload(f"shear_{n}^3_R16_Ca{ca}_w{w}", n, n, n, 1.0, -u_wall, u_wall, cells=[cell], steps=steps)


def paper_box_shear(ca: float = 0.2, w: float = 0.5, steps: int = 10000) -> Workload:
    """The paper's single-cell shear box, 10 x 15 x 5 cell radii (Sec. 6.1,
    shear gradient along the 15 R axis), at R = 16: a 160 x 240 x 80 lattice
    (3.07 M nodes) with the same R = 16 cell at the centre, walls at -/+0.05,
    tau = 1; mu from Ca at this box's shear rate, kappa = 50 mu."""
    nx, ny, nz, u_wall = 160, 240, 80, 0.05
    mu = shear_modulus_for_ca(ca, 1.0, u_wall, ny)
    cell = sphere_cell(16.0, 1.72, ((nx - 1) / 2.0, (ny - 1) / 2.0, (nz - 1) / 2.0), mu, 50.0 * mu, w)
    return Workload(f"shear_160x240x80_R16_Ca{ca}_w{w}", nx, ny, nz, 1.0, -u_wall, u_wall, cells=[cell],
                    steps=steps)


def multicell_shear(ncells: int = 8, R: float = 16.0, h: float = 1.72, ca: float = 0.2, w: float = 0.5,
                    u_wall: float = 0.05, seed: int = 55, steps: int = 10000) -> Workload:
    """The paper's multiple-cell setup (Sec. 6.2): ncells cells of radius R
    at seeded random positions (no overlap, gap >= 2 lattice units, at least
    R + 2 from the walls, periodic in x and z) in a 5 x 8 x 4 R box with
    moving walls across its 8 R axis; 4 cells fill 11 % of the box, 8 cells
    22 %. At R = 16 the box is 80 x 128 x 64. mu from Ca, kappa = 50 mu."""
    rng = np.random.Generator(np.random.PCG64(seed))
    nx, ny, nz = int(round(5 * R)), int(round(8 * R)), int(round(4 * R))
    L = np.array([nx, ny, nz], np.float64)
    centres = []
    for _ in range(ncells):
        for _ in range(200000):
            c = np.array([rng.uniform(0, nx), rng.uniform(R + 2.0, ny - 3.0 - R), rng.uniform(0, nz)])
            ok = True
            for o in centres:
                d = np.abs(c - o)
                d[[0, 2]] = np.minimum(d[[0, 2]], L[[0, 2]] - d[[0, 2]])
                if np.sqrt((d * d).sum()) < 2 * R + 2.0:
                    ok = False
                    break
            if ok:
                break
        else:
            raise RuntimeError("could not place all cells")
        centres.append(c)
    mu = shear_modulus_for_ca(ca, 1.0, u_wall, ny)
    x, tets = sphere_tet_mesh(R, h)
    cells = [Cell(x_ref=x + c[None, :], tets=tets, y0=x + c[None, :], mu=mu, kappa=50.0 * mu, w=w) for c in centres]
    return Workload(f"multicell_{nx}x{ny}x{nz}_{ncells}cells_R{R:g}_Ca{ca}", nx, ny, nz, 1.0, -u_wall, u_wall,
                    cells=cells, steps=steps)


def precision_channel(steps: int = 2000, nx: int = 256, ny: int = 128, nz: int = 128) -> Workload:
    """Pressure-driven channel 256 x 128 x 128 (walls at rest, uniform body
    force for a centre-line velocity of 0.02 at tau = 1: g = 8 nu u_max / ny^2),
    one R = 16 cell a quarter of the width off the centre plane (in shear),
    mu = 6.51e-4 (as the 128^3 shear workload at Ca = 0.2), kappa = 50 mu,
    w = 0.5."""
    tau = 1.0
    g = 8.0 * lattice_viscosity(tau) * 0.02 / ny**2
    mu = shear_modulus_for_ca(0.2, tau, 0.05, 128)
    cell = sphere_cell(16.0, 1.72, ((nx - 1) / 2.0, ny / 4.0 + 8.0, (nz - 1) / 2.0), mu, 50.0 * mu, 0.5)
    return Workload(f"channel_{nx}x{ny}x{nz}_R16", nx, ny, nz, tau, 0.0, 0.0, body_force=(g, 0.0, 0.0),
                    cells=[cell], steps=steps)


def batched_channel(ncells: int = 400, nx: int = 512, ny: int = 256, nz: int = 256, r_min: float = 6.0,
                    r_max: float = 20.0, seed: int = 400, steps: int = 100, h: float = 1.64) -> Workload:
    """Suspension in a pressure-driven channel: ``ncells`` spheres with radii
    drawn uniformly from [r_min, r_max] (rounded to 0.5 so meshes can be
    shared), placed without overlap (gap >= 2 lattice units, periodic in x and
    z, at least R + 2 from the walls) by seeded rejection sampling; per-cell
    mu log-uniform in [2.6e-4, 1.3e-3] (Ca 0.1-0.5 at the 128^3 shear rate),
    kappa = 50 mu, w uniform in [0, 1]; centre-line velocity 0.02 at tau = 1.
    Meshes use spacing h (tets grow as R^3; ~6M tets in all for 400 cells)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    radii = np.round(rng.uniform(r_min, r_max, ncells) * 2.0) / 2.0
    order = np.argsort(-radii, kind="stable")  # place large cells first
    centres = np.zeros((ncells, 3))
    placed = []
    L = np.array([nx, ny, nz], np.float64)
    for i in order:
        R = radii[i]
        for _ in range(200000):
            c = np.array([rng.uniform(0, nx), rng.uniform(R + 2.0, ny - 3.0 - R), rng.uniform(0, nz)])
            ok = True
            for j in placed:
                d = np.abs(c - centres[j])
                d[[0, 2]] = np.minimum(d[[0, 2]], L[[0, 2]] - d[[0, 2]])
                if np.sqrt((d * d).sum()) < R + radii[j] + 2.0:
                    ok = False
                    break
            if ok:
                break
        else:
            raise RuntimeError("could not place all cells")
        centres[i] = c
        placed.append(i)
    mus = np.exp(rng.uniform(np.log(2.6e-4), np.log(1.3e-3), ncells))
    ws = rng.uniform(0.0, 1.0, ncells)
    cache = {}
    cells = []
    for i in range(ncells):
        R = float(radii[i])
        if R not in cache:
            cache[R] = sphere_tet_mesh(R, h)
        x, tets = cache[R]
        xc = x + centres[i][None, :]
        cells.append(Cell(x_ref=xc, tets=tets, y0=xc.copy(), mu=float(mus[i]), kappa=50.0 * float(mus[i]),
                          w=float(ws[i])))
    tau = 1.0
    g = 8.0 * lattice_viscosity(tau) * 0.02 / ny**2
    return Workload(f"suspension_{nx}x{ny}x{nz}_{ncells}cells", nx, ny, nz, tau, 0.0, 0.0, body_force=(g, 0.0, 0.0),
                    cells=cells, steps=steps)


@dataclass
class CompressionSet:
    """Cells to compress between plates, with their hidden moduli."""
    cells: list
    hidden_mu: np.ndarray
    hidden_kappa: np.ndarray
    hidden_w: np.ndarray
    strains: list
    steps: int
    dt: float
    damping: float
    k_plate: float
    ramp: int


def compression_set(ncells: int = 64, R: float = 10.0, h: float = 1.45, steps: int = 2000, seed: int = 5):
    """64 spheres of radius 10 (8,256 tets each) spaced apart, each with
    hidden moduli (mu log-uniform in [0.7, 1.4], kappa = 20 mu x U(0.8, 1.25),
    i.e. a Poisson ratio near 0.475, w uniform in [0.2, 0.9]); protocol: 8
    strain levels to 80 %, 2,000 damped steps per level (dt 0.03, velocity
    retention 0.95), plate stiffness 50, the plate approaching in 10 moves.
    Every cell starts from mu = 1, kappa = 20, w = 0.5."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x, tets = sphere_tet_mesh(R, h)
    cells = []
    for k in range(ncells):
        off = np.array([3.0 * R * (k % 4), 3.0 * R * ((k // 4) % 4), 3.0 * R * (k // 16)])
        cells.append(Cell(x_ref=x + off, tets=tets, y0=x + off, mu=1.0, kappa=20.0, w=0.5))
    mu = np.exp(rng.uniform(np.log(0.7), np.log(1.4), ncells))
    kappa = 20.0 * mu * rng.uniform(0.8, 1.25, ncells)
    w = rng.uniform(0.2, 0.9, ncells)
    return CompressionSet(cells, mu, kappa, w, [0.1 * (i + 1) for i in range(8)], steps, 0.03, 0.95, 50.0, 10)


def plate_schedule(z_lo, radius, strains, steps, ramp):
    """Top-plate heights of a quasi-static compression protocol (Sec. 4.2:
    the upper plate approaches step by step while the cell relaxes). Per
    strain level s the plate moves from its previous height to
    ``z_lo + 2 R (1 - s)`` in ``ramp`` equal moves of ``steps // (2 ramp)``
    relaxation steps each, then holds for the rest of the level's ``steps``.
    Yields ``(z_hi per cell, number of steps, measured)`` with ``measured``
    True for the hold that ends a level; ``ramp = 0`` jumps to the new height
    at once. The plate starts at ``z_lo + 2 R`` (touching an undeformed
    sphere of radius R resting on the lower plate)."""
    z_lo, radius = np.asarray(z_lo, np.float64), np.asarray(radius, np.float64)
    prev = z_lo + 2.0 * radius
    for s in strains:
        new = z_lo + 2.0 * radius * (1.0 - s)
        n_move = steps // (2 * ramp) if ramp > 0 else 0
        for r in range(1, ramp + 1):
            yield prev + (new - prev) * (r / ramp), n_move, False
        yield new, steps - ramp * n_move, True
        prev = new


def random_displacements(cell: Cell, amplitude: float, seed: int) -> np.ndarray:
    """Positions of ``cell`` perturbed by ``amplitude * U(-1, 1)``."""
    return perturb(cell.x_ref, amplitude, seed)


def random_populations_like(shape, scale: float, seed: int) -> np.ndarray:
    """Seeded uniform noise of the given shape (for lattice initial states)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return scale * rng.uniform(-1.0, 1.0, size=shape)
