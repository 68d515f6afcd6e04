"""Pins of the oracle's per-tet materials (Sec. 3.1: the force is local to
each tet, so regions of a cell such as a nucleus or a cortex may carry their
own parameters): regions that share one material reproduce the uniform
cell exactly, the forces superpose over regions (U is a sum over tets), and
they stay the negative gradient of the strain energy."""
import numpy as np

import oracle
from workloads.configs import Cell
from workloads.mesh import perturb, shell_regions, sphere_tet_mesh

RNG = np.random.default_rng(11)


def cell(region_materials=None, mu=1e-3, kappa=0.1, w=0.5):
    x, t = sphere_tet_mesh(4.0, 1.3)
    y = perturb(x, 0.15, 3)
    c = Cell(x, t, y, mu, kappa, w)
    if region_materials is not None:
        c.regions = shell_regions(x, t, 1.8, 3.0)
        c.region_materials = region_materials
    return c


def test_regions_cover_all_three_shells():
    c = cell([(1, 1, 1)] * 3)
    counts = np.bincount(c.regions, minlength=3)
    assert (counts > 0).all() and counts.sum() == len(c.tets)


def test_equal_region_materials_reproduce_the_uniform_cell():
    uni = cell()
    reg = cell([(1e-3, 0.1, 0.5)] * 3)
    mu_, mr = oracle.Mesh([uni]), oracle.Mesh([reg])
    assert np.array_equal(mu_.forces(uni.y0), mr.forces(reg.y0))


def test_forces_superpose_over_regions():
    mats = [(5e-3, 0.4, 0.8), (1e-3, 0.1, 0.3), (2e-3, 0.2, 0.0)]
    full = oracle.Mesh([cell(mats)]).forces(cell(mats).y0)
    parts = np.zeros_like(full)
    for r in range(3):
        only = [m if k == r else (0.0, 0.0, 0.5) for k, m in enumerate(mats)]
        c = cell(only)
        parts += oracle.Mesh([c]).forces(c.y0)
    assert np.allclose(parts, full, rtol=0, atol=1e-12 * np.abs(full).max())
    assert np.abs(full).max() > 0


def test_region_forces_are_the_energy_gradient():
    mats = [(5e-3, 0.4, 0.8), (1e-3, 0.1, 0.3), (2e-3, 0.2, 0.0)]
    c = cell(mats)
    m = oracle.Mesh([c])
    f = m.forces(c.y0)
    y = c.y0.copy()
    h = 1e-6
    for v in RNG.choice(len(y), 12, replace=False):
        for a in range(3):
            yp, ym = y.copy(), y.copy()
            yp[v, a] += h
            ym[v, a] -= h
            g = (m.energy(yp) - m.energy(ym)) / (2 * h)
            assert abs(-g - f[v, a]) <= 1e-7 * np.abs(f).max()
