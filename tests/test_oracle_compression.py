"""Pins of the oracle's plate-compression protocol (Sec. 4.2 reading: harmonic
plate penalty, damped relaxation)."""
import numpy as np

import oracle
from oracle import compression as cp
from workloads.configs import Cell
from workloads.mesh import perturb, sphere_tet_mesh

RNG = np.random.default_rng(21)


def test_plate_force_is_minus_plate_energy_gradient():
    y = RNG.uniform(-1, 1, (30, 3))
    zl, zh = np.full(30, -0.3), np.full(30, 0.4)
    f = cp.plate_forces(y, 7.0, zl, zh)
    for _ in range(10):
        v, i = int(RNG.integers(30)), int(RNG.integers(3))
        h = 1e-6
        yp, ym = y.copy(), y.copy()
        yp[v, i] += h
        ym[v, i] -= h
        fd = -(cp.plate_energy(yp, 7.0, zl, zh) - cp.plate_energy(ym, 7.0, zl, zh)) / (2 * h)
        assert abs(fd - f[v, i]) < 1e-6


def test_no_contact_no_plate_force():
    x, t = sphere_tet_mesh(3.0, 1.2)
    m = oracle.Mesh([Cell(x, t, x, 1.0, 10.0, 0.5)])
    F = cp.top_force(x, 5.0, np.full(len(x), 10.0), m.vert_ranges)
    assert F[0] == 0.0


def test_relaxation_decreases_total_energy():
    """Gradient flow with a small step: elastic + plate energy never rises."""
    x, t = sphere_tet_mesh(3.0, 1.2)
    m = oracle.Mesh([Cell(x, t, x, 1.0, 10.0, 0.5)])
    y = perturb(x, 0.1, 4)
    zl, zh = np.full(len(x), -3.0), np.full(len(x), 2.0)
    E = lambda y: m.energy(y) + cp.plate_energy(y, 10.0, zl, zh)  # noqa: E731
    e = E(y)
    for _ in range(50):
        y, _ = cp.relax(m, y, 1, 0.004 ** 0.5, 10.0, [-3.0], [2.0])
        e2 = E(y)
        assert e2 <= e + 1e-12
        e = e2


def test_compressed_cell_pushes_back():
    """A compressed cell pushes the top plate harder at larger strain."""
    x, t = sphere_tet_mesh(3.0, 1.2)
    m = oracle.Mesh([Cell(x, t, x, 1.0, 10.0, 0.5)])
    F, _ = cp.protocol(m, x, [x[:, 2].min()], [3.0], [0.1, 0.3], 200, 0.004 ** 0.5, 20.0)
    assert 0 < F[0, 0] < F[0, 1]
