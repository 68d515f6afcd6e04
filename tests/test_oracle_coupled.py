"""Pins of the oracle's coupled cell/fluid step (Sec. 6; order t -> t+1:
forces at y^t, spread, LB step, interpolate u(t) at y^t, advect)."""
import numpy as np
import pytest

import oracle
from workloads.configs import Cell, Workload
from workloads.mesh import perturb, sphere_tet_mesh


def _wl(cells, n=24, uw=0.0, tau=1.0, delta=2):
    return Workload("t", n, n, n, tau, -uw, uw, cells=cells, delta=delta)


@pytest.mark.parametrize("delta", [2, 4])
def test_massless_tracer_cell_in_couette_moves_with_the_flow(delta):
    """A cell without stiffness in steady Couette flow: each vertex moves at
    the exact linear profile u_x = u_w (2 (y + 1/2)/H - 1) (interpolation is
    exact for linear fields and y never changes)."""
    H, uw = 16, 0.01
    x, t = sphere_tet_mesh(3.0, 1.2)
    x = x + np.array([8.0, 7.3, 6.0])
    sim = oracle.Coupled(_wl([Cell(x, t, x.copy(), 0.0, 0.0, 1.0)], n=H, uw=uw, delta=delta))
    for _ in range(1500):  # the fluid alone reaches steady Couette flow
        sim.fluid.step()
    y0 = sim.y.copy()
    sim.step(7)
    v = uw * (2 * (y0[:, 1] + 0.5) / H - 1)
    assert np.allclose(sim.y[:, 0], y0[:, 0] + 7 * v, rtol=0, atol=1e-12)
    assert np.allclose(sim.y[:, 1:], y0[:, 1:], rtol=0, atol=1e-12)


@pytest.mark.parametrize("delta", [2, 4])
def test_internal_forces_leave_fluid_momentum_unchanged(delta):
    """Elastic forces of a cell sum to zero, so the spread force adds no net
    momentum to the fluid."""
    x, t = sphere_tet_mesh(5.0, 1.3)
    x = x + 11.5
    y0 = perturb(x, 0.15, 1)
    sim = oracle.Coupled(_wl([Cell(x, t, y0, 5e-3, 0.3, 0.5)], delta=delta))
    for _ in range(4):
        sim.step()
        assert np.abs(sim.fluid.total_momentum()).max() < 1e-15 * len(sim.fluid.f.reshape(-1)) ** 0.5
        assert np.abs(sim.last_forces).max() > 1e-5


def test_perturbed_cell_relaxes_and_conserves_mass():
    x, t = sphere_tet_mesh(5.0, 1.3)
    x = x + 11.5
    y0 = perturb(x, 0.15, 2)
    sim = oracle.Coupled(_wl([Cell(x, t, y0, 5e-3, 0.3, 0.5)]))
    m0 = sim.fluid.total_mass()
    e0 = sim.mesh.energy(sim.y)
    sim.step(30)
    assert sim.mesh.energy(sim.y) < 0.5 * e0
    assert abs(sim.fluid.total_mass() - m0) < 1e-12 * m0
