"""GPU parity of the immersed-boundary coupling with Peskin's four-point
delta kernel (support width 4, 64 nodes per vertex) against the FP64
oracle, through the C ABI. Same tolerance as the trilinear path: norm-wise
relative error <= 1e-5 on displacements, forces and fluid velocities."""
import numpy as np
import pytest

import oracle
from workloads import configs
from workloads.configs import Cell, Workload
from workloads.mesh import perturb, sphere_tet_mesh

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def P():
    from paper_2003_03130_gb300 import build

    build.build()
    import paper_2003_03130_gb300 as P

    return P


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def cell_at(centre, R=4.0, h=1.3, mu=2e-3, kappa=0.2, w=0.6, seed=8):
    x, t = sphere_tet_mesh(R, h)
    x = x + np.asarray(centre)
    return Cell(x, t, perturb(x, 0.1, seed), mu, kappa, w)


def pair(P, wl, steps, mode="pipelined", shape=None):
    ctx = P.cf_create(0)
    if shape:
        P.cf_set_launch_shape(ctx, shape)
    ids = P.load_workload(ctx, wl)
    if mode == "pipelined":
        P.cf_step(ctx, steps)
    elif mode == "single":
        for _ in range(steps):
            P.cf_step(ctx, 1)
    else:
        P.cf_step_profiled(ctx, steps)
    sim = oracle.Coupled(wl)
    sim.step(steps)
    y = np.concatenate([P.cf_get_positions(ctx, i) for i in ids])
    f = np.concatenate([P.cf_get_forces(ctx, i) for i in ids])
    return ctx, sim, y, f


@pytest.mark.parametrize("staged", [0, 1])
def test_small_shear_peskin(P, staged):
    """Both spread forms: one atomic per vertex and node, and the
    shared-memory staged spread."""
    wl = configs.small_shear()
    wl.delta = 4
    y0 = wl.cells[0].y0
    ctx, sim, y, f = pair(P, wl, 60, shape={"staged": staged})
    assert rel(y - y0, sim.y - y0) <= TOL
    assert rel(f, sim.last_forces) <= TOL
    assert rel(P.cf_get_velocity(ctx), sim.fluid.u) <= TOL


@pytest.mark.parametrize("mode", ["single", "profiled", "interp1"])
def test_peskin_every_launch_path(P, mode):
    """One-step graphs and plain launches clear and rebuild the 64-node
    supports the same way as the pipelined graphs; the 64-node
    interpolation in one thread per vertex (interp1)."""
    wl = configs.small_shear()
    wl.delta = 4
    y0 = wl.cells[0].y0
    if mode == "interp1":
        ctx, sim, y, _ = pair(P, wl, 20, "pipelined", shape={"interp_form": 1})
    else:
        ctx, sim, y, _ = pair(P, wl, 20, mode)
    assert rel(y - y0, sim.y - y0) <= TOL
    assert rel(P.cf_get_velocity(ctx), sim.fluid.u) <= TOL


@pytest.mark.parametrize("staged", [0, 1])
def test_peskin_across_the_periodic_seam(P, staged):
    """The staged spread's box is in unwrapped coordinates; its flush wraps
    across the seams."""
    cell = cell_at((0.3, 12.0, 23.6))
    wl = Workload("seam", 24, 24, 24, 1.0, -0.02, 0.02, cells=[cell], delta=4)
    ctx, sim, y, _ = pair(P, wl, 25, shape={"staged": staged})
    assert rel(y - cell.y0, sim.y - cell.y0) <= TOL
    assert rel(P.cf_get_velocity(ctx), sim.fluid.u) <= TOL


@pytest.mark.parametrize("staged", [0, 1])
def test_peskin_ragged_box_two_cells_body_force(P, staged):
    """Two cells: the staged spread's block that holds vertices of both has a
    box too large for shared memory and takes the global atomics."""
    cells = [cell_at((9.3, 8.7, 10.1), w=0.7, seed=5),
             cell_at((28.2, 17.4, 7.9), R=3.5, h=1.2, mu=1e-3, kappa=0.3, w=0.2, seed=6)]
    wl = Workload("ragged", 41, 27, 19, 0.9, -0.015, 0.02, body_force=(2e-6, 0.0, -1e-6), cells=cells, delta=4)
    y0 = np.concatenate([c.y0 for c in cells])
    ctx, sim, y, f = pair(P, wl, 40, shape={"staged": staged})
    assert rel(y - y0, sim.y - y0) <= TOL
    assert rel(f, sim.last_forces) <= TOL
    assert rel(P.cf_get_velocity(ctx), sim.fluid.u) <= TOL


@pytest.mark.parametrize("staged", [0, 1])
def test_peskin_production_shear_full_size(P, staged):
    """128^3, R = 16 cell (~20k tets) in the benchmark's launch configuration,
    both spread forms."""
    wl = configs.production_shear(ca=0.2, w=0.5)
    wl.delta = 4
    cell = wl.cells[0]
    cell.y0 = perturb(cell.x_ref, 0.08, 20030313)
    y0 = cell.y0.copy()
    ctx, sim, y, f = pair(P, wl, 3, shape={"staged": staged})
    assert rel(y - y0, sim.y - y0) <= TOL
    assert rel(f, sim.last_forces) <= TOL
    assert rel(P.cf_get_velocity(ctx), sim.fluid.u) <= TOL


def test_wider_support_reaches_the_wall(P):
    """A vertex at y = 0.6 has its trilinear support in rows 0..1 but its
    four-point support needs row -1: the same cell runs with one kernel and
    reports CF_EDOMAIN with the other."""
    from paper_2003_03130_gb300 import CellFSIError

    x, t = sphere_tet_mesh(3.0, 1.2)
    x = x + np.array([8.0, 3.6 - x[:, 1].min() - 3.0, 8.0])
    assert abs(x[:, 1].min() - 0.6) < 1e-12
    for kernel, ok in (("trilinear", True), ("peskin4", False)):
        ctx = P.cf_create(0)
        P.cf_set_delta(ctx, kernel)
        P.cf_lbm_init(ctx, 16, 16, 16, 1.0, 0.0, 0.0)
        cid = P.cf_mesh_init(ctx, x, t)
        P.cf_set_material(ctx, cid, 1e-3, 0.1, 0.5)
        if ok:
            P.cf_step(ctx, 2)
        else:
            with pytest.raises(CellFSIError) as e:
                P.cf_step(ctx, 2)
            assert e.value.name == "CF_EDOMAIN"
        P.cf_destroy(ctx)


def test_set_delta_validates(P):
    from paper_2003_03130_gb300 import CellFSIError

    ctx = P.cf_create(0)
    for bad in (0, 1, 3, 6):
        with pytest.raises(CellFSIError) as e:
            P.cf_set_delta(ctx, bad)
        assert e.value.name == "CF_EINVAL"
    P.cf_set_delta(ctx, "peskin4")
    P.cf_destroy(ctx)
