"""GPU: materials per tet (a stiff nucleus, cytoplasm and a cortex shell in
one cell; Sec. 3.1: the force is local to each tet) against the FP64 oracle
through the C ABI, at the parity tolerance of the uniform path (1e-5)."""
import numpy as np
import pytest

import oracle
from workloads import configs
from workloads.configs import Cell, Workload
from workloads.mesh import perturb, shell_regions, sphere_tet_mesh

pytestmark = pytest.mark.gpu

TOL = 1e-5
MATS = [(8e-3, 0.6, 0.9), (1e-3, 0.1, 0.4), (3e-3, 0.3, 0.0)]  # nucleus, cytoplasm, cortex


@pytest.fixture(scope="module")
def P():
    from paper_2003_03130_gb300 import build

    build.build()
    import paper_2003_03130_gb300 as P

    return P


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def layered_cell(centre=(12.0, 12.0, 12.0), R=5.0, seed=4, noise=0.12):
    x, t = sphere_tet_mesh(R, 1.3)
    x = x + np.asarray(centre)
    c = Cell(x, t, perturb(x, noise, seed), 1e-3, 0.1, 0.5)
    c.regions = shell_regions(x, t, 0.45 * R, 0.8 * R)
    c.region_materials = MATS
    return c


def test_forces_and_energy_match_the_oracle(P):
    c = layered_cell()
    wl = Workload("layered", 24, 24, 24, 1.0, 0.0, 0.0, cells=[c])
    ctx = P.cf_create(0)
    (cid,) = P.load_workload(ctx, wl)
    P.cf_compute_forces(ctx)
    m = oracle.Mesh([c])
    assert rel(P.cf_get_forces(ctx, cid), m.forces(c.y0)) <= TOL
    assert abs(P.cf_get_energy(ctx, cid) - m.energy(c.y0)) <= 1e-5 * m.energy(c.y0)


def test_coupled_shear_with_a_nucleus(P):
    wl = configs.small_shear()
    c = wl.cells[0]
    c.regions = shell_regions(c.x_ref, c.tets, 3.5, 6.5)
    c.region_materials = [(4e-3, 0.3, 0.8), (1e-3, 0.1, 0.5), (2e-3, 0.2, 0.2)]
    ctx = P.cf_create(0)
    (cid,) = P.load_workload(ctx, wl)
    P.cf_step(ctx, 40)
    sim = oracle.Coupled(wl)
    sim.step(40)
    assert rel(P.cf_get_positions(ctx, cid) - c.y0, sim.y - c.y0) <= TOL
    assert rel(P.cf_get_forces(ctx, cid), sim.last_forces) <= TOL
    assert rel(P.cf_get_velocity(ctx), sim.fluid.u) <= TOL


def test_uniform_again_and_cells_added_later(P):
    """cf_set_material makes a layered cell uniform; a cell added after the
    per-tet materials keeps the first cell's regions (their slots move)."""
    a = layered_cell()
    b = layered_cell(centre=(30.0, 12.0, 12.0), R=4.0, seed=9)
    ctx = P.cf_create(0)
    P.cf_lbm_init(ctx, 44, 24, 24, 1.0, 0.0, 0.0)
    ia = P.cf_mesh_init(ctx, a.x_ref, a.tets, a.y0)
    P.cf_set_material(ctx, ia, a.mu, a.kappa, a.w)
    P.cf_set_tet_materials(ctx, ia, a.regions, *np.array(MATS).T)
    ib = P.cf_mesh_init(ctx, b.x_ref, b.tets, b.y0)
    P.cf_set_material(ctx, ib, 2e-3, 0.2, 0.7)
    P.cf_compute_forces(ctx)
    b_uni = Cell(b.x_ref, b.tets, b.y0, 2e-3, 0.2, 0.7)
    m = oracle.Mesh([a, b_uni])
    f = np.concatenate([P.cf_get_forces(ctx, ia), P.cf_get_forces(ctx, ib)])
    assert rel(f, m.forces(np.concatenate([a.y0, b.y0]))) <= TOL
    P.cf_set_material(ctx, ia, a.mu, a.kappa, a.w)
    P.cf_compute_forces(ctx)
    a_uni = Cell(a.x_ref, a.tets, a.y0, a.mu, a.kappa, a.w)
    assert rel(P.cf_get_forces(ctx, ia), oracle.Mesh([a_uni]).forces(a.y0)) <= TOL


def test_jvp_uses_regions_and_parameter_gradients_refuse(P):
    from paper_2003_03130_gb300 import CellFSIError

    c = layered_cell()
    ctx = P.cf_create(0)
    (cid,) = P.cf_mesh_init_batch(ctx, [c.x_ref], [c.tets], [c.y0])
    P.cf_set_material(ctx, cid, c.mu, c.kappa, c.w)
    P.cf_set_tet_materials(ctx, cid, c.regions, *np.array(MATS).T)
    m = oracle.Mesh([c])
    v = np.random.default_rng(2).normal(size=c.y0.shape)
    y = P.cf_get_positions(ctx, cid)
    h = 1e-5
    ref = (m.forces(y + h * v) - m.forces(y - h * v)) / (2 * h)
    assert rel(P.cf_force_jvp(ctx, v), ref) <= TOL
    with pytest.raises(CellFSIError) as e:
        P.cf_force_param_vjp(ctx, v)
    assert e.value.name == "CF_ESTATE"


def test_region_arguments_are_validated(P):
    from paper_2003_03130_gb300 import CellFSIError

    c = layered_cell()
    ctx = P.cf_create(0)
    cid = P.cf_mesh_init(ctx, c.x_ref, c.tets, c.y0)
    bad = c.regions.copy()
    bad[5] = 3
    cases = [(cid, bad, MATS), (cid + 1, c.regions, MATS), (cid, c.regions, [(1e-3, 0.1, 1.5)] * 3),
             (cid, c.regions, [(-1.0, 0.1, 0.5)] * 3)]
    for cell_id, reg, mats in cases:
        with pytest.raises(CellFSIError) as e:
            P.cf_set_tet_materials(ctx, cell_id, reg, *np.array(mats).T)
        assert e.value.name == "CF_EINVAL"
