"""GPU: launch shapes and the autotuner. Every tile shape and block size
must give the oracle's result (the same tolerance as the default shape),
the autotuner must advance the state exactly like cf_step, and invalid
shapes are status codes."""
import numpy as np
import pytest

import oracle
from workloads import configs
from workloads.configs import Cell, Workload
from workloads.mesh import perturb, sphere_tet_mesh

pytestmark = pytest.mark.gpu

TOL = 1e-5
TILES = [(16, 4, 4), (32, 4, 2), (32, 2, 4), (8, 8, 4)]


@pytest.fixture(scope="module")
def P():
    from paper_2003_03130_gb300 import build

    build.build()
    import paper_2003_03130_gb300 as P

    return P


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def reference_20():
    wl = configs.small_shear()
    sim = oracle.Coupled(wl)
    sim.step(20)
    return wl, sim


@pytest.mark.parametrize("tile", TILES)
@pytest.mark.parametrize("blocks", [(64, 128, 128, 0, 0, 1, 1, 1, 1, 0, 0, 1), (256, 64, 256, 0, 1, 0, 0, 0, 0, 1, 1, 1),
                                    (128, 256, 64, 1, 0, 1, 1, 1, 1, 1, 0, 0), (64, 128, 256, 0, 1, 1, 2, 0, 1, 1, 1, 0),
                                    (256, 128, 64, 0, 0, 0, 2, 1, 0, 0, 1, 1), (128, 64, 128, 1, 1, 0, 0, 0, 1, 0, 0, 0)])
def test_every_shape_matches_the_oracle(P, reference_20, tile, blocks):
    wl, sim = reference_20
    ctx = P.cf_create(0)
    P.cf_set_launch_shape(ctx, list(tile) + list(blocks))
    (cid,) = P.load_workload(ctx, wl)
    got = P.cf_get_launch_shape(ctx)
    assert [got[k] for k in P.SHAPE_KEYS] == list(tile) + list(blocks)
    P.cf_step(ctx, 12)
    P.cf_step_profiled(ctx, 3)
    P.cf_step(ctx, 5)
    y0 = wl.cells[0].y0
    assert rel(P.cf_get_positions(ctx, cid) - y0, sim.y - y0) <= TOL
    assert rel(P.cf_get_velocity(ctx), sim.fluid.u) <= TOL
    P.cf_destroy(ctx)


def test_shape_change_between_calls(P, reference_20):
    wl, sim = reference_20
    ctx = P.cf_create(0)
    (cid,) = P.load_workload(ctx, wl)
    for k, tile in enumerate(TILES):
        P.cf_set_launch_shape(ctx, {"tile_x": tile[0], "tile_y": tile[1], "tile_z": tile[2]})
        P.cf_step(ctx, 5)
    y0 = wl.cells[0].y0
    assert rel(P.cf_get_positions(ctx, cid) - y0, sim.y - y0) <= TOL
    assert rel(P.cf_get_velocity(ctx), sim.fluid.u) <= TOL


AUTOTUNE_CANDIDATES = 32  # every value of every knob (cf_autotune)


def test_autotune_advances_like_cf_step(P):
    """32 candidates x 2 steps = 64 steps, then 10 more with the chosen
    shape: positions and fluid as the oracle's after 74 steps."""
    cells = [Cell(*_cell((9.3, 8.7, 10.1), 5)), Cell(*_cell((28.2, 17.4, 7.9), 6, R=3.5, h=1.2))]
    wl = Workload("ragged", 41, 27, 19, 0.9, -0.015, 0.02, body_force=(2e-6, 0.0, -1e-6), cells=cells)
    ctx = P.cf_create(0)
    ids = P.load_workload(ctx, wl)
    shape = P.cf_autotune(ctx, 2)
    assert (shape["tile_x"], shape["tile_y"], shape["tile_z"]) in TILES
    assert shape["tet_block"] in (64, 128, 256) and shape["gather_block"] in (64, 128, 256)
    assert shape["interp_block"] in (64, 128, 256) and shape["fused"] in (0, 1) and shape["near_rows"] in (0, 1)
    assert shape["far_spec"] in (0, 1) and shape["tet_form"] in (0, 1, 2) and shape["pop_l2"] in (0, 1)
    assert shape["pop_pairs"] in (0, 1) and shape["mark_k5"] in (0, 1) and shape["staged"] in (0, 1)
    assert P.cf_get_launch_shape(ctx) == shape
    sim = oracle.Coupled(wl)
    sim.step(2 * AUTOTUNE_CANDIDATES)
    # the last timed candidate may have run another tiling than the chosen one
    assert rel(P.cf_get_velocity(ctx), sim.fluid.u) <= TOL
    P.cf_step(ctx, 10)
    sim.step(10)
    y0 = np.concatenate([c.y0 for c in cells])
    y = np.concatenate([P.cf_get_positions(ctx, i) for i in ids])
    assert rel(y - y0, sim.y - y0) <= TOL
    assert rel(P.cf_get_velocity(ctx), sim.fluid.u) <= TOL


def test_velocity_readback_after_a_tile_change(P, reference_20):
    """After a step the force field is consumed and u(t) on the step's force
    region comes from the near field's store, looked up in the tiling that
    step ran with, also when the shape changed since."""
    wl, sim = reference_20
    ctx = P.cf_create(0)
    P.cf_set_launch_shape(ctx, {"tile_x": 32, "tile_y": 2, "tile_z": 4})
    (cid,) = P.load_workload(ctx, wl)
    P.cf_step(ctx, 20)
    u20 = P.cf_get_velocity(ctx)
    assert rel(u20, sim.fluid.u) <= TOL
    for tile in ((8, 8, 4), (16, 4, 4)):
        P.cf_set_launch_shape(ctx, {"tile_x": tile[0], "tile_y": tile[1], "tile_z": tile[2]})
        assert np.array_equal(P.cf_get_velocity(ctx), u20)
    P.cf_destroy(ctx)


def _cell(centre, seed, R=4.0, h=1.3):
    x, t = sphere_tet_mesh(R, h)
    x = x + np.asarray(centre)
    return x, t, perturb(x, 0.1, seed), 2e-3, 0.1, 0.7


def test_autotune_without_cells_keeps_the_state(P):
    ctx = P.cf_create(0)
    P.cf_lbm_init(ctx, 16, 16, 8, 0.8, -0.02, 0.02)
    P.cf_step(ctx, 10)
    u = P.cf_get_velocity(ctx)
    P.cf_autotune(ctx, 3)
    assert np.array_equal(P.cf_get_velocity(ctx), u)


def test_seam_on_a_lattice_smaller_than_two_tiles(P):
    """nx = 20 with 16-node tiles: the last tile is partial and a support
    that crosses the x seam meets both tiles."""
    x, t = sphere_tet_mesh(4.0, 1.3)
    x = x + np.array([0.3, 12.0, 17.6])
    cell = Cell(x, t, perturb(x, 0.1, 8), 2e-3, 0.2, 0.6)
    wl = Workload("seam20", 20, 24, 18, 1.0, -0.02, 0.02, cells=[cell])
    ctx = P.cf_create(0)
    (cid,) = P.load_workload(ctx, wl)
    P.cf_step(ctx, 25)
    sim = oracle.Coupled(wl)
    sim.step(25)
    assert rel(P.cf_get_positions(ctx, cid) - cell.y0, sim.y - cell.y0) <= TOL
    assert rel(P.cf_get_velocity(ctx), sim.fluid.u) <= TOL
    _, near = P.cf_step_profiled(ctx, 1)
    assert 0 < near <= 20 * 24 * 18


def test_invalid_shapes_are_status_codes(P):
    from paper_2003_03130_gb300 import CellFSIError

    ctx = P.cf_create(0)
    good = [16, 4, 4, 64, 128, 128, 0, 0, 0, 0, 0, 1, 0, 0, 0]
    for k, bad in ((0, 64), (1, 8), (2, 2), (3, 48), (4, 512), (5, 0), (5, 288), (6, 2), (7, -1), (8, 3), (9, 3),
                   (9, -1), (10, 2), (11, 2), (12, -1), (13, 2), (14, 2), (14, -1)):
        shape = list(good)
        shape[k] = bad
        with pytest.raises(CellFSIError) as e:
            P.cf_set_launch_shape(ctx, shape)
        assert e.value.name == "CF_EINVAL"
    with pytest.raises(CellFSIError) as e:
        P.cf_autotune(ctx, 2)
    assert e.value.name == "CF_ESTATE"
    P.cf_lbm_init(ctx, 8, 8, 8, 1.0, 0.0, 0.0)
    with pytest.raises(CellFSIError) as e:
        P.cf_autotune(ctx, 0)
    assert e.value.name == "CF_EINVAL"
    P.cf_destroy(ctx)


def test_fused_chain_wait_runs_out_with_a_timeout_status(P):
    """The fused cell chain's waits are bounded. With every cell's required
    tet-item count raised out of reach (a host-side setting: nothing on the
    device ever meets it) and a limit of 1,000 polls, a step returns
    CF_ETIMEOUT promptly instead of hanging; with the defaults restored the
    same context steps again and its forces match the oracle."""
    import time

    wl = configs.small_shear()
    ctx = P.cf_create(0)
    (cid,) = P.load_workload(ctx, wl)
    P.cf_set_launch_shape(ctx, {"fused": 1})
    P.cf_step(ctx, 2)
    P.cf_set_chain_wait(ctx, 1000, 1)
    t0 = time.perf_counter()
    with pytest.raises(P.CellFSIError) as e:
        P.cf_step(ctx, 1)
    assert e.value.name == "CF_ETIMEOUT"
    assert time.perf_counter() - t0 < 5.0
    with pytest.raises(P.CellFSIError) as e:
        P.cf_set_chain_wait(ctx, 0, 0)
    assert e.value.name == "CF_EINVAL"
    P.cf_set_chain_wait(ctx)
    P.cf_set_positions(ctx, cid, wl.cells[0].y0)
    P.cf_step(ctx, 3)
    P.cf_compute_forces(ctx)
    y = P.cf_get_positions(ctx, cid)
    ref = oracle.Mesh(wl.cells).forces(y)
    assert rel(P.cf_get_forces(ctx, cid), ref) <= TOL
    P.cf_destroy(ctx)
