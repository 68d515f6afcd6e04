"""GPU: the deterministic spread (cf_set_spread(ctx, CF_SPREAD_FIXED)).

The force field is accumulated in 64-bit fixed point, so the order of the
spread's atomics no longer matters: the same workload must give bit-identical
cell positions and fluid populations (compared through the density, which
is read from the populations alone) whatever the launch shape (tile shape,
block sizes, near-field form, where the region is marked, fused or separate
cell chain, eight threads or one per vertex in the interpolation) and
whatever the schedule (pipelined steps, one step per call,
the profiled path). The velocity readback takes u(t) from the near field on
the last step's force region and from the populations elsewhere, two
roundings of the same value, so where the regions differ it agrees to
rounding only. The fixed-point field must still meet the oracle at the
usual 1e-5.
"""
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


def ragged_two_cells(delta=2):
    cells = []
    for centre, R, h, mu, kappa, w, seed in (((9.3, 8.7, 10.1), 4.0, 1.3, 2e-3, 0.1, 0.7, 5),
                                             ((28.2, 17.4, 7.9), 3.5, 1.2, 1e-3, 0.3, 0.2, 6)):
        x, t = sphere_tet_mesh(R, h)
        x = x + np.asarray(centre)
        cells.append(Cell(x, t, perturb(x, 0.1, seed), mu, kappa, w))
    return Workload("ragged", 41, 27, 19, 0.9, -0.015, 0.02, body_force=(2e-6, 0.0, -1e-6), cells=cells,
                    delta=delta)


SHAPES = [
    {},
    {"tile_x": 32, "tile_y": 2, "tile_z": 4, "near_rows": 1, "tet_block": 256, "gather_block": 64,
     "interp_block": 256},
    {"tile_x": 8, "tile_y": 8, "tile_z": 4, "mark_k5": 1, "far_spec": 1, "pop_l2": 1},
    {"tile_x": 32, "tile_y": 4, "tile_z": 2, "fused": 1},
    {"interp_form": 1, "interp_block": 64},
    {"interp_form": 1, "mark_k5": 1, "tile_x": 32, "tile_y": 2, "tile_z": 4},
]


def run(P, wl, steps, shape=None, mode="pipelined", spread="fixed", fmt="f32"):
    ctx = P.cf_create(0)
    P.cf_set_spread(ctx, spread)
    P.cf_set_population_format(ctx, fmt)
    if shape:
        P.cf_set_launch_shape(ctx, shape)
    ids = P.load_workload(ctx, wl)
    if mode == "pipelined":
        P.cf_step(ctx, steps)
    elif mode == "split":  # two calls of odd lengths, each one graph
        P.cf_step(ctx, 17)
        P.cf_step(ctx, steps - 17)
    elif mode == "single":
        for _ in range(steps):
            P.cf_step(ctx, 1)
    else:
        P.cf_step_profiled(ctx, steps)
    y = np.concatenate([P.cf_get_positions(ctx, i) for i in ids])
    u = P.cf_get_velocity(ctx)
    rho = P.cf_get_density(ctx)
    P.cf_destroy(ctx)
    return y, u, rho


def same_state(a, b, utol=1e-6):
    """Bit-identical positions and populations; velocities to rounding (of
    FP32, or of the 16-bit storage, whose populations give the readback
    outside the force region)."""
    assert np.array_equal(a[0], b[0])
    assert np.array_equal(a[2], b[2])
    assert rel(a[1], b[1]) <= utol


def test_fixed_spread_matches_oracle(P):
    wl = configs.small_shear()
    y, u, _ = run(P, wl, 100)
    sim = oracle.Coupled(wl)
    sim.step(100)
    y0 = wl.cells[0].y0
    assert rel(y - y0, sim.y - y0) <= TOL
    assert rel(u, sim.fluid.u) <= TOL


@pytest.mark.parametrize("delta", [2, 4])
def test_fixed_spread_is_bit_identical_across_launch_shapes(P, delta):
    """Two cells, body force, ragged box: every shape gives the same bits
    (and the oracle's result within 1e-5)."""
    wl = ragged_two_cells(delta)
    runs = [run(P, wl, 30, shape) for shape in SHAPES]
    for r in runs[1:]:
        same_state(r, runs[0])
    sim = oracle.Coupled(wl)
    sim.step(30)
    y0 = np.concatenate([c.y0 for c in wl.cells])
    assert rel(runs[0][0] - y0, sim.y - y0) <= TOL
    assert rel(runs[0][1], sim.fluid.u) <= TOL


def test_fixed_spread_is_bit_identical_across_schedules(P):
    """40 steps as one call (the first step, three 12-step graphs, a 3-step
    remainder and the last K5), as calls of 17 and 23 steps (one graph each),
    one step per call, and the profiled path."""
    wl = configs.small_shear()
    a = run(P, wl, 40, mode="pipelined")
    for mode in ("split", "single", "profiled"):
        same_state(run(P, wl, 40, mode=mode), a)


def test_fixed_spread_with_stochastic_rounding_is_bit_identical(P):
    """16-bit storage with stochastic rounding (the rounding bits come from a
    hash of node, direction and step) and the fixed-point spread: the whole
    coupled run repeats bit for bit under another tile shape. Both runs take
    every node through the same collide: the node-pair form in the far field
    and in the row-form near field (the packed collide rounds differently
    from the one-node form, so mixing the forms differently would not)."""
    wl = configs.small_shear()
    a = run(P, wl, 40, shape={"near_rows": 1, "pop_pairs": 1}, fmt="f16sr")
    b = run(P, wl, 40, shape={"tile_x": 32, "tile_y": 2, "tile_z": 4, "near_rows": 1, "pop_pairs": 1},
            fmt="f16sr")
    same_state(a, b, utol=1e-4)


def test_fixed_spread_full_size_long_run_repeats(P):
    """The production shear at full size (128^3, R = 16 cell, Ca = 0.2) for
    5,000 steps in two launch shapes (the default, and 32 x 2 x 4 tiles with
    the near field in rows, L2-cached populations and the one-thread
    interpolation): identical positions and populations after 5,000 steps,
    where float atomics let runs drift apart."""
    wl = configs.production_shear(ca=0.2, w=0.5)
    a = run(P, wl, 5000)
    b = run(P, wl, 5000, {"tile_x": 32, "tile_y": 2, "tile_z": 4, "near_rows": 1, "pop_l2": 1,
                          "interp_form": 1})
    same_state(a, b)
    y0 = wl.cells[0].y0
    assert np.abs(a[0] - y0).max() > 0.5  # the cell has moved and deformed


def test_spread_mode_is_validated(P):
    ctx = P.cf_create(0)
    with pytest.raises(P.CellFSIError) as e:
        P.cf_set_spread(ctx, 2)
    assert e.value.name == "CF_EINVAL"
    P.cf_destroy(ctx)
