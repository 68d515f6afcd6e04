"""GPU: population storage formats.

* Row-edge shapes (nx = 2; a partial block; two blocks per row) in FP32 and
  FP16 (in FP16 the pair form: nx = 2 is one pair whose x-neighbours are
  itself).
* FP16 / BF16 storage of the deviations f_q - w_q (power-of-two scaled,
  collide in FP32), rounded to nearest or stochastically (f16sr, bf16sr),
  against the FP64 oracle: velocity fields and the Taylor deformation of a
  sheared cell. The tolerances state the error of each format as measured on
  GB300 (velocity after 600 steps of a forced Couette start-up: FP16 3.6e-3,
  BF16 5.8e-2, FP16-SR 1.9e-4, BF16-SR 1.4e-3; D after 800 steps of a sheared
  cell: FP32 3.2e-6, FP16 2.7e-5, BF16 8.6e-3, FP16-SR 3.5e-6, BF16-SR
  1.4e-5; mean velocity of a weakly forced channel after 400 steps: FP16
  7.3e-3, BF16 6.7e-2, FP16-SR 2.0e-6, BF16-SR 9.2e-5). Every 16-bit format
  but round-to-nearest BF16 meets the 1e-3 relative bound on D; stochastic
  rounding removes the stagnation of sub-ULP increments.
* The steady Poiseuille profile at the magic tau (where the oracle is exact)
  by format, and round-to-nearest against stochastic rounding in a channel
  of height 128.
"""
import numpy as np
import pytest

import oracle
from oracle import analysis
from workloads.configs import Cell, Workload
from workloads.mesh import sphere_tet_mesh

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2003_03130_gb300 import build

    build.build()
    import paper_2003_03130_gb300 as P

    return P


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def fluid_run(P, fmt, nx, ny, nz, tau, lo, hi, g, steps, pairs=1):
    ctx = P.cf_create(0)
    P.cf_set_population_format(ctx, fmt)
    P.cf_set_launch_shape(ctx, {"pop_pairs": pairs})
    P.cf_lbm_init(ctx, nx, ny, nz, tau, lo, hi, g)
    P.cf_step(ctx, steps)
    return P.cf_get_velocity(ctx), P.cf_get_density(ctx)


def oracle_fluid(nx, ny, nz, tau, lo, hi, g, steps):
    fl = oracle.Fluid(nx, ny, nz, tau, lo, hi, g)
    for _ in range(steps):
        fl.step()
    return fl


@pytest.mark.parametrize("dims", [(2, 12, 3), (130, 10, 4), (256, 6, 2)])
def test_row_edge_shapes(P, dims):
    """FP32 at 1e-5 and FP16 at its storage error against the oracle."""
    nx, ny, nz = dims
    args = (0.9, -0.02, 0.03, (1e-5, 0.0, -3e-6), 150)
    u32, rho32 = fluid_run(P, "f32", nx, ny, nz, *args)
    fl = oracle_fluid(nx, ny, nz, *args)
    assert rel(u32, fl.u) <= 1e-5
    assert np.abs(rho32 - fl.rho).max() <= 1e-6
    u16, _ = fluid_run(P, "f16", nx, ny, nz, *args)
    assert rel(u16, fl.u) <= 5e-3


@pytest.mark.parametrize("pairs", [1, 0])
@pytest.mark.parametrize("fmt,tol", [("f16", 5e-3), ("bf16", 8e-2), ("f16sr", 5e-4), ("bf16sr", 4e-3)])
def test_reduced_precision_fluid(P, fmt, tol, pairs):
    """Both forms of the 16-bit stream-collide (two nodes per thread with
    packed arithmetic, and one node per thread) at the format's error."""
    args = (16, 24, 8, 0.8, -0.02, 0.02, (2e-6, 0.0, 0.0), 600)
    u, rho = fluid_run(P, fmt, *args, pairs=pairs)
    fl = oracle_fluid(*args)
    err = rel(u, fl.u)
    print(f"{fmt} pairs={pairs}: relative velocity error {err:.2e}")
    assert err <= tol
    assert abs((rho - 1.0).sum()) <= 1e-3 * rho.size ** 0.5


def poiseuille_by_format(P, fmt, H=32, u_max=0.02, steps=12000):
    """Body-force channel of height H at the magic tau = 1/2 + sqrt(3)/4,
    where BGK with halfway bounce-back is exact (the oracle's pin): steady
    profile against u(y) = g/(2 nu) (y + 1/2)(H - y - 1/2). 12,000 steps are
    17 decay times H^2 / (pi^2 nu) of the slowest mode."""
    tau = 0.5 + np.sqrt(3) / 4
    nu = (tau - 0.5) / 3
    g = 8 * nu * u_max / H**2
    u, _ = fluid_run(P, fmt, 4, H, 4, tau, 0.0, 0.0, (g, 0.0, 0.0), steps)
    y = np.arange(H)
    exact = g / (2 * nu) * (y + 0.5) * (H - y - 0.5)
    prof = u[:, :, :, 0].mean(axis=(0, 2))
    spread = np.abs(u[:, :, :, 0] - prof[None, :, None]).max()  # the flow is uniform in x and z
    return rel(prof, exact), spread / u_max


@pytest.mark.parametrize("fmt,tol", [("f32", 3e-4), ("f16sr", 2e-3), ("bf16sr", 2e-2)])
def test_poiseuille_profile_by_format(P, fmt, tol):
    """FP32 meets the exact profile to its accumulated rounding (the same
    algorithm emulated in FP64 ends 6e-8 from it, in FP32 3e-5; the GPU's
    FP32 operation order measured 9e-5); stochastic rounding keeps the 16-bit
    formats within a few units of their last place (2^-11 FP16, 2^-8 BF16)."""
    err, spread = poiseuille_by_format(P, fmt)
    print(f"{fmt}: Poiseuille profile error {err:.2e}, spread across x and z {spread:.1e}")
    assert err <= tol
    assert spread <= tol


def test_stochastic_rounding_beats_nearest_in_a_wide_channel(P):
    """In a channel of height 128 (u_max 0.02) the per-step increments of the
    slow start-up fall below half an FP16 unit of the stored populations:
    round-to-nearest loses them, stochastic rounding keeps them in
    expectation. Profiles after 20,000 steps against FP32's."""
    H, tau = 128, 1.0
    nu = (tau - 0.5) / 3
    g = 8 * nu * 0.02 / H**2
    prof = {}
    for fmt in ("f32", "f16", "f16sr"):
        u, _ = fluid_run(P, fmt, 4, H, 4, tau, 0.0, 0.0, (g, 0.0, 0.0), 20000)
        prof[fmt] = u[:, :, :, 0].mean(axis=(0, 2))
    e_rn, e_sr = rel(prof["f16"], prof["f32"]), rel(prof["f16sr"], prof["f32"])
    print(f"profile vs FP32 after 20,000 steps: f16 {e_rn:.2e}, f16sr {e_sr:.2e}")
    assert e_sr <= 1e-3
    assert e_sr < e_rn


def sheared_cell():
    """R = 6 cell at the centre of a 32^3 box, walls -/+0.04 (shear rate
    2.5e-3), Ca = 0.2 with w = 0.5, kappa = 20 mu."""
    x, t = sphere_tet_mesh(6.0, 1.2)
    x = x + 15.5
    gamma = 2 * 0.04 / 32
    mu = (0.5 / 3) * gamma / 0.2
    return Workload("shear_32^3_R6", 32, 32, 32, 1.0, -0.04, 0.04,
                    cells=[Cell(x, t, x.copy(), mu, 20 * mu, 0.5)])


@pytest.fixture(scope="module")
def sheared_oracle():
    wl = sheared_cell()
    sim = oracle.Coupled(wl)
    sim.step(800)
    return wl, sim.y.copy(), analysis.taylor(sim.y, sim.mesh.tets)["D"]


@pytest.mark.parametrize("fmt,tol", [("f32", 1e-5), ("f16", 1e-3), ("bf16", 2e-2), ("f16sr", 2e-5), ("bf16sr", 2e-4)])
def test_taylor_deformation_by_format(P, sheared_oracle, fmt, tol):
    wl, y_ref, D_ref = sheared_oracle
    ctx = P.cf_create(0)
    P.cf_set_population_format(ctx, fmt)
    (cid,) = P.load_workload(ctx, wl)
    P.cf_step(ctx, 800)
    y = P.cf_get_positions(ctx, cid)
    D = analysis.taylor(y, oracle.Mesh(wl.cells).tets)["D"]
    x0 = wl.cells[0].x_ref
    print(f"{fmt}: D {D:.6f} (oracle {D_ref:.6f}), rel err D {abs(D - D_ref) / D_ref:.2e}, "
          f"displacement {rel(y - x0, y_ref - x0):.2e}")
    assert D_ref > 0.02
    assert abs(D - D_ref) <= tol * D_ref


@pytest.mark.parametrize("fmt,tol", [("f16", 1e-3), ("f16sr", 2e-5), ("bf16sr", 2e-4)])
@pytest.mark.parametrize("near_rows", [0, 1])
def test_taylor_deformation_pair_and_single_forms(P, sheared_oracle, fmt, tol, near_rows):
    """The sheared cell with the 16-bit stream-collide in both forms (node
    pairs / one node per thread) and both near-field forms (tile list / rows
    over the lattice, the row form also in pairs): every far, near and
    whole-lattice launch path of the 16-bit formats against the oracle."""
    wl, y_ref, D_ref = sheared_oracle
    for pairs in (1, 0):
        ctx = P.cf_create(0)
        P.cf_set_population_format(ctx, fmt)
        P.cf_set_launch_shape(ctx, {"pop_pairs": pairs, "near_rows": near_rows})
        (cid,) = P.load_workload(ctx, wl)
        P.cf_step(ctx, 800)
        y = P.cf_get_positions(ctx, cid)
        D = analysis.taylor(y, oracle.Mesh(wl.cells).tets)["D"]
        print(f"{fmt} pairs={pairs} near_rows={near_rows}: rel err D {abs(D - D_ref) / D_ref:.2e}")
        assert abs(D - D_ref) <= tol * D_ref
        P.cf_destroy(ctx)


@pytest.fixture(scope="module")
def channel_oracle():
    """The precision workload at full size (256 x 128 x 128 channel with a
    body force, one R = 16 cell off the centre plane), 30 coupled steps of
    the FP64 oracle from rest."""
    from workloads import configs

    wl = configs.precision_channel()
    sim = oracle.Coupled(wl)
    sim.step(30)
    return wl, sim.y.copy(), sim.fluid.u.copy()


@pytest.mark.parametrize("fmt,tol_u,tol_y", [("f32", 1e-5, 1e-5), ("f16", 3e-3, 3e-3), ("f16sr", 6e-4, 1e-4),
                                             ("bf16", 2e-2, 2e-2), ("bf16sr", 4e-3, 5e-4)])
def test_precision_channel_full_size_by_format(P, channel_oracle, fmt, tol_u, tol_y):
    """Every storage format on the full-size precision workload against the
    FP64 oracle (not against FP32): velocity field, the velocity on the
    nodes around the cell and the cell's displacement after 30 steps.
    Measured on GB300 (field / near the cell / displacement): FP32 4.4e-7 /
    2.7e-7 / 2.6e-7; FP16 6.9e-4 / 1.1e-3 / 9.8e-4; FP16-SR 2.1e-4 / 1.4e-4 /
    2.0e-5; BF16 4.1e-3 / 7.3e-3 / 5.7e-3; BF16-SR 1.4e-3 / 7.9e-4 / 1.6e-4.
    The 16-bit bounds are about three times those."""
    wl, y_ref, u_ref = channel_oracle
    ctx = P.cf_create(0)
    P.cf_set_population_format(ctx, fmt)
    (cid,) = P.load_workload(ctx, wl)
    P.cf_step(ctx, 30)
    y, u = P.cf_get_positions(ctx, cid), P.cf_get_velocity(ctx)
    P.cf_destroy(ctx)
    x0 = wl.cells[0].y0
    near = np.zeros(wl.nx * wl.ny * wl.nz, bool)
    b = np.floor(y_ref).astype(np.int64) - 1
    for dz in range(4):
        for dy in range(4):
            for dx in range(4):
                near[((b[:, 0] + dx) % wl.nx) + wl.nx * ((b[:, 1] + dy) + wl.ny * ((b[:, 2] + dz) % wl.nz))] = True
    e_u = rel(u, u_ref)
    e_near = rel(u.reshape(-1, 3)[near], u_ref.reshape(-1, 3)[near])
    e_y = rel(y - x0, y_ref - x0)
    print(f"{fmt}: velocity {e_u:.2e}, near the cell {e_near:.2e}, displacement {e_y:.2e}")
    assert e_u <= tol_u
    assert e_near <= tol_u
    assert e_y <= tol_y


def test_stochastic_rounding_keeps_small_increments(P):
    """A weak body force in a channel at rest: per step each population
    changes by far less than half an FP16 unit in the last place, so
    round-to-nearest stores lose the increments and the flow stagnates;
    stochastic rounding keeps them on average. Mean x velocity after 400
    steps against the FP64 oracle."""
    args = (16, 48, 8, 1.0, 0.0, 0.0, (2e-7, 0.0, 0.0), 400)
    fl = oracle_fluid(*args)
    ref = fl.u[..., 0].mean()
    errs = {}
    for fmt in ("f32", "f16", "f16sr", "bf16", "bf16sr"):
        u, _ = fluid_run(P, fmt, *args)
        errs[fmt] = abs(u[..., 0].mean() - ref) / abs(ref)
    print("relative error of the mean velocity:", {k: f"{v:.2e}" for k, v in errs.items()})
    assert errs["f32"] <= 1e-5
    assert errs["f16sr"] <= 1e-4 and errs["bf16sr"] <= 1e-3
    assert errs["f16sr"] <= errs["f16"] / 20 and errs["bf16sr"] <= errs["bf16"] / 20


def test_stochastic_rounding_is_reproducible_and_seeded_per_step(P):
    """The same run twice gives the same result (the rounding bits come from
    a hash of node, direction and a per-step seed); the seed advances every
    step, also across separate cf_step calls."""
    args = (16, 24, 8, 0.8, -0.02, 0.02, (2e-6, 0.0, 0.0))
    for pairs in (1, 0):
        runs = []
        for split in ((300,), (100, 1, 199)):
            ctx = P.cf_create(0)
            P.cf_set_population_format(ctx, "f16sr")
            P.cf_set_launch_shape(ctx, {"pop_pairs": pairs})
            P.cf_lbm_init(ctx, *args)
            for n in split:
                P.cf_step(ctx, n)
            runs.append(P.cf_get_velocity(ctx))
        assert np.array_equal(runs[0], runs[1])


def test_format_is_validated(P):
    from paper_2003_03130_gb300 import CellFSIError

    ctx = P.cf_create(0)
    for bad in (5, 7, -1):
        with pytest.raises(CellFSIError) as e:
            P.cf_set_population_format(ctx, bad)
        assert e.value.name == "CF_EINVAL"
