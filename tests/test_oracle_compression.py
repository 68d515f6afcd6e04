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


# ---------------------------------------------------------------- damped relaxation dynamics
#
# Pins of relax() against what does not depend on its code: a closed form of
# the two-step recurrence for a linear force, and the force balance its
# fixed point must satisfy whatever the damping and step.


def _free_cell(R=3.0, h=1.2):
    """A cell with zero moduli: its elastic force vanishes at any shape, so
    only the plate acts and every vertex moves on its own."""
    x, t = sphere_tet_mesh(R, h)
    return x, oracle.Mesh([Cell(x, t, x, 0.0, 0.0, 0.5)])


def _closed_form(e0, n, a, c):
    """e_n of e_{k+1} = (1 + c - a) e_k - c e_{k-1} with e_1 = (1 - a) e_0
    (unit mass, force -k e, a = k dt^2, at rest at step 0): the velocity
    update v_1 = dt f_0 = -dt k e_0 followed by the position update with the
    new velocity. Solved through the roots of r^2 - (1 + c - a) r + c = 0."""
    if c == 0.0:
        return e0 * (1.0 - a) ** n
    r1, r2 = np.roots([1.0, -(1.0 + c - a), c])
    A = (1.0 - a - r2) / (r1 - r2)
    return np.real(e0 * (A * r1**n + (1.0 - A) * r2**n))


def test_free_cell_has_zero_elastic_force():
    x, m = _free_cell()
    assert np.abs(m.forces(perturb(x, 0.2, 7))).max() == 0.0


def test_damped_relaxation_matches_closed_form_under_the_lower_plate():
    """Every vertex below the lower plate feels k (z_lo - z): a harmonic
    force with its rest at z_lo. The damped steps (force at the old
    positions, position update with the new velocity) then follow the
    closed form of the linear recurrence exactly; x and y never move."""
    x, m = _free_cell()
    k, dt = 50.0, 0.003
    a = k * dt * dt
    z_lo = float(x[:, 2].max()) + 0.5  # every vertex starts below the plate
    e0 = x[:, 2] - z_lo
    for c in (0.0, 0.95):
        for n in (1, 2, 3, 10, 400, 2000):
            ce = _closed_form(e0, n, a, c)
            assert (ce < 0).all()  # never reaches the plate: the force stays on
            y, v = cp.relax(m, x.copy(), n, dt, k, [z_lo], [z_lo + 100.0], c=c)
            assert np.array_equal(y[:, :2], x[:, :2])
            np.testing.assert_allclose(y[:, 2] - z_lo, ce, rtol=1e-11, atol=1e-13)
            # velocity of the last step: (e_n - e_{n-1}) / dt
            cp_prev = _closed_form(e0, n - 1, a, c)
            np.testing.assert_allclose(v[:, 2], (ce - cp_prev) / dt, rtol=1e-9, atol=1e-12)


def test_damped_relaxation_continues_from_its_state():
    """n steps in one call equal n1 + n2 steps in two calls that hand over
    positions and velocities."""
    x, t = sphere_tet_mesh(3.0, 1.2)
    m = oracle.Mesh([Cell(x, t, x, 1.0, 10.0, 0.5)])
    zl, zh = [x[:, 2].min()], [x[:, 2].max() - 1.0]
    y0 = perturb(x, 0.05, 11)
    ya, va = cp.relax(m, y0, 30, 0.03, 20.0, zl, zh, c=0.95)
    y1, v1 = cp.relax(m, y0, 12, 0.03, 20.0, zl, zh, c=0.95)
    yb, vb = cp.relax(m, y1, 18, 0.03, 20.0, zl, zh, v=v1, c=0.95)
    assert np.array_equal(ya, yb) and np.array_equal(va, vb)


def _relax_to_rest(m, y, dt, c, zl, zh, k=20.0, tol=1e-11, max_steps=40000):
    zlv, zhv = cp.per_vertex(zl, m.vert_ranges), cp.per_vertex(zh, m.vert_ranges)
    v, n = None, 0
    while n < max_steps:
        y, v = cp.relax(m, y, 500, dt, k, zl, zh, v=v, c=c)
        n += 500
        r = np.abs(m.forces(y) + cp.plate_forces(y, k, zlv, zhv)).max()
        if r < tol:
            return y
    raise AssertionError(f"no rest after {n} steps (residual {r:.2e})")


def test_relaxation_rests_in_the_same_force_balance_for_every_damping_and_step():
    """The fixed point of the damped steps is f_el + f_plate = 0, whatever c
    and dt: gradient flow (c = 0) and two damped forms reach the same
    compressed shape. The shape is compared through what the plate problem
    fixes: the elastic energy, the plate forces, every z coordinate and every
    vertex distance (a translation in x-y or a turn about z costs nothing)."""
    from scipy.spatial.distance import pdist

    x, t = sphere_tet_mesh(3.0, 1.2)
    m = oracle.Mesh([Cell(x, t, x, 1.0, 10.0, 0.5)])
    zl = [float(x[:, 2].min())]
    zh = [zl[0] + 0.7 * float(x[:, 2].max() - x[:, 2].min())]  # 30 % strain
    rests = [_relax_to_rest(m, x.copy(), dt, c, zl, zh) for c, dt in ((0.0, 0.08), (0.95, 0.03), (0.9, 0.05))]
    ref = rests[0]
    zlv, zhv = cp.per_vertex(zl, m.vert_ranges), cp.per_vertex(zh, m.vert_ranges)
    for y in rests[1:]:
        assert np.abs(y[:, 2] - ref[:, 2]).max() < 1e-8
        assert np.abs(pdist(y) - pdist(ref)).max() < 1e-8
        assert abs(m.energy(y) - m.energy(ref)) < 1e-8 * abs(m.energy(ref))
        assert abs(cp.top_force(y, 20.0, zhv, m.vert_ranges)[0] -
                   cp.top_force(ref, 20.0, zhv, m.vert_ranges)[0]) < 1e-8
    assert m.energy(ref) > 0 and cp.top_force(ref, 20.0, zhv, m.vert_ranges)[0] > 0


def test_each_cell_at_rest_pushes_both_plates_equally():
    """Internal forces sum to zero over a cell (Sec. 3.1: per-tet balance),
    so at rest the top plate's force on a cell equals the bottom plate's.
    Two cells of different moduli and heights, compressed to different
    strains, relaxed together."""
    x, t = sphere_tet_mesh(3.0, 1.2)
    x2 = x + np.array([10.0, 0.0, 0.5])
    m = oracle.Mesh([Cell(x, t, x, 1.0, 10.0, 0.5), Cell(x2, t, x2, 2.0, 30.0, 0.2)])
    y0 = np.concatenate([x, x2])
    zl = [float(x[:, 2].min()), float(x2[:, 2].min())]
    zh = [zl[0] + 4.2, zl[1] + 5.0]
    y = _relax_to_rest(m, y0, 0.03, 0.95, zl, zh)
    zlv, zhv = cp.per_vertex(zl, m.vert_ranges), cp.per_vertex(zh, m.vert_ranges)
    top = cp.top_force(y, 20.0, zhv, m.vert_ranges)
    bottom = np.array([(20.0 * np.maximum(zlv - y[:, 2], 0.0))[a:b].sum() for a, b in m.vert_ranges])
    assert (top > 0).all()
    np.testing.assert_allclose(top, bottom, rtol=1e-9)
    fel = m.forces(y)
    for a, b in m.vert_ranges:
        assert np.abs(fel[a:b].sum(0)).max() < 1e-9 * top.max()


# ---------------------------------------------------------------- plate schedule (input generator)

def test_plate_schedule_levels_and_ramp():
    """Per level the step counts add up to ``steps``, the level ends at
    z_lo + 2 R (1 - s), the plate only moves down, and each move is an equal
    share of the level's travel."""
    from workloads.configs import plate_schedule

    z_lo, R = np.array([0.0, 5.0]), np.array([10.0, 6.0])
    strains, steps = [0.1, 0.25, 0.8], 2000
    for ramp in (0, 1, 4, 10):
        sched = list(plate_schedule(z_lo, R, strains, steps, ramp))
        assert len(sched) == len(strains) * (ramp + 1)
        prev = z_lo + 2 * R
        for lv, s in enumerate(strains):
            level = sched[lv * (ramp + 1):(lv + 1) * (ramp + 1)]
            assert sum(n for _, n, _ in level) == steps
            assert [m for _, _, m in level] == [False] * ramp + [True]
            end = z_lo + 2 * R * (1 - s)
            np.testing.assert_allclose(level[-1][0], end, rtol=0, atol=1e-12)
            heights = [prev] + [z for z, _, _ in level]
            for a, b in zip(heights, heights[1:]):
                assert (b <= a + 1e-12).all()
            if ramp:
                moves = np.diff(np.array(heights[:ramp + 1]), axis=0)
                np.testing.assert_allclose(moves, np.broadcast_to((end - prev) / ramp, moves.shape), atol=1e-12)
                assert all(n == steps // (2 * ramp) for _, n, _ in level[:-1])
            prev = end
