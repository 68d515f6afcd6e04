"""Pins of the oracle's tet mesh mechanics (Sec. 3.1-3.2): precompute of B and
V_0, orientation, vertex incidence rows, and the nodal forces on whole meshes.
"""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
from workloads.configs import Cell
from workloads.mesh import perturb, sphere_tet_mesh

RNG = np.random.default_rng(11)


def mesh_of(R=4.0, h=1.3, mu=1.0, kappa=5.0, w=0.5):
    x, t = sphere_tet_mesh(R, h)
    return oracle.Mesh([Cell(x, t, x.copy(), mu, kappa, w)])


@pytest.fixture(scope="module")
def m():
    return mesh_of()


def test_prepare_orients_and_inverts(m):
    e = m.x[m.tets[:, :3]] - m.x[m.tets[:, 3:4]]  # rows: x^k - x^4
    Jm = np.transpose(e, (0, 2, 1))  # J_ik = x_i^k - x_i^4
    assert (np.linalg.det(Jm) > 0).all()
    assert np.allclose(np.einsum("tkj,tjl->tkl", m.B, Jm), np.eye(3), atol=1e-12)
    assert np.allclose(m.V0, np.linalg.det(Jm) / 6.0, rtol=1e-13)
    # the raw mesh has both orientations; only corners 1 and 2 were swapped
    x, t = sphere_tet_mesh(4.0, 1.3)
    raw = np.linalg.det(x[t[:, :3]] - x[t[:, 3:4]])
    assert (raw < 0).any() and (raw > 0).any()
    flip = raw < 0
    assert (m.tets[flip][:, [1, 0, 2, 3]] == t[flip]).all() and (m.tets[~flip] == t[~flip]).all()


def test_volume_of_unsnapped_grid():
    """Kuhn tets of kept cubes tile them exactly: total V_0 = cubes * h^3."""
    x, t = sphere_tet_mesh(3.0, 1.0, min_det_frac=10.0)  # no vertex may move
    _, _, V0 = oracle.mesh_prepare(x, t)
    assert np.isclose(V0.sum(), len(t) / 6 * 1.0, rtol=1e-14)


@pytest.mark.parametrize("bad,code", [("range", 1), ("repeat", 2), ("flat", 3)])
def test_prepare_rejects(bad, code):
    x = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 0]], float)
    t = np.array([[0, 1, 2, 3], [1, 2, 3, 4]], np.int32)
    if bad == "range":
        t[1, 2] = 7
    elif bad == "repeat":
        t[1, 2] = 1
    else:
        t[1] = [0, 1, 2, 4]  # four coplanar points
    with pytest.raises(oracle.MeshError) as e:
        oracle.mesh_prepare(x, t)
    assert e.value.code == code and e.value.tet == 1


def test_csr_brute_force(m):
    rows = [[] for _ in range(len(m.x))]
    for t, tet in enumerate(m.tets):
        for c, v in enumerate(tet):
            rows[v].append(4 * t + c)
    ptr = np.cumsum([0] + [len(r) for r in rows])
    idx = np.concatenate([np.array(r, np.int32) for r in rows])
    assert (m.ptr == ptr).all() and (m.idx == idx).all()


def test_rest_state_has_no_force(m):
    f = m.forces(m.x)
    assert np.abs(f).max() < 1e-14


def test_rigid_motion_has_no_force(m):
    for _ in range(3):
        Q = Rotation.random(random_state=int(RNG.integers(1 << 30))).as_matrix()
        y = m.x @ Q.T + RNG.uniform(-5, 5, 3)
        f, en = m.forces(y, energy=True)
        assert np.abs(f).max() < 1e-12 and np.abs(en).max() < 1e-12


def test_per_tet_balance(m):
    """Each tet's four corner forces sum to zero and exert no torque."""
    y = perturb(m.x, 0.15, 5)
    fc = oracle.tet_forces(m.tets, m.B, m.V0, y - m.x, m.tmat, m.mu, m.kappa, m.w)
    scale = np.abs(fc).max()
    assert np.abs(fc.sum(1)).max() < 1e-13 * scale * 10
    torque = np.cross(y[m.tets], fc).sum(1)
    assert np.abs(torque).max() < 1e-12 * scale * 10


def test_force_is_minus_energy_gradient(m):
    """f_v = -dE/dy_v with E = sum_t V_0 U (Sec. 3.1), by central differences."""
    for amp, mat in ((0.15, (1.0, 5.0, 0.5)), (0.18, (2.0, 100.0, 0.0)), (0.1, (1.0, 0.0, 1.0))):
        m.mu[:], m.kappa[:], m.w[:] = mat
        y = perturb(m.x, amp, int(RNG.integers(1 << 30)))
        f = m.forces(y)
        assert np.isfinite(f).all()
        for _ in range(6):
            v, i = int(RNG.integers(len(y))), int(RNG.integers(3))
            h = 1e-5
            yp, ym = y.copy(), y.copy()
            yp[v, i] += h
            ym[v, i] -= h
            fd = -(m.energy(yp) - m.energy(ym)) / (2 * h)
            assert abs(fd - f[v, i]) <= 1e-7 * np.abs(f).max()
    m.mu[:], m.kappa[:], m.w[:] = 1.0, 5.0, 0.5


def test_patch_test(m):
    """Affine y = F0 x: interior vertices carry no force, the mesh carries
    no net force, and sum_v f_v (x) x_v = -Vol P(F0) (the discrete virial of
    a uniform stress, exact for linear tets)."""
    F0 = np.eye(3) + 0.2 * RNG.uniform(-1, 1, (3, 3))
    y = m.x @ F0.T + 1.5
    f = m.forces(y)
    counts = np.diff(m.ptr)
    # interior vertices of the Kuhn mesh touch 24 tets
    interior = counts == 24
    assert interior.sum() > 10
    scale = np.abs(f).max()
    assert np.abs(f[interior]).max() < 1e-12 * scale * 100
    assert np.abs(f.sum(0)).max() < 1e-12 * scale * 100
    P = oracle.mr_eval(F0, 0.5, 0.5, 5.0)["P"]
    vir = np.einsum("vi,vj->ij", f, m.x)
    assert np.allclose(vir, -m.V0.sum() * P, rtol=1e-11, atol=1e-11 * scale)


def test_two_cells_are_independent():
    """Cells share no tets: forces of a two-cell mesh are the per-cell forces."""
    x1, t1 = sphere_tet_mesh(3.0, 1.2)
    c1 = Cell(x1, t1, x1, 1.0, 5.0, 0.3)
    c2 = Cell(x1 + 20.0, t1, x1 + 20.0, 2.0, 7.0, 0.9)
    both = oracle.Mesh([c1, c2])
    y = perturb(both.x, 0.15, 3)
    f = both.forces(y)
    n = len(x1)
    f1 = oracle.Mesh([c1]).forces(y[:n])
    f2 = oracle.Mesh([c2]).forces(y[n:])
    assert np.array_equal(f[:n], f1) and np.array_equal(f[n:], f2)
