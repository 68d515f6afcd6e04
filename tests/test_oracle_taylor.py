"""Pins of the oracle's Taylor deformation diagnostic (Sec. 3.3)."""
import itertools

import numpy as np

from oracle import analysis
from workloads.mesh import sphere_tet_mesh

RNG = np.random.default_rng(9)


def test_jacobi_matches_library_eigh():
    for _ in range(20):
        A = RNG.normal(size=(3, 3))
        S = A + A.T
        lam, V = analysis.jacobi_eigh(S)
        ref = np.linalg.eigh(S)[0]
        assert np.allclose(np.sort(lam), ref, rtol=0, atol=1e-12 * np.abs(ref).max())
        assert np.allclose(S @ V, V * lam, atol=1e-11)


def test_inertia_tensor_by_definition():
    """Theta = sum_l V_l (r.r I - r r^T), r = centroid - volume-weighted centre."""
    x, t = sphere_tet_mesh(2.5, 1.0)
    y = x + RNG.uniform(-0.1, 0.1, x.shape)
    theta, M = analysis.inertia_tensor(y, t)
    ref = np.zeros((3, 3))
    cen, vols = [], []
    for tet in t:
        p = y[tet]
        cen.append(p.mean(0))
        vols.append(abs(np.linalg.det(np.array([p[0] - p[3], p[1] - p[3], p[2] - p[3]]))) / 6)
    cen, vols = np.array(cen), np.array(vols)
    c0 = (vols[:, None] * cen).sum(0) / vols.sum()
    for r, V in zip(cen - c0, vols):
        ref += V * (r @ r * np.eye(3) - np.outer(r, r))
    assert np.allclose(theta, ref, rtol=1e-12) and np.isclose(M, vols.sum())


def _symmetric_ball():
    """Tet set invariant under the 48 symmetries of the cube (reflections and
    axis permutations), so its second-moment tensor is isotropic."""
    x, t = sphere_tet_mesh(4.0, 1.1)
    xs, ts = [], []
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product((1, -1), repeat=3):
            xs.append(x[:, perm] * np.array(signs))
            ts.append(t + len(x) * len(ts))
    return np.concatenate(xs), np.concatenate(ts)


def test_sphere_has_zero_deformation():
    y, t = _symmetric_ball()
    assert abs(analysis.taylor(y, t)["D"]) < 1e-12


def test_affinely_stretched_ball():
    """y = diag(a) x: centroids and volumes map affinely, so Theta's semi-axes
    scale by a and D = (a3 - a1) / (a3 + a1) exactly; rotating the stretch
    in the x-y plane sets the inclination."""
    y, t = _symmetric_ball()
    a = np.array([0.8, 1.0, 1.3])
    r = analysis.taylor(y * a, t)
    assert np.isclose(r["D"], (a[2] - a[0]) / (a[2] + a[0]), rtol=1e-12)
    assert np.isclose(r["D_literal"], (a[2] ** 2 - a[0] ** 2) / (a[2] ** 2 + a[0] ** 2), rtol=1e-12)
    b = np.array([1.4, 0.9, 1.0])
    phi = np.radians(30.0)
    Rz = np.array([[np.cos(phi), -np.sin(phi), 0], [np.sin(phi), np.cos(phi), 0], [0, 0, 1]])
    r2 = analysis.taylor(y @ (Rz @ np.diag(b)).T, t)
    assert np.isclose(r2["inclination"], 30.0, atol=1e-9)
    assert np.isclose(r2["D"], (1.4 - 0.9) / (1.4 + 0.9), rtol=1e-12)


def test_solid_ellipsoid_semi_axes():
    """For a solid ellipsoid theta_1 = M (a2^2 + a3^2)/5 etc.; the square root
    reading of the semi-axis formula returns the axes."""
    a = np.array([2.0, 3.0, 5.0])
    M = 7.0
    theta = M / 5 * np.array([a[1] ** 2 + a[2] ** 2, a[0] ** 2 + a[2] ** 2, a[0] ** 2 + a[1] ** 2])
    got = np.sqrt(analysis._semi_axes_sq(theta, M))
    assert np.allclose(got, a, rtol=1e-14)


def test_cell_strain_brute_force():
    y = RNG.normal(size=(40, 3))
    d = max(np.linalg.norm(p - q) for p in y for q in y)
    assert np.isclose(analysis.cell_strain(y, 1.5), (d - 3.0) / 3.0, rtol=1e-14)
