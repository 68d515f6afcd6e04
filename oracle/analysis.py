"""Shape diagnostics of a deformed cell, FP64 (test infrastructure only).

* Taylor deformation parameter D (Sec. 3.3): inertia tensor of the tet mesh
  from tet centroids and current volumes, its eigenvalues, the semi-axes of
  the equivalent ellipsoid and D = (a3 - a1) / (a3 + a1).
* Inclination: angle between the major axis and x in the x-y plane (the paper
  plots shapes but does not define an angle; this is the usual reading).
* Cell strain (Sec. 6.1): (d_max - 2R) / 2R with d_max the largest distance
  between two vertices.

Readings where the paper is silent or garbled:

* the tet centroids are taken relative to the volume-weighted centroid of the
  cell (the paper does not say where the origin of r^l is);
* the printed semi-axis expressions (5/2M)(+-theta...) have units of length
  squared: for a solid ellipsoid theta_1 = M (a2^2 + a3^2) / 5, so the printed
  expression equals a_i^2 and a_i is its square root. ``taylor_literal``
  returns D computed from the printed expression as it stands.
"""
from __future__ import annotations

import numpy as np


def jacobi_eigh(S, tol=1e-15, max_sweeps=50):
    """Eigenvalues and eigenvectors (columns) of a symmetric 3x3 matrix by
    cyclic Jacobi rotations (Golub & Van Loan, Sec. 8.5)."""
    A = np.array(S, dtype=np.float64, copy=True)
    V = np.eye(3)
    for _ in range(max_sweeps):
        off = A[0, 1] ** 2 + A[0, 2] ** 2 + A[1, 2] ** 2
        if off <= tol * tol * max(1.0, float(np.sum(np.diag(A) ** 2))):
            break
        for p in range(2):
            for q in range(p + 1, 3):
                if A[p, q] == 0.0:
                    continue
                theta = (A[q, q] - A[p, p]) / (2.0 * A[p, q])
                t = np.sign(theta) / (abs(theta) + np.sqrt(theta * theta + 1.0)) if theta != 0 else 1.0
                c = 1.0 / np.sqrt(t * t + 1.0)
                s = t * c
                R = np.eye(3)
                R[p, p] = R[q, q] = c
                R[p, q] = s
                R[q, p] = -s
                A = R.T @ A @ R
                V = V @ R
    return np.diag(A).copy(), V


def tet_centroids_volumes(y, tets):
    """Centroid and signed volume of every tet at current positions y."""
    p = y[tets]  # [T,4,3]
    centroid = p.mean(axis=1)
    e = p[:, :3, :] - p[:, 3:4, :]  # rows are edge vectors
    vol = np.linalg.det(e) / 6.0
    return centroid, vol


def inertia_tensor(y, tets):
    """Theta_ij = sum_l V_l (r^l.r^l delta_ij - r^l_i r^l_j) (Sec. 3.3)."""
    r, V = tet_centroids_volumes(y, tets)
    V = np.abs(V)
    centre = (V[:, None] * r).sum(0) / V.sum()
    r = r - centre
    theta = np.zeros((3, 3))
    for l in range(len(V)):
        theta += V[l] * (np.dot(r[l], r[l]) * np.eye(3) - np.outer(r[l], r[l]))
    return theta, float(V.sum())


def _semi_axes_sq(theta_desc, M):
    t1, t2, t3 = theta_desc
    pre = 5.0 / (2.0 * M)
    return np.array([pre * (-t1 + t2 + t3), pre * (t1 - t2 + t3), pre * (t1 + t2 - t3)])


def taylor(y, tets):
    """Returns dict with D, D_literal, semi-axes a1 <= a2 <= a3, inclination
    (degrees, in (-90, 90]) and the eigenvalues theta1 >= theta2 >= theta3."""
    theta, M = inertia_tensor(y, tets)
    lam, vec = jacobi_eigh(theta)
    order = np.argsort(-lam)
    lam, vec = lam[order], vec[:, order]
    a2 = _semi_axes_sq(lam, M)
    a = np.sqrt(np.maximum(a2, 0.0))
    D = (a[2] - a[0]) / (a[2] + a[0])
    D_lit = (a2[2] - a2[0]) / (a2[2] + a2[0])
    major = vec[:, 2]  # axis of the smallest moment of inertia
    ang = np.degrees(np.arctan2(major[1], major[0]))
    if ang <= -90.0:
        ang += 180.0
    elif ang > 90.0:
        ang -= 180.0
    return {"D": float(D), "D_literal": float(D_lit), "a": a, "theta": lam, "inclination": float(ang)}


def cell_strain(y, R):
    """(d_max - 2R) / 2R, d_max by brute force over all vertex pairs."""
    d = 0.0
    for i in range(len(y)):
        di = np.sqrt(((y[i + 1:] - y[i]) ** 2).sum(1))
        if len(di):
            d = max(d, float(di.max()))
    return (d - 2.0 * R) / (2.0 * R)
