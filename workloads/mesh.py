"""Seeded synthetic tetrahedral sphere meshes (input generator only).

The paper builds its cells from a uniformly tetrahedralised sphere of
2,000-5,000 vertices and about 10k-30k tets (Sec. 4.2); the mesher itself is
in its supplement, which is not available. This module stands in for it with
a plain construction:

* a cubic grid of spacing ``h`` centred on the origin;
* every cube whose centre lies inside radius ``R`` is kept and split into the
  six Kuhn (Freudenthal) tetrahedra that share the cube's main diagonal;
* vertices on the outer surface of the kept cubes are moved radially onto the
  sphere ``|y| = R``, except where that would flatten an incident tet below
  ``min_det_frac * h**3`` (those vertices keep their grid position).

Half of the Kuhn tets come out negatively oriented, on purpose: both the
oracle and the CUDA path must orient tets themselves (Sec. 3.2 gives no
orientation convention).

Nothing here computes any part of the method: no deformation gradient, no
energy, no force. It only produces coordinates and connectivity.
"""
from __future__ import annotations

import itertools

import numpy as np

_UNIT = np.eye(3, dtype=np.int64)


def sphere_tet_mesh(R: float, h: float, min_det_frac: float = 0.25):
    """Return ``(x, tets)``: vertices ``float64 [V,3]`` centred on the origin
    and tets ``int32 [T,4]`` (corner 3 is the paper's vertex 4)."""
    n = int(np.ceil(R / h)) + 1
    idx = np.arange(-n, n, dtype=np.int64)
    I, J, K = np.meshgrid(idx, idx, idx, indexing="ij")
    centres = np.stack([(I + 0.5) * h, (J + 0.5) * h, (K + 0.5) * h], -1)
    keep = np.linalg.norm(centres, axis=-1) < R
    cubes = np.stack([I[keep], J[keep], K[keep]], -1)  # lower corners, [nc,3]

    # six Kuhn tets per cube: walk 000 -> 111 along the axes in each order
    corners = []
    for perm in itertools.permutations(range(3)):
        p0 = np.zeros(3, np.int64)
        p1 = p0 + _UNIT[perm[0]]
        p2 = p1 + _UNIT[perm[1]]
        p3 = p2 + _UNIT[perm[2]]
        corners.append(np.stack([p0, p1, p2, p3]))
    corners = np.stack(corners)  # [6,4,3]
    grid_pts = cubes[:, None, None, :] + corners[None]  # [nc,6,4,3]
    grid_pts = grid_pts.reshape(-1, 3)
    uniq, inv = np.unique(grid_pts, axis=0, return_inverse=True)
    tets = inv.reshape(-1, 4).astype(np.int32)

    # a grid vertex is on the surface if fewer than 8 kept cubes touch it
    kept = set(map(tuple, cubes.tolist()))
    touch = np.zeros(len(uniq), np.int64)
    for d in itertools.product((0, 1), repeat=3):
        lower = uniq - np.asarray(d)
        touch += np.fromiter((tuple(c) in kept for c in lower.tolist()), bool, len(lower))
    surface = touch < 8

    x = uniq.astype(np.float64) * h
    snapped = x.copy()
    r = np.linalg.norm(x[surface], axis=1)
    snapped[surface] = x[surface] * (R / r)[:, None]

    # revert snaps that leave a tet too flat; repeat until none does
    use_snap = surface.copy()
    for _ in range(100):
        y = np.where(use_snap[:, None], snapped, x)
        e = y[tets[:, :3]] - y[tets[:, 3:4]]  # [T,3,3] edge vectors (rows)
        vol6 = np.abs(np.linalg.det(e))
        bad = vol6 <= min_det_frac * h**3
        if not bad.any():
            break
        use_snap[np.unique(tets[bad])] = False
    y = np.where(use_snap[:, None], snapped, x)
    return y, tets


def perturb(x: np.ndarray, amplitude: float, seed: int) -> np.ndarray:
    """``x + amplitude * U(-1, 1)`` per coordinate (numpy PCG64 with ``seed``)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return x + amplitude * rng.uniform(-1.0, 1.0, size=x.shape)


def replicate_meshes(x: np.ndarray, tets: np.ndarray, offsets: np.ndarray):
    """Concatenate copies of one mesh shifted by ``offsets [n,3]``; returns a
    list of ``(x_i, tets)`` pairs (tets stay local to each copy)."""
    return [(x + o[None, :], tets) for o in np.asarray(offsets, np.float64)]


def shell_regions(x, tets, r_inner, r_outer):
    """Region of each tet by the distance of its centroid from the mesh's
    centre: 0 inside r_inner (a nucleus), 2 beyond r_outer (a cortex), 1 in
    between."""
    x = np.asarray(x, np.float64)
    c = x[np.asarray(tets)].mean(axis=1)
    r = np.linalg.norm(c - x.mean(axis=0), axis=1)
    return np.where(r < r_inner, 0, np.where(r > r_outer, 2, 1)).astype(np.int32)
