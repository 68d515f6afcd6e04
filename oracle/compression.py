"""Compression between plates, FP64 (test infrastructure only).

The paper compresses a cell between a resting plate and a moving one with a
repulsive force that keeps vertices out of the plates (Sec. 4.2; the form of
that force is given only in the supplement). Reading used here: a one-sided
harmonic penalty per vertex, E_plate = k/2 [(z_lo - z)_+^2 + (z - z_hi)_+^2],
so f_plate,z = k (z_lo - z)_+ - k (z - z_hi)_+, and quasi-static relaxation
of unit-mass vertices by damped second-order steps
    v <- c v + dt (f_el(y) + f_plate(y)),   y <- y + dt v,
where the force is taken at the positions before the step and the position
update uses the new velocity (c = 0 is the gradient flow
y <- y + dt^2 (f_el + f_plate)). The measured force is the top plate's,
F = sum_v k (z_v - z_hi)_+. The plate heights of a protocol come from the
input generator ``workloads.configs.plate_schedule``.
"""
from __future__ import annotations

import numpy as np

from workloads.configs import plate_schedule


def plate_forces(y, k, z_lo, z_hi):
    """Per-vertex plate force [V,3]; z_lo, z_hi per vertex."""
    f = np.zeros_like(y)
    z = y[:, 2]
    f[:, 2] = k * np.maximum(z_lo - z, 0.0) - k * np.maximum(z - z_hi, 0.0)
    return f


def plate_energy(y, k, z_lo, z_hi):
    z = y[:, 2]
    return 0.5 * k * float((np.maximum(z_lo - z, 0.0) ** 2).sum() + (np.maximum(z - z_hi, 0.0) ** 2).sum())


def top_force(y, k, z_hi, ranges):
    """F per cell: sum over its vertices of k (z - z_hi)_+."""
    pen = k * np.maximum(y[:, 2] - z_hi, 0.0)
    return np.array([pen[a:b].sum() for a, b in ranges])


def per_vertex(values, ranges):
    out = np.zeros(ranges[-1][1])
    for (a, b), v in zip(ranges, values):
        out[a:b] = v
    return out


def relax(mesh, y, n, dt, k, z_lo, z_hi, v=None, c=0.0):
    """n damped steps of unit-mass vertices, v <- c v + dt f, y <- y + dt v
    (c = 0: gradient flow with step dt^2); z_lo, z_hi per cell. Returns
    (y, v)."""
    zl = per_vertex(z_lo, mesh.vert_ranges)
    zh = per_vertex(z_hi, mesh.vert_ranges)
    v = np.zeros_like(y) if v is None else v
    for _ in range(n):
        v = c * v + dt * (mesh.forces(y) + plate_forces(y, k, zl, zh))
        y = y + dt * v
    return y, v


def protocol(mesh, y0, z_lo, radius, strains, steps, dt, k, ramp=0, c=0.0):
    """Top-plate force per cell at the end of each strain level [ncells, nlevels]."""
    y = np.array(y0, dtype=np.float64)
    v = np.zeros_like(y)
    out = []
    for z_hi, n, measured in plate_schedule(z_lo, radius, strains, steps, ramp):
        if n == 0:
            continue
        y, v = relax(mesh, y, n, dt, k, z_lo, z_hi, v, c)
        if measured:
            out.append(top_force(y, k, per_vertex(z_hi, mesh.vert_ranges), mesh.vert_ranges))
    return np.stack(out, axis=1), y
