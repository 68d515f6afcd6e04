"""Differentiable compression experiment (PyTorch autograd over the C ABI).

``CompressionCurve.apply(mu, kappa, w, run)`` returns the top-plate force of
every cell at the end of each strain level of a quasi-static compression
protocol (``run``: a :class:`Compression`), as a ``[ncells, nlevels]``
tensor; its backward pass reverses the recorded relaxation calls with
``cf_relax_adjoint`` (hand-written adjoint in the CUDA library, positions
recomputed from checkpoints) and returns dL/d(mu, kappa, w) per cell. All
numerics run in the library; this module only orders the calls.
"""
from __future__ import annotations

import numpy as np
import torch

from workloads.configs import plate_schedule

from . import (CF_ALL_CELLS, cf_adjoint_gradients, cf_plate_force, cf_plates_set, cf_relax, cf_relax_adjoint,
               cf_set_materials, cf_set_positions, cf_tape_clear, cf_tape_generation)


class Compression:
    """Protocol: cells start at y0 on the lower plate z_lo; for each strain
    s in ``strains`` the upper plate approaches z_lo + 2 R (1 - s) (see
    plate_schedule) while the cells relax with damped steps (size ``dt``,
    velocity retention ``damping``); the top-plate force is measured at the
    end of each level."""

    def __init__(self, ctx, ids, y0, z_lo, radius, strains, steps, dt, k_plate, ramp=0, damping=0.0):
        self.ctx, self.ids = ctx, list(ids)
        self.y0 = np.ascontiguousarray(y0, dtype=np.float64)
        self.z_lo = np.asarray(z_lo, np.float64)
        self.radius = np.asarray(radius, np.float64)
        self.strains = list(strains)
        self.steps, self.dt, self.k_plate, self.ramp, self.damping = steps, dt, k_plate, ramp, damping
        self.measured = []  # per recorded cf_relax call: True at the end of a level

    def run(self, mu, kappa, w, record):
        c = self.ctx
        cf_set_materials(c, self.ids, mu, kappa, w)
        cf_set_positions(c, CF_ALL_CELLS, self.y0)
        cf_tape_clear(c)
        forces, self.measured = [], []
        for z_hi, n, measured in plate_schedule(self.z_lo, self.radius, self.strains, self.steps, self.ramp):
            if n == 0:
                continue
            cf_plates_set(c, self.k_plate, self.z_lo, z_hi)
            cf_relax(c, n, self.dt, self.damping, record=record)
            self.measured.append(measured)
            if measured:
                forces.append(cf_plate_force(c))
        return np.stack(forces, axis=1)


class CompressionCurve(torch.autograd.Function):
    @staticmethod
    def forward(fctx, mu, kappa, w, run: Compression):
        F = run.run(mu.detach().cpu().numpy(), kappa.detach().cpu().numpy(), w.detach().cpu().numpy(), record=True)
        fctx.run = run
        # the tape lives in the library's context: remember which recording is this forward's
        fctx.tape_gen = cf_tape_generation(run.ctx)
        fctx.measured = list(run.measured)
        return torch.as_tensor(F, dtype=torch.float64)

    @staticmethod
    def backward(fctx, dF):
        run = fctx.run
        if cf_tape_generation(run.ctx) != fctx.tape_gen or run.measured != fctx.measured:
            raise RuntimeError("the context's tape was cleared or re-recorded after this forward pass "
                               "(another CompressionCurve forward ran on the same context before this backward)")
        dF = dF.detach().cpu().numpy()
        level = dF.shape[1]
        zero = np.zeros(dF.shape[0])
        for measured in reversed(fctx.measured):  # recorded cf_relax calls, last first
            if measured:
                level -= 1
                cf_relax_adjoint(run.ctx, np.ascontiguousarray(dF[:, level]))
            else:
                cf_relax_adjoint(run.ctx, zero)
        g = torch.as_tensor(cf_adjoint_gradients(run.ctx), dtype=torch.float64)
        return g[:, 0], g[:, 1], g[:, 2], None
