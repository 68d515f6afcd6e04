"""Writes ``oracle_small_shear.json``: a regression record of the FP64 oracle
on the 32^3 single-cell shear workload (R = 8 sphere, mu = 1e-3, kappa = 0.1,
w = 0.5, 1 % noise, walls -/+0.01, tau = 1). It calls only ``oracle/`` and
the seeded input generators; a change in these numbers means the oracle's
arithmetic changed and must be justified by the passage of the paper it
follows.

Run from the repository root: ``python tests/golden/make_golden.py``.
"""
import json
import os
import sys

import numpy as np

sys.path.insert(0, os.path.abspath(os.path.join(os.path.dirname(__file__), "..", "..")))

import oracle  # noqa: E402
from oracle import analysis  # noqa: E402
from workloads import configs  # noqa: E402

STEPS = 20


def record():
    wl = configs.small_shear()
    sim = oracle.Coupled(wl)
    f0, en0 = sim.mesh.forces(sim.y, energy=True)
    out = {
        "workload": wl.name,
        "n_verts": int(len(sim.y)),
        "n_tets": int(len(sim.mesh.tets)),
        "energy_t0": float(en0.sum()),
        "force_norm_t0": float(np.linalg.norm(f0)),
        "force_v0_t0": f0[0].tolist(),
        "steps": STEPS,
    }
    sim.step(STEPS)
    disp = sim.y - wl.cells[0].y0
    out["disp_norm"] = float(np.linalg.norm(disp))
    out["disp_v0"] = disp[0].tolist()
    out["fluid_u_node_0_16_0"] = sim.fluid.u[0, 16, 0].tolist()
    out["fluid_mass"] = sim.fluid.total_mass()
    out["taylor_D"] = analysis.taylor(sim.y, sim.mesh.tets)["D"]
    return out


if __name__ == "__main__":
    path = os.path.join(os.path.dirname(__file__), "oracle_small_shear.json")
    with open(path, "w") as fh:
        json.dump(record(), fh, indent=1)
    print("wrote", path)
