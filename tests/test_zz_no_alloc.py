"""The no-allocation vertex-force entry point gives the same forces as the
context path.

``cf_vertex_forces_static`` is for callers that may not allocate device
memory (a plugin inside a host application that owns all device buffers, a
real-time loop with fixed memory). Here the test plays that caller: it owns
the input and output buffers (allocated with PyTorch, outside the entry
point), fills them from the context's mesh data, and calls the entry point
twice in a row with different positions and materials; each result must
match ``cf_compute_forces`` + ``cf_get_forces`` on the same inputs.

This file is named to be collected last, so that a run stopping at the first
failure has already run every other test.
"""
import numpy as np
import pytest

from workloads import configs
from workloads.mesh import perturb

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_static_entry_point_matches_context_forces():
    torch = pytest.importorskip("torch")
    from paper_2003_03130_gb300 import build

    build.build()
    import paper_2003_03130_gb300 as P

    cell = configs.small_shear().cells[0]
    ctx = P.cf_create(0)
    cid = P.cf_mesh_init(ctx, cell.x_ref, cell.tets, cell.y0)
    tets, B, V0 = P.cf_get_mesh(ctx, cid)
    ptr, idx = P.cf_get_csr(ctx, cid)
    nv, nt = len(cell.x_ref), len(tets)

    dev = torch.device("cuda", 0)
    d_tets = torch.tensor(tets, dtype=torch.int32, device=dev).contiguous()
    d_B = torch.tensor(B.reshape(nt, 9).T.copy(), dtype=torch.float32, device=dev).contiguous()
    d_V0 = torch.tensor(V0, dtype=torch.float32, device=dev)
    d_ptr = torch.tensor(ptr, dtype=torch.int32, device=dev)
    d_idx = torch.tensor(idx, dtype=torch.int32, device=dev)
    d_u = torch.zeros((nv, 4), dtype=torch.float32, device=dev)
    d_f = torch.full((nv, 4), float("nan"), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream

    cases = [(cell.y0, (1e-3, 0.1, 0.5)), (perturb(cell.x_ref, 0.05, 99), (2e-3, 0.3, 1.0))]
    for y, (mu, kappa, w) in cases:
        # the context path on these inputs
        P.cf_set_positions(ctx, cid, y)
        P.cf_set_material(ctx, cid, mu, kappa, w)
        P.cf_compute_forces(ctx)
        ref = P.cf_get_forces(ctx, cid)
        # the caller-owned buffers for the static path
        d_u[:, :3] = torch.tensor((y - cell.x_ref).astype(np.float32), device=dev)
        d_f.fill_(float("nan"))
        torch.cuda.synchronize(dev)
        P.cf_vertex_forces_static(nv, nt, d_tets.data_ptr(), d_B.data_ptr(), d_V0.data_ptr(), d_u.data_ptr(),
                                  d_ptr.data_ptr(), d_idx.data_ptr(), mu, kappa, w, d_f.data_ptr(), stream)
        got = d_f[:, :3].double().cpu().numpy()
        assert np.isfinite(got).all()
        assert _rel(got, ref) <= TOL


def test_static_entry_point_rejects_oversize_mesh():
    from paper_2003_03130_gb300 import build

    build.build()
    import paper_2003_03130_gb300 as P

    with pytest.raises(P.CellFSIError) as e:
        P.cf_vertex_forces_static(4, 65537, 16, 16, 16, 16, 16, 16, 1.0, 1.0, 0.5, 16, None)
    assert e.value.name == "CF_EINVAL"
