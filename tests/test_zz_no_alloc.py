"""The no-allocation vertex-force entry point against the oracle and against
the context path.

``cf_vertex_forces_static`` is for callers that may not allocate device
memory (a plugin inside a host application that owns all device buffers, a
real-time loop with fixed memory). Here the test plays that caller: it owns
the input and output buffers (allocated with PyTorch, outside the entry
point), fills them with the mesh data that ``cf_mesh_init`` prepared, and
calls the entry point twice in a row with different positions and
materials. Each result must match the FP64 oracle's vertex forces
(``oracle.Mesh.forces``) at the tolerance of the other force tests, and the
context path (``cf_compute_forces``) on the same inputs. A mesh just below
the static array's capacity exercises the upper part of the array, and an
inverted configuration must report CF_EINVERTED without leaving the error
word set for the next call.

This file is named to be collected last, so that a run stopping at the first
failure has already run every other test.
"""
import numpy as np
import pytest

import oracle
from workloads import configs
from workloads.configs import Cell
from workloads.mesh import perturb, sphere_tet_mesh

pytestmark = pytest.mark.gpu

TOL = 1e-5
CAP = 65536  # CF_STATIC_MAX_TETS


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def P():
    from paper_2003_03130_gb300 import build

    build.build()
    import paper_2003_03130_gb300 as P

    return P


class CallerBuffers:
    """Device buffers a caller owns for one mesh: the mesh data that
    cf_mesh_init prepared (oriented tets, B, V0, incidence rows), the
    displacements and the output forces."""

    def __init__(self, P, torch, ctx, cid, x_ref):
        tets, B, V0 = P.cf_get_mesh(ctx, cid)
        ptr, idx = P.cf_get_csr(ctx, cid)
        self.nv, self.nt = len(x_ref), len(tets)
        self.x_ref = x_ref
        self.tets = tets
        dev = torch.device("cuda", 0)
        self.torch, self.dev = torch, dev
        self.d_tets = torch.tensor(tets, dtype=torch.int32, device=dev).contiguous()
        self.d_B = torch.tensor(B.reshape(self.nt, 9).T.copy(), dtype=torch.float32, device=dev).contiguous()
        self.d_V0 = torch.tensor(V0, dtype=torch.float32, device=dev)
        self.d_ptr = torch.tensor(ptr, dtype=torch.int32, device=dev)
        self.d_idx = torch.tensor(idx, dtype=torch.int32, device=dev)
        self.d_u = torch.zeros((self.nv, 4), dtype=torch.float32, device=dev)
        self.d_f = torch.full((self.nv, 4), float("nan"), dtype=torch.float32, device=dev)
        self.stream = torch.cuda.current_stream(dev).cuda_stream

    def forces(self, P, y, mu, kappa, w):
        """Vertex forces at positions y through the static entry point
        (raises CellFSIError on a status other than CF_OK)."""
        torch = self.torch
        self.d_u[:, :3] = torch.tensor((y - self.x_ref).astype(np.float32), device=self.dev)
        self.d_f.fill_(float("nan"))
        torch.cuda.synchronize(self.dev)
        P.cf_vertex_forces_static(self.nv, self.nt, self.d_tets.data_ptr(), self.d_B.data_ptr(),
                                  self.d_V0.data_ptr(), self.d_u.data_ptr(), self.d_ptr.data_ptr(),
                                  self.d_idx.data_ptr(), mu, kappa, w, self.d_f.data_ptr(), self.stream)
        return self.d_f[:, :3].double().cpu().numpy()


def _oracle_forces(x_ref, tets, y, mu, kappa, w):
    return oracle.Mesh([Cell(x_ref, tets, y, mu, kappa, w)]).forces(y)


def test_static_entry_point_matches_oracle_and_context_forces(P):
    torch = pytest.importorskip("torch")
    cell = configs.small_shear().cells[0]
    ctx = P.cf_create(0)
    cid = P.cf_mesh_init(ctx, cell.x_ref, cell.tets, cell.y0)
    buf = CallerBuffers(P, torch, ctx, cid, cell.x_ref)

    cases = [(cell.y0, (1e-3, 0.1, 0.5)), (perturb(cell.x_ref, 0.05, 99), (2e-3, 0.3, 1.0))]
    for y, (mu, kappa, w) in cases:  # two calls in a row
        got = buf.forces(P, y, mu, kappa, w)
        assert np.isfinite(got).all()
        assert _rel(got, _oracle_forces(cell.x_ref, cell.tets, y, mu, kappa, w)) <= TOL
        # the context path on the same inputs
        P.cf_set_positions(ctx, cid, y)
        P.cf_set_material(ctx, cid, mu, kappa, w)
        P.cf_compute_forces(ctx)
        assert _rel(got, P.cf_get_forces(ctx, cid)) <= TOL
    P.cf_destroy(ctx)


def test_static_entry_point_near_capacity(P):
    """A 64,608-tet mesh (98.6 % of the static array) at two shapes."""
    torch = pytest.importorskip("torch")
    x, t = sphere_tet_mesh(24.0, 1.75)
    x = x + 30.0
    assert 0.95 * CAP < len(t) <= CAP
    ctx = P.cf_create(0)
    cid = P.cf_mesh_init(ctx, x, t, None)
    buf = CallerBuffers(P, torch, ctx, cid, x)
    for seed, (mu, kappa, w) in ((5, (1e-3, 5e-2, 0.3)), (6, (4e-4, 2e-2, 0.9))):
        y = perturb(x, 0.05, seed)
        got = buf.forces(P, y, mu, kappa, w)
        assert np.isfinite(got).all()
        assert _rel(got, _oracle_forces(x, t, y, mu, kappa, w)) <= TOL
    P.cf_destroy(ctx)


def test_static_entry_point_reports_inversion_then_recovers(P):
    """Every tet inverted (the cell mirrored through its centre, F = -I):
    CF_EINVERTED. The next call on a valid shape returns CF_OK with the
    oracle's forces: each call starts from a clear error word."""
    torch = pytest.importorskip("torch")
    cell = configs.small_shear().cells[0]
    ctx = P.cf_create(0)
    cid = P.cf_mesh_init(ctx, cell.x_ref, cell.tets, cell.y0)
    buf = CallerBuffers(P, torch, ctx, cid, cell.x_ref)
    c = cell.x_ref.mean(0)
    with pytest.raises(P.CellFSIError) as e:
        buf.forces(P, 2 * c - cell.x_ref, 1e-3, 0.1, 0.5)
    assert e.value.name == "CF_EINVERTED"
    y = perturb(cell.x_ref, 0.05, 3)
    got = buf.forces(P, y, 1e-3, 0.1, 0.5)
    assert _rel(got, _oracle_forces(cell.x_ref, cell.tets, y, 1e-3, 0.1, 0.5)) <= TOL
    P.cf_destroy(ctx)


def test_static_entry_point_rejects_oversize_mesh(P):
    with pytest.raises(P.CellFSIError) as e:
        P.cf_vertex_forces_static(4, CAP + 1, 16, 16, 16, 16, 16, 16, 1.0, 1.0, 0.5, 16, None)
    assert e.value.name == "CF_EINVAL"
