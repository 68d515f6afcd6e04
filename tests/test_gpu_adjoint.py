"""GPU: compression between plates and the hand-written adjoint, against the
FP64 oracle (Sec. 4.2 set-up; Sec. 4.3 fits E and w to force-deformation
curves). The adjoint's gradients must agree with finite differences of the
oracle's loss to 1e-4."""
import numpy as np
import pytest

import oracle
from oracle import compression as cp
from workloads.configs import Cell
from workloads.mesh import perturb, sphere_tet_mesh

pytestmark = pytest.mark.gpu

RNG = np.random.default_rng(33)
STRAINS = [0.1, 0.2, 0.3]
STEPS, DT, KP, RAMP = 60, 0.004 ** 0.5, 20.0, 3


@pytest.fixture(scope="module")
def P():
    from paper_2003_03130_gb300 import build

    build.build()
    import paper_2003_03130_gb300 as P

    return P


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def two_cells(mu=(1.0, 0.7), kappa=(20.0, 15.0), w=(0.5, 0.2)):
    cells = []
    for k, (R, h, x0) in enumerate(((4.0, 1.3, 10.0), (5.0, 1.4, 30.0))):
        x, t = sphere_tet_mesh(R, h)
        x = x + np.array([x0, 12.0, 12.0])
        cells.append(Cell(x, t, x.copy(), mu[k], kappa[k], w[k]))
    return cells


def setup(P, cells, y=None):
    ctx = P.cf_create(0)
    ids = P.cf_mesh_init_batch(ctx, [c.x_ref for c in cells], [c.tets for c in cells],
                               None if y is None else [y[a:b] for a, b in oracle.Mesh(cells).vert_ranges])
    P.cf_set_materials(ctx, ids, [c.mu for c in cells], [c.kappa for c in cells], [c.w for c in cells])
    return ctx, ids


def protocol_geometry(cells):
    z_lo = np.array([c.x_ref[:, 2].min() for c in cells])
    radius = np.array([0.5 * (c.x_ref[:, 2].max() - c.x_ref[:, 2].min()) for c in cells])
    return z_lo, radius


def test_force_jvp_matches_oracle_hessian(P):
    cells = two_cells()
    m = oracle.Mesh(cells)
    y = perturb(m.x, 0.1, 5)
    v = RNG.normal(size=y.shape)
    ctx, _ = setup(P, cells, y)
    got = P.cf_force_jvp(ctx, v)
    y_gpu = P.cf_get_positions(ctx, P.CF_ALL_CELLS)
    h = 1e-5
    ref = (m.forces(y_gpu + h * v) - m.forces(y_gpu - h * v)) / (2 * h)
    assert rel(got, ref) <= 1e-5


def test_force_param_vjp_matches_oracle(P):
    cells = two_cells()
    m = oracle.Mesh(cells)
    y = perturb(m.x, 0.1, 6)
    lam = RNG.normal(size=y.shape)
    ctx, _ = setup(P, cells, y)
    got = P.cf_force_param_vjp(ctx, lam)
    y_gpu = P.cf_get_positions(ctx, P.CF_ALL_CELLS)
    ref = np.zeros((2, 3))
    for c in range(2):
        for k, attr in enumerate(("mu", "kappa", "w")):
            a = getattr(m, attr)
            h = 1e-6 * max(1.0, abs(a[c]))
            a0 = a[c]
            a[c] = a0 + h
            fp = m.forces(y_gpu)
            a[c] = a0 - h
            fm = m.forces(y_gpu)
            a[c] = a0
            ref[c, k] = np.sum(lam * (fp - fm)) / (2 * h)
    assert rel(got, ref) <= 1e-5


def test_compression_matches_oracle(P):
    from paper_2003_03130_gb300.adjoint import Compression

    cells = two_cells()
    m = oracle.Mesh(cells)
    z_lo, radius = protocol_geometry(cells)
    ctx, ids = setup(P, cells)
    run = Compression(ctx, ids, m.x, z_lo, radius, STRAINS, STEPS, DT, KP, RAMP)
    F = run.run(m.mu, m.kappa, m.w, record=False)
    F_ref, y_ref = cp.protocol(m, m.x, z_lo, radius, STRAINS, STEPS, DT, KP, RAMP)
    assert (F_ref > 0).all()
    assert rel(F, F_ref) <= 1e-5
    assert rel(P.cf_get_positions(ctx, P.CF_ALL_CELLS) - m.x, y_ref - m.x) <= 1e-5


def oracle_loss(cells, theta, target, z_lo, radius, dt=DT, damping=0.0):
    m = oracle.Mesh(cells)
    m.mu[:], m.kappa[:], m.w[:] = theta[:, 0], theta[:, 1], theta[:, 2]
    F, _ = cp.protocol(m, m.x, z_lo, radius, STRAINS, STEPS, dt, KP, RAMP, damping)
    return float(((F - target) ** 2).sum())


@pytest.mark.parametrize("damping", [0.0, 0.8])
def test_adjoint_gradient_matches_oracle_finite_differences(P, damping):
    torch = pytest.importorskip("torch")
    from paper_2003_03130_gb300.adjoint import Compression, CompressionCurve

    hidden = two_cells(mu=(1.2, 0.9), kappa=(24.0, 12.0), w=(0.7, 0.4))
    cells = two_cells()
    m = oracle.Mesh(cells)
    z_lo, radius = protocol_geometry(cells)
    dt = DT if damping == 0.0 else 0.05
    target, _ = cp.protocol(oracle.Mesh(hidden), m.x, z_lo, radius, STRAINS, STEPS, dt, KP, RAMP, damping)

    ctx, ids = setup(P, cells)
    run = Compression(ctx, ids, m.x, z_lo, radius, STRAINS, STEPS, dt, KP, RAMP, damping)
    mu = torch.tensor(m.mu, dtype=torch.float64, requires_grad=True)
    kappa = torch.tensor(m.kappa, dtype=torch.float64, requires_grad=True)
    w = torch.tensor(m.w, dtype=torch.float64, requires_grad=True)
    F = CompressionCurve.apply(mu, kappa, w, run)
    loss = ((F - torch.as_tensor(target)) ** 2).sum()
    loss.backward()
    got = np.stack([mu.grad.numpy(), kappa.grad.numpy(), w.grad.numpy()], axis=1)

    theta = np.stack([m.mu, m.kappa, m.w], axis=1)
    fd = np.zeros_like(theta)
    for c in range(2):
        for k in range(3):
            h = 1e-5 * max(1.0, abs(theta[c, k]))
            tp, tm = theta.copy(), theta.copy()
            tp[c, k] += h
            tm[c, k] -= h
            fd[c, k] = (oracle_loss(cells, tp, target, z_lo, radius, dt, damping) -
                        oracle_loss(cells, tm, target, z_lo, radius, dt, damping)) / (2 * h)
    print("damping", damping, "adjoint", got.tolist(), "fd", fd.tolist(), "rel", rel(got, fd))
    assert rel(got, fd) <= 1e-4
    assert abs(loss.item() - oracle_loss(cells, theta, target, z_lo, radius, dt, damping)) <= 1e-4 * loss.item()


def test_fit_recovers_hidden_moduli(P):
    """Adam on (log mu, log kappa, logit w) with adjoint gradients brings the
    loss of a synthetic force-strain curve down and moves the moduli towards
    the hidden ones."""
    torch = pytest.importorskip("torch")
    from paper_2003_03130_gb300.adjoint import Compression, CompressionCurve

    hidden = two_cells(mu=(1.3, 0.8), kappa=(22.0, 16.0), w=(0.75, 0.3))
    cells = two_cells(mu=(1.0, 1.0), kappa=(20.0, 20.0), w=(0.5, 0.5))
    m = oracle.Mesh(cells)
    z_lo, radius = protocol_geometry(cells)
    strains, steps, dt, damping = [0.1, 0.2, 0.3, 0.4], 200, 0.05, 0.9
    ctx, ids = setup(P, cells)
    run = Compression(ctx, ids, m.x, z_lo, radius, strains, steps, dt, KP, RAMP, damping)
    hm = oracle.Mesh(hidden)
    target = torch.as_tensor(run.run(hm.mu, hm.kappa, hm.w, record=False))
    th = torch.tensor([[0.0, np.log(20.0), 0.0]] * 2, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([th], lr=0.05)
    losses = []
    for _ in range(40):
        F = CompressionCurve.apply(torch.exp(th[:, 0]), torch.exp(th[:, 1]), torch.sigmoid(th[:, 2]), run)
        loss = (((F - target) ** 2).sum(1) / (target ** 2).sum(1)).sum()
        opt.zero_grad()
        loss.backward()
        opt.step()
        losses.append(loss.item())
    mu = torch.exp(th[:, 0]).detach().numpy()
    print("losses", losses[0], losses[-1], "mu", mu, "hidden", hm.mu)
    assert losses[-1] < 0.05 * losses[0]
    assert np.abs(mu / hm.mu - 1).max() < np.abs(1.0 / hm.mu - 1).max()


def test_compression_full_size_matches_oracle(P):
    """The 64-cell compression set at full size (8,256 tets per cell) with
    the benchmark's hidden moduli, plate stiffness, time step, damping and
    plate ramp: the first two strain levels, shortened to 40 damped steps
    each, against the oracle."""
    from paper_2003_03130_gb300.adjoint import Compression
    from workloads import configs

    cs = configs.compression_set()
    cells = [Cell(c.x_ref, c.tets, c.y0, mu, ka, w)
             for c, mu, ka, w in zip(cs.cells, cs.hidden_mu, cs.hidden_kappa, cs.hidden_w)]
    m = oracle.Mesh(cells)
    z_lo, radius = protocol_geometry(cells)
    strains, steps = cs.strains[:2], 40
    ctx, ids = setup(P, cells)
    run = Compression(ctx, ids, m.x, z_lo, radius, strains, steps, cs.dt, cs.k_plate, cs.ramp, cs.damping)
    F = run.run(m.mu, m.kappa, m.w, record=False)
    F_ref, y_ref = cp.protocol(m, m.x, z_lo, radius, strains, steps, cs.dt, cs.k_plate, cs.ramp, cs.damping)
    assert len(ids) == 64 and (F_ref > 0).all()
    assert rel(F, F_ref) <= 1e-5
    assert rel(P.cf_get_positions(ctx, P.CF_ALL_CELLS) - m.x, y_ref - m.x) <= 1e-5


def test_backward_refuses_a_tape_of_another_forward(P):
    """The tape lives in the context: a second forward on the same context
    re-records it, so the first forward's backward must refuse instead of
    reversing the wrong recording; and a material changed after a recorded
    relaxation makes its reverse pass a state error."""
    torch = pytest.importorskip("torch")
    from paper_2003_03130_gb300.adjoint import Compression, CompressionCurve

    cells = two_cells()
    m = oracle.Mesh(cells)
    z_lo, radius = protocol_geometry(cells)
    ctx, ids = setup(P, cells)
    run = Compression(ctx, ids, m.x, z_lo, radius, STRAINS[:2], 20, DT, KP, RAMP, 0.8)
    th = [torch.tensor(getattr(m, a), dtype=torch.float64, requires_grad=True) for a in ("mu", "kappa", "w")]
    F1 = CompressionCurve.apply(*th, run)
    g0 = P.cf_tape_generation(ctx)
    F2 = CompressionCurve.apply(th[0] * 1.1, th[1], th[2], run)
    assert P.cf_tape_generation(ctx) > g0
    with pytest.raises(RuntimeError):
        F1.sum().backward(retain_graph=True)
    F2.sum().backward()  # its own tape: fine
    assert all(t.grad is not None and torch.isfinite(t.grad).all() for t in th)

    # materials changed between a recorded relaxation and its reverse pass
    P.cf_set_materials(ctx, ids, m.mu, m.kappa, m.w)
    P.cf_tape_clear(ctx)
    P.cf_plates_set(ctx, KP, z_lo, z_lo + 2 * radius * 0.9)
    P.cf_relax(ctx, 10, DT, 0.8, record=True)
    P.cf_set_material(ctx, ids[1], 0.9 * m.mu[1], m.kappa[1], m.w[1])
    with pytest.raises(P.CellFSIError) as e:
        P.cf_relax_adjoint(ctx, np.ones(2))
    assert e.value.name == "CF_ESTATE"
    P.cf_set_material(ctx, ids[1], m.mu[1], m.kappa[1], m.w[1])  # back as recorded
    P.cf_relax_adjoint(ctx, np.ones(2))
