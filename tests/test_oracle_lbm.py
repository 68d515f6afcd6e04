"""Pins of the oracle's lattice-Boltzmann fluid: D3Q19 BGK, Guo forcing,
halfway bounce-back with moving walls at y = -1/2 and y = ny - 1/2, periodic
x and z. The paper states only that ESPResSo's LB is used (Sec. 6); these
closed forms come from lattice-Boltzmann theory, not from the oracle."""
import numpy as np
import pytest

import oracle

RNG = np.random.default_rng(5)


def test_lattice_moments():
    """D3Q19 isotropy: sum w = 1, sum w c = 0, sum w c c = I/3,
    sum w c_a c_b c_c c_d = (d_ab d_cd + d_ac d_bd + d_ad d_bc)/9."""
    c, w = oracle.lattice()
    c = c.astype(float)
    assert np.isclose(w.sum(), 1.0, rtol=0, atol=1e-15)
    assert np.allclose(w @ c, 0.0, atol=1e-16)
    assert np.allclose(np.einsum("i,ia,ib->ab", w, c, c), np.eye(3) / 3, atol=1e-16)
    d = np.eye(3)
    iso = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d) + np.einsum("ad,bc->abcd", d, d)) / 9
    assert np.allclose(np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c), iso, atol=1e-16)
    assert len({tuple(v) for v in c.astype(int).tolist()}) == 19
    for v in c:
        assert any((u == -v).all() for u in c)


def test_rest_state_is_a_fixed_point():
    fl = oracle.Fluid(4, 5, 3, 0.8, 0.0, 0.0)
    f0 = fl.f.copy()
    for _ in range(5):
        fl.step()
    assert np.abs(fl.f - f0).max() < 1e-16


@pytest.mark.parametrize("tau", [1.0, 0.8, 1.7])
def test_couette_profile_is_exact(tau):
    """Steady plane Couette flow between walls moving at -/+u_w is linear:
    u_x = u_w (2 (y + 1/2) / H - 1) with H = ny (Sec. 6.1, u_wall = H gamma/2)."""
    H = 8
    fl = oracle.Fluid(2, H, 1, tau, -0.01, 0.01)
    for _ in range(2500):
        fl.step()
    y = np.arange(H)
    exact = 0.01 * (2 * (y + 0.5) / H - 1)
    assert np.abs(fl.u[0, :, 0, 0] - exact).max() < 1e-13
    assert np.abs(fl.u[..., 1:]).max() < 1e-13
    assert np.allclose(fl.u[..., 0], fl.u[:1, :, :1, 0], atol=1e-16)  # independent of x, z


def _poiseuille(H, tau, g, steps):
    fl = oracle.Fluid(2, H, 1, tau, 0.0, 0.0, (g, 0.0, 0.0))
    for _ in range(steps):
        fl.step()
    nu = (tau - 0.5) / 3
    y = np.arange(H)
    exact = g / (2 * nu) * (y + 0.5) * (H - y - 0.5)
    return fl.u[0, :, 0, 0], exact


def test_poiseuille_exact_at_magic_tau():
    """With halfway bounce-back, BGK reproduces the parabolic profile exactly
    when (tau - 1/2)^2 = 3/16 (Ginzburg & d'Humieres' magic parameter)."""
    ux, exact = _poiseuille(10, 0.5 + np.sqrt(3) / 4, 1e-5, 6000)
    assert np.abs(ux - exact).max() < 1e-10 * exact.max()


def test_poiseuille_converges_second_order_at_tau_one():
    """At tau = 1 the wall slip is O(H^-2) relative to u_max."""
    errs = []
    for H in (6, 12):
        g = 1e-4 / H**2
        ux, exact = _poiseuille(H, 1.0, g, 400 * H * H // 6 + 2000)
        errs.append(np.abs(ux - exact).max() / exact.max())
    assert errs[0] < 2e-2
    assert 3.5 < errs[0] / errs[1] < 4.5


def test_mass_is_conserved_with_walls_and_forces():
    fl = oracle.Fluid(6, 7, 5, 0.9, -0.02, 0.03, (1e-5, -2e-5, 3e-6))
    m0 = fl.total_mass()
    for _ in range(40):
        fl.step(RNG.normal(scale=1e-4, size=(5, 7, 6, 3)))
    assert abs(fl.total_mass() - m0) < 1e-12 * m0


def test_guo_forcing_adds_exactly_F_per_step():
    """Total momentum grows by exactly sum F per step while the disturbance
    has not reached the (resting) walls."""
    fl = oracle.Fluid(8, 16, 8, 1.0, 0.0, 0.0)
    Fn = np.zeros((8, 16, 8, 3))
    Fn[3:5, 7:9, 2:6] = RNG.normal(scale=1e-3, size=(2, 2, 4, 3))
    P = np.zeros(3)
    for _ in range(4):
        fl.step(Fn)
        P += Fn.sum((0, 1, 2))
        assert np.allclose(fl.total_momentum(), P, rtol=1e-10, atol=1e-13)


def test_post_collision_momentum_identity():
    """After collision with force F: sum_i c_i f*_i = rho u + F/2 at every
    node (the collision moves momentum by exactly F and rho u includes F/2).
    The GPU interpolation reconstructs u(t) from post-collision populations
    through this identity."""
    fl = oracle.Fluid(5, 6, 4, 0.7, -0.01, 0.02, (2e-6, 0.0, 0.0))
    for _ in range(3):
        fl.step(RNG.normal(scale=1e-4, size=(4, 6, 5, 3)))
    Fn = RNG.normal(scale=1e-4, size=(4, 6, 5, 3))
    fl.step(Fn)
    c, _ = oracle.lattice()
    mom = np.einsum("zyxi,ia->zyxa", fl.f, c.astype(float))
    Ftot = Fn + fl.g
    assert np.allclose(mom - Ftot / 2, fl.rho[..., None] * fl.u, rtol=0, atol=1e-16)
    assert np.allclose(fl.f.sum(-1), fl.rho, rtol=0, atol=1e-15)
