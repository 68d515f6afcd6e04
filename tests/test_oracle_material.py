"""Pins of the oracle's material law (Sec. 2) and derivative table (Sec. 3.2).

The oracle evaluates the paper's table entry by entry and chains them as the
force equation of Sec. 3.1 does. These tests check it against things other
than itself: finite differences of its own invariants and energy, a computer
algebra derivative of the energy density, the textbook neo-Hookean stress,
a hand-derived uniaxial closed form, linear elasticity at small strain, the
rest state and frame invariance.
"""
import numpy as np
import pytest

import oracle

RNG = np.random.default_rng(7)


def random_F(scale=0.3, rng=RNG):
    while True:
        F = np.eye(3) + scale * rng.uniform(-1, 1, (3, 3))
        if np.linalg.det(F) > 0.3:
            return F


def fd_matrix(fun, F, h=1e-6):
    G = np.zeros((3, 3))
    for i in range(3):
        for j in range(3):
            Fp, Fm = F.copy(), F.copy()
            Fp[i, j] += h
            Fm[i, j] -= h
            G[i, j] = (fun(Fp) - fun(Fm)) / (2 * h)
    return G


MATS = [(1e-3, 0.0, 0.1), (0.0, 1e-3, 0.1), (0.6, 0.4, 50.0), (1.0, 0.0, 0.0), (0.0, 1.0, 0.0), (0.0, 0.0, 1.0)]


@pytest.mark.parametrize("mat", MATS)
def test_P_is_energy_gradient(mat):
    """dU/dF assembled from the table equals the finite-difference gradient
    of the energy density U(F)."""
    mu1, mu2, kappa = mat
    for _ in range(5):
        F = random_F()
        P = oracle.mr_eval(F, mu1, mu2, kappa)["P"]
        G = fd_matrix(lambda X: oracle.mr_eval(X, mu1, mu2, kappa)["U"], F)
        scale = max(np.abs(G).max(), 1e-300)
        assert np.abs(P - G).max() <= 1e-7 * scale


def test_matrix_entries_by_finite_differences():
    """dT_C/dF, dJ/dF and dT_C2/dF against finite differences of T_C, J, T_C2."""
    for _ in range(5):
        F = random_F()
        d = oracle.mr_eval(F, 1.0, 1.0, 1.0)
        for name, key in (("dTC_dF", "T_C"), ("dJ_dF", "J"), ("dTC2_dF", "T_C2")):
            G = fd_matrix(lambda X: oracle.mr_eval(X, 1.0, 1.0, 1.0)[key], F)
            assert np.allclose(d[name], G, rtol=1e-7, atol=1e-8), name


def test_scalar_entries_by_finite_differences():
    """The scalar entries reproduce the F-gradients of I and K:
    dI/dF = dI/dT_C dT_C/dF + dI/dJ dJ/dF, and
    dK/dF = dK/dT_C dT_C/dF + dK/dJ dJ/dF + dK/dT_C2 dT_C2/dF;
    the three matrices are linearly independent for a generic F, so each
    scalar entry is pinned. dU/dI, dU/dK, dU/dJ are pinned by varying the
    moduli and J."""
    for _ in range(5):
        F = random_F()
        d = oracle.mr_eval(F, 1.0, 1.0, 1.0)
        gI = fd_matrix(lambda X: oracle.mr_eval(X, 1.0, 1.0, 1.0)["I"], F)
        gK = fd_matrix(lambda X: oracle.mr_eval(X, 1.0, 1.0, 1.0)["K"], F)
        assert np.allclose(d["dI_dTC"] * d["dTC_dF"] + d["dI_dJ"] * d["dJ_dF"], gI, rtol=1e-7, atol=1e-8)
        assert np.allclose(d["dK_dTC"] * d["dTC_dF"] + d["dK_dJ"] * d["dJ_dF"] + d["dK_dTC2"] * d["dTC2_dF"], gK,
                           rtol=1e-7, atol=1e-8)
        # U is linear in (mu1, mu2): dU/dI = mu1/2 means U(mu1) - U(0) = mu1 (I - 3) / 2
        u1 = oracle.mr_eval(F, 2.0, 0.0, 0.0)
        assert np.isclose(u1["dU_dI"], 1.0) and np.isclose(u1["U"], u1["dU_dI"] * (u1["I"] - 3.0))
        u2 = oracle.mr_eval(F, 0.0, 2.0, 0.0)
        assert np.isclose(u2["dU_dK"], 1.0) and np.isclose(u2["U"], u2["dU_dK"] * (u2["K"] - 3.0))
        # dU/dJ = kappa (J - 1): along F(s) = s^(1/3) F, T_C J^-2/3 and K are constant
        s = 1.0 + 1e-6
        a = oracle.mr_eval(F * s ** (1 / 3), 0.0, 0.0, 3.0)
        b = oracle.mr_eval(F / s ** (1 / 3), 0.0, 0.0, 3.0)
        assert np.isclose((a["U"] - b["U"]) / (a["J"] - b["J"]), d["dU_dJ"] * 3.0, rtol=1e-6)


def test_against_computer_algebra():
    """P from the table equals the symbolic derivative of the energy density
    written from the definitions of Sec. 2 (sympy)."""
    sp = pytest.importorskip("sympy")
    Fs = sp.Matrix(3, 3, sp.symbols("f0:9"))
    mu1, mu2, kap = sp.symbols("mu1 mu2 kappa", positive=True)
    C = Fs.T * Fs
    J = Fs.det()
    TC = C.trace()
    TC2 = (C * C).trace()
    U = mu1 / 2 * (TC * J ** sp.Rational(-2, 3) - 3) + mu2 / 2 * (
        (TC**2 - TC2) / 2 * J ** sp.Rational(-4, 3) - 3) + kap / 2 * (J - 1) ** 2
    grads = [sp.lambdify((Fs, mu1, mu2, kap), sp.diff(U, Fs[i, j]), "numpy") for i in range(3) for j in range(3)]
    for _ in range(4):
        F = random_F()
        m = (0.7, 0.3, 20.0)
        ref = np.array([g(sp.Matrix(F), *m) for g in grads], dtype=float).reshape(3, 3)
        P = oracle.mr_eval(F, *m)["P"]
        assert np.allclose(P, ref, rtol=1e-11, atol=1e-12)


def test_rest_state():
    d = oracle.mr_eval(np.eye(3), 0.7, 0.3, 20.0)
    assert d["J"] == 1.0 and d["I"] == 3.0 and d["K"] == 3.0
    assert abs(d["U"]) < 1e-15
    assert np.abs(d["P"]).max() < 1e-13


def test_neo_hookean_limit():
    """w = 1 (mu_2 = 0) gives the textbook compressible neo-Hookean stress
    P = mu J^-2/3 (F - T_C/3 F^-T) + kappa (J - 1) J F^-T (Bower, Ch. 3)."""
    for _ in range(5):
        F = random_F()
        mu, kappa = 0.8, 11.0
        J = np.linalg.det(F)
        FinvT = np.linalg.inv(F).T
        TC = np.trace(F.T @ F)
        ref = mu * J ** (-2 / 3) * (F - TC / 3 * FinvT) + kappa * (J - 1) * J * FinvT
        assert np.allclose(oracle.mr_eval(F, mu, 0.0, kappa)["P"], ref, rtol=1e-12, atol=1e-13)


def test_uniaxial_closed_form():
    """F = diag(lam, 1, 1): J = lam, T_C = lam^2 + 2, K = (2 lam^2 + 1) lam^-4/3
    and P_11 = dU/dlam derived by hand."""
    mu1, mu2, kappa = 0.6, 0.4, 9.0
    for lam in (0.5, 0.8, 1.0, 1.3, 2.8):
        d = oracle.mr_eval(np.diag([lam, 1.0, 1.0]), mu1, mu2, kappa)
        I = (lam**2 + 2) * lam ** (-2 / 3)
        K = (2 * lam**2 + 1) * lam ** (-4 / 3)
        U = mu1 / 2 * (I - 3) + mu2 / 2 * (K - 3) + kappa / 2 * (lam - 1) ** 2
        dI = 2 * lam ** (1 / 3) - 2 / 3 * (lam**2 + 2) * lam ** (-5 / 3)
        dK = 4 * lam ** (-1 / 3) - 4 / 3 * (2 * lam**2 + 1) * lam ** (-7 / 3)
        P11 = mu1 / 2 * dI + mu2 / 2 * dK + kappa * (lam - 1)
        assert np.isclose(d["I"], I, rtol=1e-14) and np.isclose(d["K"], K, rtol=1e-14)
        assert np.isclose(d["U"], U, rtol=1e-12, atol=1e-15)
        assert np.isclose(d["P"][0, 0], P11, rtol=1e-12, atol=1e-14)
        assert np.allclose(d["P"][[0, 0, 1, 1, 2, 2], [1, 2, 0, 2, 0, 1]], 0.0, atol=1e-14)


def test_small_strain_is_linear_elasticity():
    """P -> 2 mu eps_dev + kappa tr(eps) I with mu = mu_1 + mu_2 (Sec. 2)."""
    mu1, mu2, kappa = 0.6, 0.4, 9.0
    G = RNG.uniform(-1, 1, (3, 3))
    errs = []
    for e in (1e-3, 1e-4):
        H = e * G
        eps = 0.5 * (H + H.T)
        lin = 2 * (mu1 + mu2) * (eps - np.trace(eps) / 3 * np.eye(3)) + kappa * np.trace(eps) * np.eye(3)
        P = oracle.mr_eval(np.eye(3) + H, mu1, mu2, kappa)["P"]
        errs.append(np.abs(P - lin).max() / np.abs(lin).max())
    assert errs[0] < 1e-2 and errs[1] < errs[0] / 5  # O(eps) relative error


def test_frame_invariance():
    """U depends on F only through C = F^T F: U(QF) = U(F), P(QF) = Q P(F)."""
    from scipy.spatial.transform import Rotation

    for _ in range(5):
        F = random_F()
        Q = Rotation.random(random_state=int(RNG.integers(1 << 30))).as_matrix()
        a = oracle.mr_eval(F, 0.6, 0.4, 9.0)
        b = oracle.mr_eval(Q @ F, 0.6, 0.4, 9.0)
        assert np.isclose(a["U"], b["U"], rtol=1e-12, atol=1e-15)
        assert np.allclose(Q @ a["P"], b["P"], rtol=1e-11, atol=1e-13)
