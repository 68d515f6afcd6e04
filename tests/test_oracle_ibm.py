"""Pins of the oracle's immersed-boundary transfer (trilinear delta kernel)."""
import numpy as np
import pytest

import oracle

RNG = np.random.default_rng(3)
NX, NY, NZ = 12, 10, 8


def points(n, lo=(1.0, 1.0, 1.0), hi=(NX - 2.0, NY - 2.0, NZ - 2.0)):
    return RNG.uniform(lo, hi, (n, 3))


def test_partition_of_unity_and_first_moment():
    """sum_x F(x) = sum_v f_v and sum_x x F(x)^T = sum_v y_v f_v^T (away from
    the periodic seams, so node coordinates are not wrapped)."""
    y, f = points(50), RNG.normal(size=(50, 3))
    Fn = oracle.spread(y, f, NX, NY, NZ)
    assert np.allclose(Fn.sum((0, 1, 2)), f.sum(0), rtol=0, atol=1e-12)
    zz, yy, xx = np.meshgrid(np.arange(NZ), np.arange(NY), np.arange(NX), indexing="ij")
    X = np.stack([xx, yy, zz], -1).astype(float)
    first = np.einsum("zyxa,zyxb->ab", X, Fn)
    assert np.allclose(first, y.T @ f, rtol=0, atol=1e-11)


def test_spread_brute_force():
    """Against the definition evaluated on every node: delta_h(x - y) =
    phi(dx) phi(dy) phi(dz), phi(r) = max(0, 1 - |r|), x and z periodic."""
    y, f = points(7, lo=(0.0, 0.5, 0.0), hi=(NX, NY - 1.5, NZ)), RNG.normal(size=(7, 3))
    Fn = oracle.spread(y, f, NX, NY, NZ)
    ref = np.zeros_like(Fn)
    for v in range(len(y)):
        for z in range(NZ):
            for yy in range(NY):
                for x in range(NX):
                    dx = min(abs(x - y[v, 0]), NX - abs(x - y[v, 0]))
                    dz = min(abs(z - y[v, 2]), NZ - abs(z - y[v, 2]))
                    d = max(0, 1 - dx) * max(0, 1 - abs(yy - y[v, 1])) * max(0, 1 - dz)
                    ref[z, yy, x] += d * f[v]
    assert np.allclose(Fn, ref, rtol=0, atol=1e-13)


def test_interpolation_exact_for_linear_fields():
    a = RNG.normal(size=3)
    G = RNG.normal(size=(3, 3))
    zz, yy, xx = np.meshgrid(np.arange(NZ), np.arange(NY), np.arange(NX), indexing="ij")
    X = np.stack([xx, yy, zz], -1).astype(float)
    u = a + X @ G.T
    y = points(40)
    assert np.allclose(oracle.interp(y, u), a + y @ G.T, rtol=0, atol=1e-12)


def test_spread_and_interp_are_adjoint():
    y, f = points(30), RNG.normal(size=(30, 3))
    u = RNG.normal(size=(NZ, NY, NX, 3))
    lhs = np.sum(oracle.spread(y, f, NX, NY, NZ) * u)
    rhs = np.sum(f * oracle.interp(y, u))
    assert np.isclose(lhs, rhs, rtol=1e-13)


@pytest.mark.parametrize("yv", [-0.2, NY - 1 + 0.1])
def test_support_outside_walls_is_rejected(yv):
    y = np.array([[3.0, yv, 3.0]])
    with pytest.raises(oracle.DomainError):
        oracle.spread(y, np.ones((1, 3)), NX, NY, NZ)
    with pytest.raises(oracle.DomainError):
        oracle.interp(y, np.zeros((NZ, NY, NX, 3)))
