"""Pins of the oracle's immersed-boundary transfer: the trilinear delta
kernel (support width 2) and Peskin's four-point kernel (width 4; C. S.
Peskin, The immersed boundary method, Acta Numerica 11, 2002, Sec. 6, which
derives it from the conditions pinned here: partition of unity, zero first
moment, equal even and odd sums, and a constant sum of squares 3/8)."""
import numpy as np
import pytest

import oracle

RNG = np.random.default_rng(3)
NX, NY, NZ = 12, 10, 8


def points(n, lo=(2.0, 2.0, 2.0), hi=(NX - 3.0, NY - 3.0, NZ - 3.0)):
    return RNG.uniform(lo, hi, (n, 3))


WIDTHS = [2, 4]


@pytest.mark.parametrize("width", WIDTHS)
def test_partition_of_unity_and_first_moment(width):
    """sum_x F(x) = sum_v f_v and sum_x x F(x)^T = sum_v y_v f_v^T (away from
    the periodic seams, so node coordinates are not wrapped)."""
    y, f = points(50), RNG.normal(size=(50, 3))
    Fn = oracle.spread(y, f, NX, NY, NZ, width=width)
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


@pytest.mark.parametrize("width", WIDTHS)
def test_interpolation_exact_for_linear_fields(width):
    a = RNG.normal(size=3)
    G = RNG.normal(size=(3, 3))
    zz, yy, xx = np.meshgrid(np.arange(NZ), np.arange(NY), np.arange(NX), indexing="ij")
    X = np.stack([xx, yy, zz], -1).astype(float)
    u = a + X @ G.T
    y = points(40)
    assert np.allclose(oracle.interp(y, u, width=width), a + y @ G.T, rtol=0, atol=1e-12)


@pytest.mark.parametrize("width", WIDTHS)
def test_spread_and_interp_are_adjoint(width):
    y, f = points(30), RNG.normal(size=(30, 3))
    u = RNG.normal(size=(NZ, NY, NX, 3))
    lhs = np.sum(oracle.spread(y, f, NX, NY, NZ, width=width) * u)
    rhs = np.sum(f * oracle.interp(y, u, width=width))
    assert np.isclose(lhs, rhs, rtol=1e-13)


@pytest.mark.parametrize("width,yv", [(2, -0.2), (2, NY - 1 + 0.1), (4, 0.9), (4, NY - 2 + 0.1)])
def test_support_outside_walls_is_rejected(width, yv):
    y = np.array([[3.0, yv, 3.0]])
    with pytest.raises(oracle.DomainError):
        oracle.spread(y, np.ones((1, 3)), NX, NY, NZ, width=width)
    with pytest.raises(oracle.DomainError):
        oracle.interp(y, np.zeros((NZ, NY, NX, 3)), width=width)


@pytest.mark.parametrize("yv", [1.0, NY - 3 + 0.999])
def test_peskin_support_touching_the_walls_is_accepted(yv):
    y = np.array([[3.0, yv, 3.0]])
    Fn = oracle.spread(y, np.ones((1, 3)), NX, NY, NZ, width=4)
    assert np.isclose(Fn.sum(), 3.0, rtol=1e-14)


def test_peskin_sum_of_squares_and_even_odd_split():
    """For one unit force at any point: sum_x delta_h^2 = (3/8)^3, and on each
    axis the nodes of even and of odd index carry half of the force each."""
    zz, yy, xx = np.meshgrid(np.arange(NZ), np.arange(NY), np.arange(NX), indexing="ij")
    for y in points(20):
        Fn = oracle.spread(y[None], np.array([[1.0, 0.0, 0.0]]), NX, NY, NZ, width=4)[..., 0]
        assert np.isclose((Fn ** 2).sum(), (3 / 8) ** 3, rtol=1e-13)
        for idx in (xx, yy, zz):
            assert np.isclose(Fn[idx % 2 == 0].sum(), 0.5, rtol=1e-13)
        assert np.count_nonzero(Fn) <= 64


def test_peskin_values_on_a_node():
    """A point on a node: phi(0) = 1/2, phi(1) = 1/4, phi(2) = 0 per axis."""
    y = np.array([[5.0, 4.0, 3.0]])
    Fn = oracle.spread(y, np.array([[1.0, 0.0, 0.0]]), NX, NY, NZ, width=4)[..., 0]
    phi = {0: 0.5, 1: 0.25, 2: 0.0}
    for dz in (-2, -1, 0, 1, 2):
        for dy in (-2, -1, 0, 1, 2):
            for dx in (-2, -1, 0, 1, 2):
                want = phi[abs(dx)] * phi[abs(dy)] * phi[abs(dz)]
                assert np.isclose(Fn[3 + dz, 4 + dy, 5 + dx], want, rtol=0, atol=1e-15)
    assert np.isclose(Fn.sum(), 1.0, rtol=1e-14)


def test_peskin_spread_across_the_periodic_seam():
    """Near x = 0 and z = 0 the support wraps: moments taken with the nodes'
    unwrapped coordinates hold."""
    y = np.array([[0.3, 4.6, NZ - 0.4]])
    f = np.array([[0.7, -1.1, 0.4]])
    Fn = oracle.spread(y, f, NX, NY, NZ, width=4)
    assert np.allclose(Fn.sum((0, 1, 2)), f[0], rtol=0, atol=1e-14)
    zz, yy, xx = np.meshgrid(np.arange(NZ), np.arange(NY), np.arange(NX), indexing="ij")
    xu = np.where(xx > NX // 2, xx - NX, xx).astype(float)   # nodes left of the seam at negative x
    zu = np.where(zz < NZ // 2, zz + NZ, zz).astype(float)   # nodes right of z = NZ at z >= NZ
    for coord, yc in ((xu, y[0, 0]), (yy.astype(float), y[0, 1]), (zu, y[0, 2])):
        assert np.allclose(np.einsum("zyx,zyxb->b", coord, Fn), yc * f[0], rtol=0, atol=1e-13)
