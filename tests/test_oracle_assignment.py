"""Pins of the oracle's assignment function and stencil (readings R1, R2).

The paper (Sec. 3.1) only says the stencil coefficients are a product of three
1-D polynomials of order S.  These tests pin the oracle's B-spline to facts it
does not compute itself: textbook NGP/CIC/TSC shapes, its Fourier transform
sinc^P by quadrature, partition of unity and symmetry.
"""
import math

import numpy as np
import pytest

from oracle import bspline, bspline_deriv, stencil, make_rho, wrap_positions

ORDERS = [1, 2, 3, 4, 5, 6, 7]


def test_ngp_cic_tsc_textbook():
    s = np.linspace(-2.0, 2.0, 4001)
    ngp = np.where((s >= -0.5) & (s < 0.5), 1.0, 0.0)
    cic = np.maximum(0.0, 1.0 - np.abs(s))
    a = np.abs(s)
    tsc = np.where(a < 0.5, 0.75 - a * a, np.where(a < 1.5, 0.5 * (1.5 - a) ** 2, 0.0))
    np.testing.assert_array_equal(bspline(1, s), ngp)
    np.testing.assert_allclose(bspline(2, s), cic, atol=1e-15)
    np.testing.assert_allclose(bspline(3, s), tsc, atol=1e-15)


@pytest.mark.parametrize("P", ORDERS)
def test_partition_of_unity_and_symmetry(P):
    r = np.random.default_rng(11)
    u = r.uniform(-50, 50, 2000)
    _, s = stencil(u, P, 97)
    np.testing.assert_allclose(bspline(P, s).sum(axis=1), 1.0, atol=1e-14)
    t = r.uniform(-P / 2, P / 2, 500)
    np.testing.assert_allclose(bspline(P, t), bspline(P, -t), atol=1e-15)
    # support [-P/2, P/2]
    assert np.all(bspline(P, np.array([-P / 2 - 1e-9, P / 2 + 1e-9])) == 0.0)


@pytest.mark.parametrize("P", ORDERS)
def test_fourier_transform_is_sinc_power(P):
    """int M_P(s) e^{-i k s} ds = sinc^P(k/2) (P-fold convolution of the
    top-hat), by Gauss-Legendre on each unit piece."""
    xg, wg = np.polynomial.legendre.leggauss(24)
    lo = -P / 2.0
    nodes = np.concatenate([lo + j + 0.5 * (xg + 1) for j in range(P)])
    weights = np.concatenate([0.5 * wg for _ in range(P)])
    for k in [0.0, 0.3, 1.0, 2.5, math.pi, 5.0, 9.0]:
        val = np.sum(weights * bspline(P, nodes) * np.cos(k * nodes))
        ref = np.sinc(k / (2 * math.pi)) ** P
        assert abs(val - ref) < 1e-13


@pytest.mark.parametrize("P", ORDERS[1:])
def test_derivative_matches_finite_difference(P):
    r = np.random.default_rng(5)
    s = r.uniform(-P / 2 + 0.01, P / 2 - 0.01, 400)
    # keep away from the knots, where the derivative of P=2 jumps
    knots = np.arange(-P / 2, P / 2 + 1)
    s = s[np.min(np.abs(s[:, None] - knots[None, :]), axis=1) > 1e-3]
    h = 1e-6
    fd = (bspline(P, s + h) - bspline(P, s - h)) / (2 * h)
    np.testing.assert_allclose(bspline_deriv(P, s), fd, atol=5e-8)


@pytest.mark.parametrize("P", ORDERS)
def test_stencil_anchor(P):
    u = np.array([0.0, 0.49, 0.51, 3.2, 3.7, 9.99])
    pts, s = stencil(u, P, 10)
    n = np.floor(u + 0.5) if P % 2 else np.floor(u)
    first = np.mod(n - (P - 1) // 2, 10)
    np.testing.assert_array_equal(pts[:, 0], first)
    # every stencil offset lies inside the support of M_P
    assert np.all(np.abs(s) <= P / 2 + 1e-12)
    if P % 2:
        # odd P: the anchor is the nearest grid point
        assert np.all(np.abs(s[:, (P - 1) // 2]) <= 0.5)


def test_wrap_positions():
    box = np.array([10.0, 20.0, 30.0])
    x = np.array([[-1e-17, 20.0, 61.0], [10.0, -20.0, -0.5]])
    xw = wrap_positions(x, box)
    assert np.all(xw >= 0) and np.all(xw < box)
    np.testing.assert_allclose(xw[1], [0.0, 0.0, 29.5])


@pytest.mark.parametrize("P", [3, 5, 7])
def test_single_charge_on_mesh_point(P):
    """A charge on a mesh point (odd P) fills exactly its P^3 stencil with the
    separable product M_P(i) M_P(j) M_P(k) / h^3."""
    box, mesh = (8.0, 8.0, 8.0), (16, 16, 16)
    h = 0.5
    x = np.array([[3.0, 2.5, 6.0]])
    rho = make_rho(x, np.array([2.0]), box, mesh, P)
    w1 = bspline(P, np.arange(P) - (P - 1) // 2)
    ref = np.zeros(mesh)
    c = (6, 5, 12)
    r = (P - 1) // 2
    for a in range(P):
        for b in range(P):
            for cc in range(P):
                ref[(c[0] - r + a) % 16, (c[1] - r + b) % 16, (c[2] - r + cc) % 16] += 2.0 * w1[a] * w1[b] * w1[cc] / h ** 3
    np.testing.assert_allclose(rho, ref, atol=1e-14)
    assert np.count_nonzero(rho) == P ** 3


@pytest.mark.parametrize("P", [2, 3, 4, 5, 6, 7])
def test_charge_conservation(P):
    r = np.random.default_rng(3)
    box = np.array([9.0, 11.0, 13.0])
    mesh = (9, 12, 10)
    x = r.uniform(-5, 25, (300, 3))
    q = r.normal(size=300)
    rho = make_rho(x, q, box, mesh, P)
    hv = np.prod(box / np.array(mesh))
    assert abs(rho.sum() * hv - q.sum()) <= 1e-13 * np.abs(q).sum()
