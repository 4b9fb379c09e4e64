"""Pins of the oracle's 1D DGSEM operators (Sec. 3.1: Lagrange polynomials on
Legendre-Gauss nodes, collocated Gauss quadrature) and of the low-storage Runge-Kutta
tables (Sec. 3.1, Kennedy & Carpenter)."""
import math

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg
from numpy.polynomial import polynomial as nppoly


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 7, 15])
def test_gauss_legendre_vs_numpy(orc, n):
    x, w = orc.gauss_legendre(n)
    xr, wr = npleg.leggauss(n)
    assert np.allclose(x, xr, atol=1e-15, rtol=0)
    assert np.allclose(w, wr, atol=1e-15, rtol=0)
    assert abs(w.sum() - 2.0) < 1e-14
    for k in range(2 * n):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.dot(w, x ** k) - exact) < 1e-14


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6])
def test_lagrange_and_derivative_matrix(orc, N):
    xi, _ = orc.gauss_legendre(N + 1)
    # cardinal property and partition of unity
    for i in range(N + 1):
        l = orc.lagrange_at(N, xi, xi[i])
        assert np.allclose(l, np.eye(N + 1)[i], atol=1e-14)
    for x in (-1.0, -0.3, 0.77, 1.0):
        assert abs(orc.lagrange_at(N, xi, x).sum() - 1.0) < 1e-13
    D = orc.dmatrix(N, xi)
    rng = np.random.default_rng(N)
    for _ in range(3):
        c = rng.normal(size=N + 1)  # random polynomial of degree N
        f = nppoly.polyval(xi, c)
        df = nppoly.polyval(xi, nppoly.polyder(c))
        assert np.allclose(D @ f, df, atol=1e-11 * max(1, np.abs(df).max()))
        # interpolation to the element ends is exact for degree N
        for x in (-1.0, 1.0):
            assert abs(orc.lagrange_at(N, xi, x) @ f - nppoly.polyval(x, c)) < 1e-12


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5])
def test_weak_lifting_equals_strong(orc, N):
    """Discrete integration by parts of the collocated Gauss DGSEM (summation by parts):
    with face values equal to the element's own traces the weak-form BR1 gradient
    sum_l Dhat_il f_l + (l_i(1) f(1) - l_i(-1) f(-1))/w_i equals the strong form D f."""
    xi, w = orc.gauss_legendre(N + 1)
    D = orc.dmatrix(N, xi)
    Dhat = -(w[None, :] / w[:, None]) * D.T
    lm, lp = orc.lagrange_at(N, xi, -1.0), orc.lagrange_at(N, xi, 1.0)
    f = np.random.default_rng(7).normal(size=N + 1)
    weak = Dhat @ f + (lp * (lp @ f) - lm * (lm @ f)) / w
    assert np.allclose(weak, D @ f, atol=1e-12)


def _stability_poly(A, B, z):
    """Apply the 2N-storage recursion to y' = z y for one step of size 1."""
    y, g = 1.0 + 0j, 0j
    for a, b in zip(A, B):
        g = a * g + z * y
        y = y + b * g
    return y


@pytest.mark.parametrize("rk,order", [(3, 3), (4, 4)])
def test_rk_order_conditions(orc, rk, order):
    """Linear order conditions: the stability polynomial matches exp(z) up to z^order."""
    A, B, c = orc.rk_coeffs(rk)
    zs = 0.3 * np.exp(2j * np.pi * np.arange(16) / 16)
    vals = np.array([_stability_poly(A, B, z) for z in zs])
    # fit the polynomial of degree = number of stages
    ns = len(A)
    V = np.vander(zs, ns + 1, increasing=True)
    coef = np.linalg.lstsq(V, vals, rcond=None)[0].real
    fact = np.array([1.0 / math.factorial(k) for k in range(ns + 1)])
    assert np.allclose(coef[: order + 1], fact[: order + 1], atol=1e-10)
    if order + 1 <= ns:  # and not beyond: the order is exactly `order`
        assert abs(coef[order + 1] - fact[order + 1]) > 1e-6


@pytest.mark.parametrize("rk", [3, 4])
def test_rk_stage_times(orc, rk):
    """Stage times c_s are the times at which the 2N recursion evaluates the right-hand
    side: integrating y' = t^k exactly for k < order pins them (quadrature conditions)."""
    A, B, c = orc.rk_coeffs(rk)
    order = 3 if rk == 3 else 4
    for k in range(order):
        y, g = 0.0, 0.0
        for a, b, cs in zip(A, B, c):
            g = a * g + cs ** k
            y = y + b * g
        assert abs(y - 1.0 / (k + 1)) < 1e-12
