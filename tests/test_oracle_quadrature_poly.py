"""Pins for the oracle's quadrature and polynomial routines (CPU only)."""
import numpy as np
import pytest
import scipy.special as ss

from oracle.polynomials import jacobi, jacobi_deriv, lagrange, lagrange_deriv
from oracle.quadrature import gauss_jacobi, gauss_legendre, gauss_lobatto_legendre


@pytest.mark.parametrize("m", [1, 2, 3, 5, 8, 10, 12])
def test_gauss_legendre_exact_monomials(m):
    x, w = gauss_legendre(m)
    for k in range(2 * m):
        exact = 2.0 / (k + 1) if k % 2 == 0 else 0.0
        assert abs(np.sum(w * x ** k) - exact) < 1e-14
    # degree 2m is not integrated exactly: the rule is genuinely m-point
    assert abs(np.sum(w * x ** (2 * m)) - 2.0 / (2 * m + 1)) > 1e-10


@pytest.mark.parametrize("m", [2, 6, 10])
def test_gauss_legendre_matches_numpy(m):
    x, w = gauss_legendre(m)
    xr, wr = np.polynomial.legendre.leggauss(m)
    assert np.allclose(x, xr, atol=1e-14) and np.allclose(w, wr, atol=1e-14)


def test_gauss_jacobi_weighted_exactness():
    a, b = 1.0, 1.0
    x, w = gauss_jacobi(4, a, b)
    # int (1-x)(1+x) x^2 dx = 4/15
    assert abs(np.sum(w * x ** 2) - 4.0 / 15.0) < 1e-14


def test_gll_known_points():
    assert np.allclose(gauss_lobatto_legendre(2), [-1, 0, 1], atol=1e-15)
    assert np.allclose(gauss_lobatto_legendre(3), [-1, -1 / np.sqrt(5), 1 / np.sqrt(5), 1], atol=1e-15)
    assert np.allclose(gauss_lobatto_legendre(4), [-1, -np.sqrt(3 / 7), 0, np.sqrt(3 / 7), 1], atol=1e-15)


@pytest.mark.parametrize("P", [2, 5, 8])
def test_gll_quadrature_exact(P):
    # GLL weights 2 / (P (P+1) L_P(x)^2) integrate degree 2P-1 exactly
    x = gauss_lobatto_legendre(P)
    w = 2.0 / (P * (P + 1) * jacobi(P, 0.0, 0.0, x) ** 2)
    for k in range(2 * P):
        exact = 2.0 / (k + 1) if k % 2 == 0 else 0.0
        assert abs(np.sum(w * x ** k) - exact) < 1e-13


@pytest.mark.parametrize("n,a,b", [(0, 1, 1), (3, 1, 1), (6, 1, 1), (5, 0, 0), (4, 2, 0.5)])
def test_jacobi_matches_scipy(n, a, b):
    x = np.linspace(-1, 1, 13)
    assert np.allclose(jacobi(n, a, b, x), ss.eval_jacobi(n, a, b, x), atol=1e-12)
    h = 1e-6
    fd = (jacobi(n, a, b, x + h) - jacobi(n, a, b, x - h)) / (2 * h)
    assert np.allclose(jacobi_deriv(n, a, b, x), fd, atol=1e-6)


def test_jacobi_orthogonality():
    x, w = gauss_jacobi(12, 1.0, 1.0)
    G = np.array([[np.sum(w * jacobi(i, 1, 1, x) * jacobi(j, 1, 1, x)) for j in range(8)] for i in range(8)])
    off = G - np.diag(np.diag(G))
    assert np.abs(off).max() < 1e-12


def test_lagrange_collocation_and_partition():
    nodes = gauss_lobatto_legendre(6)
    L = np.array([lagrange(nodes, a, nodes) for a in range(7)])
    assert np.allclose(L, np.eye(7), atol=1e-14)
    x = np.linspace(-1, 1, 17)
    assert np.allclose(sum(lagrange(nodes, a, x) for a in range(7)), 1.0, atol=1e-13)
    assert np.allclose(sum(lagrange_deriv(nodes, a, x) for a in range(7)), 0.0, atol=1e-11)
    h = 1e-6
    for a in range(7):
        fd = (lagrange(nodes, a, x + h) - lagrange(nodes, a, x - h)) / (2 * h)
        assert np.allclose(lagrange_deriv(nodes, a, x), fd, atol=1e-6)


@pytest.mark.parametrize("P", [1, 2, 3, 5, 8])
def test_gll_rule_exactness(P):
    from oracle.quadrature import gauss_lobatto_legendre_rule
    x, w = gauss_lobatto_legendre_rule(P)
    for k in range(2 * P):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.sum(w * x ** k) - exact) < 1e-13
    if P >= 2:
        # degree 2P is not integrated exactly (P + 1 point Lobatto rule)
        assert abs(np.sum(w * x ** (2 * P)) - 2.0 / (2 * P + 1)) > 1e-6


def test_gll_rule_textbook_values():
    from oracle.quadrature import gauss_lobatto_legendre_rule
    x, w = gauss_lobatto_legendre_rule(2)
    assert np.allclose(x, [-1, 0, 1]) and np.allclose(w, [1 / 3, 4 / 3, 1 / 3])
    x, w = gauss_lobatto_legendre_rule(3)
    assert np.allclose(x, [-1, -1 / np.sqrt(5), 1 / np.sqrt(5), 1]) and np.allclose(w, [1 / 6, 5 / 6, 5 / 6, 1 / 6])
