"""Pins for the oracle's 1D rules and Lagrange basis (CPU only).

The 1D tables are the building block of Eq. (2) (B_abc,ijk = B1d_ai B1d_bj B1d_ck).  They are
pinned against closed forms, a library routine (numpy's Gauss-Legendre), exactness on monomials
and finite differences -- nothing here re-types the oracle's own formulas.
"""
import math

import numpy as np
import pytest

from oracle.quadrature import gauss_legendre, gauss_lobatto, lagrange, basis_1d


def test_gauss_legendre_matches_numpy_leggauss():
    for q in range(1, 13):
        x, w = gauss_legendre(q)
        xr, wr = np.polynomial.legendre.leggauss(q)
        np.testing.assert_allclose(x, (xr + 1) / 2, atol=2e-16, rtol=0)
        np.testing.assert_allclose(w, wr / 2, atol=1e-15, rtol=0)


def test_gauss_legendre_4pt_closed_form():
    x, w = gauss_legendre(4)
    s = math.sqrt(6.0 / 5.0)
    inner = math.sqrt(3.0 / 7.0 - 2.0 / 7.0 * s)
    outer = math.sqrt(3.0 / 7.0 + 2.0 / 7.0 * s)
    xe = np.array([1 - outer, 1 - inner, 1 + inner, 1 + outer]) / 2
    wi, wo = (18 + math.sqrt(30)) / 72, (18 - math.sqrt(30)) / 72
    np.testing.assert_allclose(x, xe, atol=1e-16, rtol=0)
    np.testing.assert_allclose(w, [wo, wi, wi, wo], atol=1e-16, rtol=0)


def test_gauss_lobatto_closed_forms():
    np.testing.assert_allclose(gauss_lobatto(2), [0, 1], atol=0)
    np.testing.assert_allclose(gauss_lobatto(3), [0, 0.5, 1], atol=1e-16)
    r5 = math.sqrt(5) / 10
    np.testing.assert_allclose(gauss_lobatto(4), [0, 0.5 - r5, 0.5 + r5, 1], atol=1e-16)
    r21 = math.sqrt(21) / 14
    np.testing.assert_allclose(gauss_lobatto(5), [0, 0.5 - r21, 0.5, 0.5 + r21, 1], atol=1e-16)


@pytest.mark.parametrize("q", range(1, 12))
def test_gauss_exact_to_degree_2q_minus_1(q):
    x, w = gauss_legendre(q)
    assert abs(w.sum() - 1.0) < 1e-15
    for k in range(2 * q):
        assert abs(np.sum(w * x ** k) - 1.0 / (k + 1)) < 1e-15 * (k + 1)
    # and not beyond: the first monomial past the degree is integrated with an error (it shrinks
    # fast with q, so look only where it is far above round-off)
    if q <= 8:
        assert abs(np.sum(w * x ** (2 * q)) - 1.0 / (2 * q + 1)) > 1e-12


@pytest.mark.parametrize("d", range(2, 11))
def test_gll_nodes_are_lobatto(d):
    """GLL with d points integrates degree 2d-3 exactly when weighted by the Lobatto weights
    w_i = 2 / (n (n+1) P_n(x_i)^2) (on [-1, 1]); check it through numpy's Legendre class."""
    t = gauss_lobatto(d)
    n = d - 1
    Pn = np.polynomial.legendre.Legendre.basis(n)
    x = 2 * t - 1
    w = 2.0 / (n * (n + 1) * Pn(x) ** 2) / 2
    for k in range(2 * d - 2):
        assert abs(np.sum(w * t ** k) - 1.0 / (k + 1)) < 2e-15 * (k + 1)
    # interior nodes are the roots of P_n'
    if n > 1:
        assert np.max(np.abs(Pn.deriv()(x[1:-1]))) < 1e-12


@pytest.mark.parametrize("p", range(1, 9))
def test_lagrange_properties(p):
    nodes = gauss_lobatto(p + 1)
    L, dL = lagrange(nodes, nodes)
    np.testing.assert_allclose(L, np.eye(p + 1), atol=1e-15)
    xs = np.linspace(-0.1, 1.1, 37)
    L, dL = lagrange(nodes, xs)
    np.testing.assert_allclose(L.sum(axis=1), 1.0, atol=1e-12)
    np.testing.assert_allclose(dL.sum(axis=1), 0.0, atol=1e-10)
    # exact interpolation of monomials up to degree p (values and derivatives)
    for k in range(p + 1):
        np.testing.assert_allclose(L @ nodes ** k, xs ** k, atol=1e-12)
        dk = k * xs ** (k - 1) if k > 0 else np.zeros_like(xs)
        np.testing.assert_allclose(dL @ nodes ** k, dk, atol=1e-10)
    # derivative against central differences
    h = 1e-6
    Lp, _ = lagrange(nodes, xs + h)
    Lm, _ = lagrange(nodes, xs - h)
    np.testing.assert_allclose(dL, (Lp - Lm) / (2 * h), atol=1e-6 * (p + 1) ** 3)


def test_basis_symmetry():
    """GLL nodes and GL points are symmetric about 1/2, so B1d[Q-1-q, D-1-d] = B1d[q, d] and
    G1d[Q-1-q, D-1-d] = -G1d[q, d]."""
    for p in range(1, 9):
        B, G, _, _, _ = basis_1d(p, p + 2)
        np.testing.assert_allclose(B[::-1, ::-1], B, atol=1e-14)
        np.testing.assert_allclose(G[::-1, ::-1], -G, atol=1e-12)
