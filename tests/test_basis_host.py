"""The library's 1D tables (Eq. (2)'s B1d and its derivative, the GLL nodes and the Gauss rule),
read through the host-only C-ABI entry fe_basis_1d, against closed forms and the oracle (CPU)."""
import math

import numpy as np
import pytest

from oracle.quadrature import basis_1d as oracle_basis_1d


def _lib():
    from tests.gpu_util import lib
    return lib()


def test_closed_forms():
    fe = _lib()
    _, pts, wts, _, _ = fe.fe_basis_1d(2, 4)
    a, b = math.sqrt(3 / 7 - 2 / 7 * math.sqrt(6 / 5)), math.sqrt(3 / 7 + 2 / 7 * math.sqrt(6 / 5))
    np.testing.assert_allclose(pts, sorted([0.5 * (1 - b), 0.5 * (1 - a), 0.5 * (1 + a),
                                            0.5 * (1 + b)]), rtol=0, atol=1e-15)
    wa, wb = (18 + math.sqrt(30)) / 72, (18 - math.sqrt(30)) / 72
    np.testing.assert_allclose(wts, [wb, wa, wa, wb], rtol=0, atol=1e-15)
    gll = {2: [0, 0.5, 1], 3: [0, 0.5 - math.sqrt(5) / 10, 0.5 + math.sqrt(5) / 10, 1],
           4: [0, 0.5 - math.sqrt(21) / 14, 0.5, 0.5 + math.sqrt(21) / 14, 1]}
    for p, ref in gll.items():
        nodes = fe.fe_basis_1d(p, p + 2)[0]
        np.testing.assert_allclose(nodes, ref, rtol=0, atol=1e-15)


@pytest.mark.parametrize("p", range(1, 9))
def test_rule_exactness_and_basis_identities(p):
    fe = _lib()
    q = p + 2
    nodes, pts, wts, B, G = fe.fe_basis_1d(p, q)
    for k in range(2 * q):
        assert abs(wts @ pts ** k - 1.0 / (k + 1)) <= 2e-15
    np.testing.assert_allclose(B.sum(axis=1), 1.0, rtol=0, atol=1e-13)     # partition of unity
    np.testing.assert_allclose(G.sum(axis=1), 0.0, rtol=0, atol=1e-11)
    # l_d reproduces the monomials up to degree p; l_d' their derivatives
    for k in range(p + 1):
        np.testing.assert_allclose(B @ nodes ** k, pts ** k, rtol=0, atol=1e-13)
        np.testing.assert_allclose(G @ nodes ** k, k * pts ** max(k - 1, 0) if k else 0 * pts,
                                   rtol=0, atol=1e-11)


@pytest.mark.parametrize("p", range(1, 9))
def test_matches_oracle_tables(p):
    fe = _lib()
    q = p + 2
    nodes, pts, wts, B, G = fe.fe_basis_1d(p, q)
    Bo, Go, po, wo, no = oracle_basis_1d(p, q)
    for got, ref, tol in ((nodes, no, 1e-15), (pts, po, 1e-15), (wts, wo, 1e-15), (B, Bo, 1e-14),
                          (G, Go, 1e-12)):
        np.testing.assert_allclose(got, ref, rtol=0, atol=tol)


@pytest.mark.parametrize("p", range(1, 9))
def test_reversal_symmetry_of_the_tables(p):
    """The even-odd FP64 contractions rely on B[Q-1-q][D-1-d] = B[q][d] and
    G[Q-1-q][D-1-d] = -G[q][d] (nodes and points symmetric about 1/2); the same holds for the
    oracle's tables, built independently."""
    fe = _lib()
    q = p + 2
    nodes, pts, wts, B, G = fe.fe_basis_1d(p, q)
    np.testing.assert_allclose(nodes[::-1], 1.0 - nodes, rtol=0, atol=1e-15)
    np.testing.assert_allclose(pts[::-1], 1.0 - pts, rtol=0, atol=1e-15)
    for Bt, Gt in ((B, G), oracle_basis_1d(p, q)[:2]):
        assert np.abs(Bt[::-1, ::-1] - Bt).max() <= 1e-14
        assert np.abs(Gt[::-1, ::-1] + Gt).max() <= 1e-12 * np.abs(Gt).max()


@pytest.mark.parametrize("order,q1d", [(0, 2), (9, 11), (3, 0), (3, 11)])
def test_bad_arguments(order, q1d):
    fe = _lib()
    with pytest.raises(fe.FEError) as e:
        fe.fe_basis_1d(order, q1d)
    assert e.value.status == fe.FE_ERR_ARG
