"""Pins for the oracle's global operator, its rows and diagonal, and the brute-force agreement of
the element-matrix apply with the independent sum-factorised apply (CPU only)."""
import numpy as np
import pytest

from oracle import operator as op
from oracle import sumfact
from oracle.element import DIFFUSION, MASS
from oracle.mesh import boundary_mask, dof_map, ndofs
from paper_2603_09038_gb300.inputs import perturbed_vertices, uniform_vector, lognormal_coefficient


def _prob(n, p, seed=1234, coeff=True):
    V = perturbed_vertices(n, n, n, seed=seed)
    c = lognormal_coefficient(n ** 3, 1.0) if coeff else None
    return op.Problem(n, n, n, p, V, coeff=c)


@pytest.mark.parametrize("p", range(1, 9))
@pytest.mark.parametrize("kind", [DIFFUSION, MASS])
def test_brute_force_element_matrix_vs_sum_factorised(p, kind):
    """Eq. (2): sum factorisation only reorders exact arithmetic, so both routes agree to
    round-off on tiny meshes (1^3, 2^3, and 3^3 for p <= 4)."""
    for n in ([1, 2, 3] if p <= 4 else [1, 2]):
        prob = _prob(n, p)
        x = uniform_vector(prob.ndofs, seed=n)
        y1 = op.apply(prob, x, kind, batch=8)
        y2 = sumfact.apply(prob, x, kind)
        assert np.abs(y1 - y2).max() <= 1e-13 * np.abs(y1).max()


def test_apply_rows_match_full_apply():
    prob = _prob(3, 3)
    x = uniform_vector(prob.ndofs, seed=0)
    rows = np.random.default_rng(0).choice(prob.ndofs, 40, replace=False)
    rows = np.concatenate([rows, [0, prob.ndofs - 1]])
    for kind in (DIFFUSION, MASS):
        y = op.apply(prob, x, kind)
        np.testing.assert_allclose(op.apply_rows(prob, x, kind, rows), y[rows],
                                   atol=1e-14 * np.abs(y).max(), rtol=0)


def test_elements_of_dof_counts():
    """A dof has 1 (corner of the cube) to 8 (interior vertex) elements in its closure."""
    prob = _prob(3, 2)
    counts = np.zeros(prob.ndofs, dtype=int)
    for row in dof_map(3, 3, 3, 2):
        counts[row] += 1
    for g in range(prob.ndofs):
        els = op.elements_of_dof(prob, g)
        assert len(els) == counts[g]
        for e in els:
            assert g in dof_map(3, 3, 3, 2, [e])[0]


@pytest.mark.parametrize("kind", [DIFFUSION, MASS])
def test_diagonal_is_unit_vector_probe(kind):
    prob = _prob(2, 2)
    d = op.diagonal(prob, kind)
    for g in range(prob.ndofs):
        e = np.zeros(prob.ndofs)
        e[g] = 1.0
        assert abs(sumfact.apply(prob, e, kind)[g] - d[g]) < 1e-13 * np.abs(d).max()


def test_global_symmetry_null_space_and_assembly():
    prob = _prob(3, 3)
    x = uniform_vector(prob.ndofs, seed=1)
    y = uniform_vector(prob.ndofs, seed=2)
    for kind in (DIFFUSION, MASS):
        Ax, Ay = op.apply(prob, x, kind), op.apply(prob, y, kind)
        assert abs(y @ Ax - x @ Ay) < 1e-14 * np.abs(Ax).max() * np.abs(y).sum()
        A = op.assemble(prob, kind)
        np.testing.assert_allclose(A @ x, Ax, atol=1e-14 * np.abs(Ax).max(), rtol=0)
        assert abs(A - A.T).max() < 1e-14 * abs(A).max()
    A1 = op.apply(prob, np.ones(prob.ndofs), DIFFUSION)
    Anorm = abs(op.assemble(prob, DIFFUSION)).sum(axis=1).max()
    assert np.abs(A1).max() <= 1e-13 * Anorm


def test_boundary_mask_and_dof_count():
    for n, p in [(1, 1), (2, 3), (3, 2)]:
        m = boundary_mask(n, n, n, p)
        N = n * p + 1
        assert m.size == ndofs(n, n, n, p) == N ** 3
        assert m.sum() == N ** 3 - (N - 2) ** 3


def test_constrained_operator():
    prob = _prob(2, 2)
    m = boundary_mask(2, 2, 2, 2)
    Abc = op.constrained(lambda v: op.apply(prob, v, DIFFUSION), m)
    x = uniform_vector(prob.ndofs, seed=3)
    y = Abc(x)
    np.testing.assert_array_equal(y[m == 1], x[m == 1])
    xi = x * (1 - m)
    np.testing.assert_allclose(y[m == 0], op.apply(prob, xi, DIFFUSION)[m == 0])
