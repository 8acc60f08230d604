"""Pins for the oracle's mixed gradient / divergence pair (H1 order 4 -> L2 order 3 vector), CPU
only: constants in the kernel, the divergence theorem for linear pressures, adjointness, closed-form
integrals on an affine mesh, and the element matrix on the unit cube against 1D matrices built by
exact polynomial integration."""
import numpy as np
import pytest

from oracle.mesh import dof_coordinates
from oracle.mixed import MixedProblem, element_gradient_matrices, l2_nodes
from oracle.quadrature import gauss_lobatto
from paper_2603_09038_gb300.inputs import perturbed_vertices, uniform_vector


def _lattice(nx, ny, nz):
    zs, ys, xs = np.meshgrid(np.arange(nz + 1.0), np.arange(ny + 1.0), np.arange(nx + 1.0),
                             indexing="ij")
    return np.stack([xs.reshape(-1), ys.reshape(-1), zs.reshape(-1)], axis=1)


def test_constants_have_no_gradient():
    M = MixedProblem(3, 2, 2, perturbed_vertices(3, 2, 2, seed=4))
    g = M.gradient(np.ones(M.ndof_h))
    assert np.abs(g).max() < 1e-14


def test_linear_pressure_integrates_to_the_volume():
    """sum_a psi_a = 1, so summing G p over an element's L2 nodes gives int_e grad p; for
    p = alpha . x on the perturbed unit cube that is alpha times the volume, 1 in total."""
    n = 3
    V = perturbed_vertices(n, n, n, seed=9)
    M = MixedProblem(n, n, n, V)
    X = dof_coordinates(V, n, n, n, M.p_h)
    alpha = np.array([0.7, -1.3, 2.1])
    g = M.gradient(X @ alpha).reshape(M.ne, 3, -1)
    np.testing.assert_allclose(g.sum(axis=(0, 2)), alpha, rtol=0, atol=1e-13)


def test_divergence_is_the_transpose():
    M = MixedProblem(2, 3, 2, perturbed_vertices(2, 3, 2, seed=1))
    p = uniform_vector(M.ndof_h, seed=3)
    u = uniform_vector(M.ndof_l, seed=4)
    lhs, rhs = u @ M.gradient(p), p @ M.divergence(u)
    assert abs(lhs - rhs) <= 1e-13 * (np.abs(u).sum() + np.abs(p).sum())


def test_affine_closed_forms():
    """Unit-spacing lattice [0,3] x [0,2] x [0,2], p = x y^2 (in the order-4 space), u an
    interpolant of a linear field (exact in the order-3 space):
    int (d_x p) z = nx ny^3 nz^2 / 6, int (d_y p) x = 2 (nx^3/3)(ny^2/2) nz."""
    nx, ny, nz = 3, 2, 2
    V = _lattice(nx, ny, nz)
    M = MixedProblem(nx, ny, nz, V)
    X = dof_coordinates(V, nx, ny, nz, M.p_h)
    p = X[:, 0] * X[:, 1] ** 2
    g = M.gradient(p).reshape(M.ne, 3, -1)
    Y = M.l2_node_coords()                                   # [ne, D_l^3, 3]
    assert abs((g[:, 0, :] * Y[..., 2]).sum() - nx * ny ** 3 * nz ** 2 / 6.0) < 1e-11
    assert abs((g[:, 1, :] * Y[..., 0]).sum() - 2 * (nx ** 3 / 3) * (ny ** 2 / 2) * nz) < 1e-11
    assert abs((g[:, 2, :]).sum()) < 1e-12                  # d_z p = 0


def _lagrange_polys(nodes):
    out = []
    for d, t in enumerate(nodes):
        others = np.delete(nodes, d)
        out.append(np.poly1d(np.poly(others) / np.prod(t - others)))
    return out


@pytest.mark.parametrize("p_h,p_l", [(4, 3), (2, 1), (3, 3)])
def test_unit_cube_element_matrix_by_exact_1d_integrals(p_h, p_l):
    """On [0,1]^3 (J = I) the element matrix is a Kronecker product of 1D matrices,
    X[a, b] = int_0^1 l_b' psi_a, B[a, b] = int_0^1 l_b psi_a, integrated here exactly as
    polynomials (no quadrature): G_x = B (x) B (x) X, etc. (z slowest)."""
    V = _lattice(1, 1, 1)
    Ge = element_gradient_matrices(V, 1, 1, 1, p_h, p_l)[0]  # [3, Dl^3, Dh^3]
    lh = _lagrange_polys(gauss_lobatto(p_h + 1))
    ll = _lagrange_polys(l2_nodes(p_l))

    def integral(poly):
        P = np.polyint(poly)
        return P(1.0) - P(0.0)

    B1 = np.array([[integral(lb * la) for lb in lh] for la in ll])
    X1 = np.array([[integral(np.polyder(lb) * la) for lb in lh] for la in ll])
    ref = [np.kron(np.kron(B1, B1), X1), np.kron(np.kron(B1, X1), B1), np.kron(np.kron(X1, B1), B1)]
    for c in range(3):
        np.testing.assert_allclose(Ge[c], ref[c], rtol=0, atol=1e-13)
