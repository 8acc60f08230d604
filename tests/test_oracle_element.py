"""Pins for the oracle's element matrices (CPU only).

Each check fixes the element matrices of the standard Galerkin forms (the H1 reading of
Eq. (1)'s D and B) by something other than the oracle's own code: textbook closed forms,
a surface-integral volume, exact integrals of polynomials, affine and rigid-motion invariants.
``test_planted_*`` plant a plausible mistake in a copy of the oracle and show that a pin fails.
"""
import os

import numpy as np
import pytest

from oracle.element import element_matrices, reference_basis, geometry, DIFFUSION, MASS
from oracle.mesh import element_vertices, dof_coordinates, trilinear
from oracle.operator import Problem, apply
from paper_2603_09038_gb300.inputs import perturbed_vertices, lognormal_coefficient

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_1d():
    rows = {"M30": [], "K3": []}
    for line in open(os.path.join(GOLDEN, "p2_1d_element_matrices.txt")):
        if line.startswith("#") or not line.strip():
            continue
        tag, *vals = line.split()
        rows[tag].append([float(v) for v in vals])
    return np.array(rows["M30"]), np.array(rows["K3"])


def test_golden_1d_matrices_rederived():
    sp = pytest.importorskip("sympy")
    t, h = sp.symbols("t h", positive=True)
    ls = [(1 - 2 * t) * (1 - t), 4 * t * (1 - t), t * (2 * t - 1)]
    M = sp.Matrix(3, 3, lambda a, b: sp.integrate(ls[a] * ls[b] * h, (t, 0, 1)))
    K = sp.Matrix(3, 3, lambda a, b: sp.integrate(sp.diff(ls[a], t) * sp.diff(ls[b], t) / h, (t, 0, 1)))
    M30, K3 = _golden_1d()
    M30 = sp.Matrix(M30.astype(int).tolist())
    K3 = sp.Matrix(K3.astype(int).tolist())
    assert sp.simplify(M - M30 * h / 30) == sp.zeros(3, 3)
    assert sp.simplify(K - K3 / (3 * h)) == sp.zeros(3, 3)


@pytest.mark.parametrize("n", [1, 2, 3])
def test_p2_cube_element_matrices_are_kronecker_of_textbook_1d(n):
    M30, K3 = _golden_1d()
    h = 1.0 / n
    M1, K1 = M30 * h / 30.0, K3 / (3.0 * h)
    V = perturbed_vertices(n, n, n, amp=0.0)
    # local index a = i + 3 j + 9 k (x fastest)  <->  kron(z, kron(y, x))
    Mref = np.kron(M1, np.kron(M1, M1))
    Kref = np.kron(M1, np.kron(M1, K1)) + np.kron(M1, np.kron(K1, M1)) + np.kron(K1, np.kron(M1, M1))
    Ke = element_matrices(V, n, n, n, 2, 4, None, DIFFUSION)
    Me = element_matrices(V, n, n, n, 2, 4, None, MASS)
    for e in range(n ** 3):
        np.testing.assert_allclose(Me[e], Mref, atol=1e-15 * h ** 3, rtol=0)
        np.testing.assert_allclose(Ke[e], Kref, atol=2e-14 / h, rtol=0)


def _volume_by_divergence(Xe):
    """vol = (1/3) sum over the six bilinear faces of the flux of x through the face, each face
    integral by a 2x2 Gauss rule (exact: the integrand is bilinear in each face variable)."""
    g = np.array([0.5 - 0.5 / np.sqrt(3), 0.5 + 0.5 / np.sqrt(3)])
    vol = 0.0
    for axis in range(3):
        for side in (0, 1):
            for s in g:
                for t in g:
                    xi = np.empty(3)
                    xi[axis] = side
                    others = [a for a in range(3) if a != axis]
                    xi[others[0]], xi[others[1]] = s, t
                    x, J = trilinear(Xe[None], xi[None])
                    x, J = x[0, 0], J[0, 0]
                    # area normal dx/ds x dx/dt, oriented outward for a right-handed map
                    nrm = np.cross(J[:, others[0]], J[:, others[1]])
                    sign = (1 if side == 1 else -1) * (1 if axis != 1 else -1)
                    vol += 0.25 * sign * x @ nrm / 3.0
    return vol


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_mass_volume_per_element_and_total(p):
    n = 3
    V = perturbed_vertices(n, n, n, seed=7)
    Me = element_matrices(V, n, n, n, p, p + 2, None, MASS)
    EV = element_vertices(V, n, n, n)
    vols = np.array([_volume_by_divergence(EV[e]) for e in range(n ** 3)])
    np.testing.assert_allclose(Me.sum(axis=(1, 2)), vols, rtol=1e-13)
    assert abs(vols.sum() - 1.0) < 1e-14
    c = lognormal_coefficient(n ** 3, 1.0, seed=3)
    prob = Problem(n, n, n, p, V, coeff=c)
    one = np.ones(prob.ndofs)
    assert abs(one @ apply(prob, one, MASS) - c @ vols) < 1e-13 * (c @ vols)


@pytest.mark.parametrize("p", [1, 2, 3, 5, 8])
def test_diffusion_null_space_symmetry_definiteness(p):
    n = 2
    V = perturbed_vertices(n, n, n, seed=11)
    c = lognormal_coefficient(n ** 3, 1.0)
    Ke = element_matrices(V, n, n, n, p, p + 2, c, DIFFUSION)
    Me = element_matrices(V, n, n, n, p, p + 2, c, MASS)
    for e in range(n ** 3):
        scale = np.abs(Ke[e]).max()
        assert np.abs(Ke[e].sum(axis=1)).max() < 1e-13 * scale * (p + 1) ** 3
        np.testing.assert_allclose(Ke[e], Ke[e].T, atol=1e-14 * scale)
        np.testing.assert_allclose(Me[e], Me[e].T, atol=1e-15 * np.abs(Me[e]).max())
        ev = np.linalg.eigvalsh(Ke[e])
        assert ev[0] > -1e-12 * ev[-1] and ev[1] > 1e-8 * ev[-1]      # one-dimensional kernel
        assert np.linalg.eigvalsh(Me[e])[0] > 0


@pytest.mark.parametrize("p", [1, 2, 3, 4, 6])
def test_mass_quadrature_is_exact_at_q_p_plus_2(p):
    """phi_a phi_b det J has degree <= 2p+2 per axis on a trilinear element, and Q = p+2 Gauss
    points integrate degree 2p+3: a higher rule must give the same matrix."""
    n = 2
    V = perturbed_vertices(n, n, n, seed=5)
    A = element_matrices(V, n, n, n, p, p + 2, None, MASS)
    B = element_matrices(V, n, n, n, p, p + 5, None, MASS)
    np.testing.assert_allclose(A, B, atol=1e-14 * np.abs(B).max(), rtol=0)
    # and a too-low rule does not (the check has teeth)
    C = element_matrices(V, n, n, n, p, p, None, MASS)
    assert np.abs(C - B).max() > 1e-10 * np.abs(B).max()


def test_polynomial_integrals_on_unit_cube():
    """u = x^2 y and v = x z + 1 lie in Q_2; on an undistorted mesh, v^T M u = int u v = 11/48
    and v^T K u = int grad u . grad v = int 2 x y z = 1/4."""
    for n in (1, 2, 3):
        V = perturbed_vertices(n, n, n, amp=0.0)
        prob = Problem(n, n, n, 2, V)
        X = dof_coordinates(V, n, n, n, 2)
        u = X[:, 0] ** 2 * X[:, 1]
        v = X[:, 0] * X[:, 2] + 1.0
        assert abs(v @ apply(prob, u, MASS) - 11.0 / 48.0) < 1e-15
        assert abs(v @ apply(prob, u, DIFFUSION) - 0.25) < 1e-13


def test_affine_mesh_linear_functions():
    """On an affine image x' = A x + b of the cube mesh, for linear u = g.x', v = k.x':
    v^T K u = (g . k) |det A| and 1^T M 1 = |det A| (pins the J^{-T} transforms)."""
    rng = np.random.default_rng(0)
    A = np.eye(3) + 0.3 * rng.standard_normal((3, 3))
    b = rng.standard_normal(3)
    g, k = rng.standard_normal(3), rng.standard_normal(3)
    n = 2
    V = perturbed_vertices(n, n, n, amp=0.0) @ A.T + b
    for p in (1, 2, 3):
        prob = Problem(n, n, n, p, V)
        X = dof_coordinates(V, n, n, n, p)
        u, v = X @ g, X @ k
        detA = abs(np.linalg.det(A))
        assert abs(v @ apply(prob, u, DIFFUSION) - (g @ k) * detA) < 1e-13 * max(1, abs(g @ k) * detA)
        one = np.ones(prob.ndofs)
        assert abs(one @ apply(prob, one, MASS) - detA) < 1e-14


def test_rigid_motion_and_scaling_invariance():
    """Rotating and translating a mesh leaves K and M unchanged; scaling by s multiplies K by s
    and M by s^3 (three dimensions)."""
    n, p = 2, 3
    V = perturbed_vertices(n, n, n, seed=9)
    rng = np.random.default_rng(1)
    R, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    if np.linalg.det(R) < 0:
        R[:, 0] *= -1
    K0 = element_matrices(V, n, n, n, p, p + 2, None, DIFFUSION)
    M0 = element_matrices(V, n, n, n, p, p + 2, None, MASS)
    Vr = V @ R.T + np.array([0.3, -2.0, 1.5])
    np.testing.assert_allclose(element_matrices(Vr, n, n, n, p, p + 2, None, DIFFUSION), K0,
                               atol=1e-13 * np.abs(K0).max())
    np.testing.assert_allclose(element_matrices(Vr, n, n, n, p, p + 2, None, MASS), M0,
                               atol=1e-15 * np.abs(M0).max())
    s = 2.5
    np.testing.assert_allclose(element_matrices(s * V, n, n, n, p, p + 2, None, DIFFUSION), s * K0,
                               atol=1e-13 * s * np.abs(K0).max())
    np.testing.assert_allclose(element_matrices(s * V, n, n, n, p, p + 2, None, MASS), s ** 3 * M0,
                               atol=1e-15 * s ** 3 * np.abs(M0).max())


def test_inverted_element_is_rejected():
    V = perturbed_vertices(1, 1, 1, amp=0.0)
    V[[0, 1]] = V[[1, 0]]          # swap two corners: the map folds over
    with pytest.raises(ValueError):
        geometry(V, 1, 1, 1, 4)


# ----- planted mistakes: each copy of the oracle below is wrong in one plausible way, and one
# ----- of the pins above catches it (so the pins would catch the same slip in the oracle).

def _mats_planted(V, n, p, q1d, kind, mistake):
    phi, grad, w, _ = reference_basis(p, q1d)
    J, detJ = geometry(V, n, n, n, q1d)
    if mistake == "no_detJ":
        detJ = np.ones_like(detJ)
    scale = w[None, :] * detJ
    if kind == MASS:
        return np.einsum('eq,qa,qb->eab', scale, phi, phi)
    Jinv = np.linalg.inv(J)
    if mistake == "transposed_inverse":
        Jinv = np.swapaxes(Jinv, -1, -2)
    if mistake == "swapped_gradient":
        grad = grad[:, :, [1, 0, 2]]
    gphys = np.einsum('eqrs,qar->eqas', Jinv, grad)
    return np.einsum('eq,eqas,eqbs->eab', scale, gphys, gphys)


def test_planted_missing_detJ_fails_volume_pin():
    n, p = 2, 2
    V = perturbed_vertices(n, n, n, amp=0.0) * 0.5
    M = _mats_planted(V, n, p, p + 2, MASS, "no_detJ")
    assert abs(M.sum() - 0.125) > 1e-3          # true volume of the half-size cube is 1/8


def test_planted_transposed_inverse_fails_affine_pin():
    rng = np.random.default_rng(0)
    A = np.eye(3) + 0.3 * rng.standard_normal((3, 3))
    n, p = 1, 1
    V = perturbed_vertices(n, n, n, amp=0.0) @ A.T
    g, k = rng.standard_normal(3), rng.standard_normal(3)
    X = dof_coordinates(V, n, n, n, p)
    Kbad = _mats_planted(V, n, p, p + 2, DIFFUSION, "transposed_inverse")[0]
    Kgood = element_matrices(V, n, n, n, p, p + 2, None, DIFFUSION)[0]
    exact = (g @ k) * abs(np.linalg.det(A))
    assert abs((X @ k) @ Kgood @ (X @ g) - exact) < 1e-13
    assert abs((X @ k) @ Kbad @ (X @ g) - exact) > 1e-3


def test_planted_swapped_gradient_fails_affine_pin():
    """Swapping two reference-gradient components is invisible on an isotropic cube (the dot
    product is symmetric), but not on a general affine element."""
    rng = np.random.default_rng(2)
    A = np.eye(3) + 0.3 * rng.standard_normal((3, 3))
    n, p = 1, 2
    V = perturbed_vertices(n, n, n, amp=0.0) @ A.T
    X = dof_coordinates(V, n, n, n, p)
    g, k = rng.standard_normal(3), rng.standard_normal(3)
    Kbad = _mats_planted(V, n, p, p + 2, DIFFUSION, "swapped_gradient")[0]
    exact = (g @ k) * abs(np.linalg.det(A))
    assert abs((X @ k) @ Kbad @ (X @ g) - exact) > 1e-3
