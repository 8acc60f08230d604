"""Element matrices by direct quadrature -- no sum factorisation (oracle; test infrastructure).

Every basis function is evaluated at every quadrature point as the plain product
``phi_a(xi) = l_i(xi_1) l_j(xi_2) l_k(xi_3)`` (Eq. (2)'s B_abc,ijk written out), and the
element matrices are the standard Galerkin sums (the paper states only the generic
decomposition of Eq. (1); the H1 forms are the textbook ones):

    diffusion  K_e[a, b] = sum_q w_q c_e det J (J^{-T} grad phi_a) . (J^{-T} grad phi_b)
    mass       M_e[a, b] = sum_q w_q c_e det J  phi_a phi_b

Cost O(ne * Q^3 * D^6): for small meshes, or for a handful of elements of a large one.
"""
import numpy as np

from .quadrature import basis_1d
from .mesh import element_vertices, trilinear

DIFFUSION = "diffusion"
MASS = "mass"


def reference_basis(p, q1d):
    """Tensor-product basis at the Q^3 Gauss points (q = qx + Q*(qy + Q*qz)).

    Returns (phi [nq, D^3], grad [nq, D^3, 3] reference gradients, w [nq], xi [nq, 3]).
    """
    B, G, pts, wts, _ = basis_1d(p, q1d)
    D, Q = p + 1, q1d
    q = np.arange(Q ** 3)
    qx, qy, qz = q % Q, (q // Q) % Q, q // (Q * Q)
    a = np.arange(D ** 3)
    i, j, k = a % D, (a // D) % D, a // (D * D)
    Bx, By, Bz = B[qx][:, i], B[qy][:, j], B[qz][:, k]
    Gx, Gy, Gz = G[qx][:, i], G[qy][:, j], G[qz][:, k]
    phi = Bx * By * Bz
    grad = np.stack([Gx * By * Bz, Bx * Gy * Bz, Bx * By * Gz], axis=2)
    w = wts[qx] * wts[qy] * wts[qz]
    xi = np.stack([pts[qx], pts[qy], pts[qz]], axis=1)
    return phi, grad, w, xi


def geometry(vertices, nx, ny, nz, q1d, elems=None):
    """Jacobians J [ne, nq, 3, 3] and det J [ne, nq] of the (listed) elements at the Gauss
    points; raises if any det J <= 0 (inverted or degenerate element)."""
    _, _, _, xi = reference_basis(1, q1d)
    Xe = element_vertices(vertices, nx, ny, nz, elems)
    _, J = trilinear(Xe, xi)
    detJ = np.linalg.det(J)
    if np.any(detJ <= 0.0):
        raise ValueError("mesh has an element with det J <= 0")
    return J, detJ


def element_matrices(vertices, nx, ny, nz, p, q1d, coeff, kind, elems=None):
    """Dense element matrices [ne, D^3, D^3] of the listed elements (all by default)."""
    phi, grad, w, _ = reference_basis(p, q1d)
    J, detJ = geometry(vertices, nx, ny, nz, q1d, elems)
    ne = J.shape[0]
    if coeff is None:
        c = np.ones(ne)
    else:
        c = np.asarray(coeff, dtype=np.float64)
        c = c if elems is None else c[np.asarray(elems)]
    scale = w[None, :] * c[:, None] * detJ                          # [ne, nq]
    if kind == MASS:
        return np.einsum('eq,qa,qb->eab', scale, phi, phi, optimize=True)
    if kind != DIFFUSION:
        raise ValueError(kind)
    Jinv = np.linalg.inv(J)                                         # [ne, nq, 3, 3]
    # physical gradient: (J^{-T} g)_s = sum_r Jinv[r, s] g_r
    gphys = np.einsum('eqrs,qar->eqas', Jinv, grad, optimize=True)  # [ne, nq, D^3, 3]
    return np.einsum('eq,eqas,eqbs->eab', scale, gphys, gphys, optimize=True)
