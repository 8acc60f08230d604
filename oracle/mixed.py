"""The paper's own operator: the off-diagonal blocks of the acoustic-gravity system (oracle; TEST
INFRASTRUCTURE, never imported by the library).

Section II-A, Eq. (block-mult): the stiffness operator couples an H1 pressure p and an L2 vector
velocity u through (grad p, tau) and -(u, grad v).  Section III-G's kernels apply these blocks
with distinct trial and test bases.  The paper fixes the spaces (order-4 continuous pressure,
order-3 discontinuous velocity components) but not their nodes, quadrature or mapping.  Readings:

* H1: order p_h (4) on the Gauss-Lobatto-Legendre nodes, the structured mesh's lexicographic
  global numbering (the same dof map as the H1 diffusion operator);
* L2: order p_l (3), one Lagrange basis per element on the p_l + 1 Gauss-Legendre points per
  axis, three components, no continuity; global layout [ne][3][D_l^3] (element-major, then
  component, then a = i + D_l*(j + D_l*k));
* quadrature: Q = p_h + 1 Gauss-Legendre points per axis (the shapes of Section III-C's
  m25n5k4 tiles: Q^2 = 25, D_h = 5, D_l = 4);
* the L2 basis is used as is on the physical element (a "value" map; no 1/det J scaling).

Then (G p)_{e,c,a} = sum_q w_q det J_e(x_q) (J_e^{-T} grad phi_b(x_q))_c psi_a(x_q) p_{g(e,b)}:
the gradient block, an [ne*3*D_l^3, ndof_h] matrix, and the divergence block is its transpose
(the system's -(u, grad v) is -G^T).  Both are computed element by element from dense element
matrices by direct quadrature (no sum factorisation).
"""
import numpy as np

from .element import geometry
from .mesh import dof_map, ndofs
from .quadrature import gauss_legendre, gauss_lobatto, lagrange


def l2_nodes(p_l):
    """The p_l + 1 Gauss-Legendre points on [0, 1] (the L2 basis nodes)."""
    return gauss_legendre(p_l + 1)[0]


def element_gradient_matrices(vertices, nx, ny, nz, p_h=4, p_l=3, q1d=None, elems=None):
    """Dense [ne, 3, D_l^3, D_h^3] element matrices of the gradient block."""
    Q = p_h + 1 if q1d is None else q1d
    pts, wts = gauss_legendre(Q)
    Dh, Dl = p_h + 1, p_l + 1
    Lh, dLh = lagrange(gauss_lobatto(Dh), pts)             # [Q, Dh]
    Ll, _ = lagrange(l2_nodes(p_l), pts)                    # [Q, Dl]
    q = np.arange(Q ** 3)
    qx, qy, qz = q % Q, (q // Q) % Q, q // (Q * Q)
    b = np.arange(Dh ** 3)
    bi, bj, bk = b % Dh, (b // Dh) % Dh, b // (Dh * Dh)
    a = np.arange(Dl ** 3)
    ai, aj, ak = a % Dl, (a // Dl) % Dl, a // (Dl * Dl)
    # reference gradients of the H1 basis [nq, Dh^3, 3] and the L2 basis [nq, Dl^3]
    grad = np.stack([dLh[qx][:, bi] * Lh[qy][:, bj] * Lh[qz][:, bk],
                     Lh[qx][:, bi] * dLh[qy][:, bj] * Lh[qz][:, bk],
                     Lh[qx][:, bi] * Lh[qy][:, bj] * dLh[qz][:, bk]], axis=2)
    psi = Ll[qx][:, ai] * Ll[qy][:, aj] * Ll[qz][:, ak]
    w = wts[qx] * wts[qy] * wts[qz]
    # geometry at the same Q-point rule
    J, detJ = geometry(vertices, nx, ny, nz, Q, elems)      # [ne, nq, 3, 3], [ne, nq]
    Jinv = np.linalg.inv(J)
    gphys = np.einsum('eqrs,qbr->eqbs', Jinv, grad, optimize=True)   # (J^{-T} g)_s
    scale = w[None, :] * detJ                                        # [ne, nq]
    return np.einsum('eq,eqbc,qa->ecab', scale, gphys, psi, optimize=True)


class MixedProblem:
    """The gradient / divergence pair on an nx x ny x nz structured mesh."""

    def __init__(self, nx, ny, nz, vertices, p_h=4, p_l=3):
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.vertices = np.asarray(vertices, dtype=np.float64).reshape(-1, 3)
        self.p_h, self.p_l = int(p_h), int(p_l)
        self.ne = self.nx * self.ny * self.nz
        self.ndof_h = ndofs(self.nx, self.ny, self.nz, self.p_h)
        self.nl = 3 * (self.p_l + 1) ** 3          # L2 values per element
        self.ndof_l = self.ne * self.nl

    def elem_mats(self, elems=None):
        return element_gradient_matrices(self.vertices, self.nx, self.ny, self.nz, self.p_h,
                                         self.p_l, elems=elems)

    def gradient(self, p):
        """u = G p: [ndof_l] from an H1 vector [ndof_h]."""
        p = np.asarray(p, dtype=np.float64)
        Ge = self.elem_mats()
        gm = dof_map(self.nx, self.ny, self.nz, self.p_h)
        return np.einsum('ecab,eb->eca', Ge, p[gm]).reshape(-1)

    def divergence(self, u):
        """v = G^T u: [ndof_h] from an L2 vector [ndof_l] (scatter-add over elements, in
        element order)."""
        u = np.asarray(u, dtype=np.float64).reshape(self.ne, 3, -1)
        Ge = self.elem_mats()
        gm = dof_map(self.nx, self.ny, self.nz, self.p_h)
        v = np.zeros(self.ndof_h)
        np.add.at(v, gm, np.einsum('ecab,eca->eb', Ge, u))
        return v

    def l2_node_coords(self):
        """Physical coordinates [ne, D_l^3, 3] of the L2 nodes (trilinear images)."""
        from .mesh import element_vertices, trilinear
        t = l2_nodes(self.p_l)
        Dl = self.p_l + 1
        a = np.arange(Dl ** 3)
        xi = np.stack([t[a % Dl], t[(a // Dl) % Dl], t[a // (Dl * Dl)]], axis=1)
        X, _ = trilinear(element_vertices(self.vertices, self.nx, self.ny, self.nz), xi)
        return X
