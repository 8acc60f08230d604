"""Jacobi-preconditioned CG, manufactured load vector and L2 error (oracle).

The paper has no solver section for this operator; these are the textbook algorithms:
preconditioned conjugate gradients (Hestenes-Stiefel, with a diagonal preconditioner), started
from zero, stopped when the recursive residual satisfies ||r||_2 <= rtol ||b||_2.
Manufactured problem: u = sin(pi x) sin(pi y) sin(pi z) on the unit cube, -div grad u = f with
f = 3 pi^2 u and u = 0 on the boundary.
"""
import numpy as np

from .element import reference_basis, geometry
from .mesh import element_vertices, trilinear, dof_map


def pcg(A, b, diag, rtol=1e-10, maxit=10000):
    """Solve A x = b; A is a callable, ``diag`` the Jacobi preconditioner (M = diag).
    Returns (x, iterations, history of ||r||/||b||)."""
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b)
    r = b.copy()
    nb = np.sqrt(b @ b)
    if nb == 0.0:
        return x, 0, [0.0]
    z = r / diag
    p = z.copy()
    rz = r @ z
    hist = [1.0]
    for it in range(1, maxit + 1):
        q = A(p)
        pq = p @ q
        if not pq > 0.0:
            raise ArithmeticError("CG breakdown: p.Ap <= 0")
        alpha = rz / pq
        x += alpha * p
        r -= alpha * q
        rel = np.sqrt(r @ r) / nb
        hist.append(rel)
        if rel <= rtol:
            return x, it, hist
        z = r / diag
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, maxit, hist


def u_exact(X):
    return np.sin(np.pi * X[..., 0]) * np.sin(np.pi * X[..., 1]) * np.sin(np.pi * X[..., 2])


def f_sine(X):
    return 3.0 * np.pi ** 2 * u_exact(X)


def load_vector(prob, f=f_sine, q1d=None, batch=1024):
    """b_a = sum_e sum_q w_q |det J| f(x(xi_q)) phi_a(xi_q), with the Q-point Gauss rule
    (Q = the operator's rule unless given)."""
    Q = q1d or prob.q1d
    phi, _, w, xi = reference_basis(prob.p, Q)
    b = np.zeros(prob.ndofs)
    for s in range(0, prob.ne, batch):
        el = np.arange(s, min(prob.ne, s + batch))
        Xe = element_vertices(prob.vertices, prob.nx, prob.ny, prob.nz, el)
        X, _ = trilinear(Xe, xi)
        _, detJ = geometry(prob.vertices, prob.nx, prob.ny, prob.nz, Q, el)
        be = np.einsum('eq,qa->ea', w[None, :] * detJ * f(X), phi)
        np.add.at(b, dof_map(prob.nx, prob.ny, prob.nz, prob.p, el), be)
    return b


def l2_error(prob, uh, u=u_exact, q1d=None, batch=1024):
    """||u_h - u||_{L2} with a Q = p + 4 Gauss rule per element (a higher rule than the
    operator's, so that the error is not polluted by quadrature)."""
    Q = q1d or prob.p + 4
    phi, _, w, xi = reference_basis(prob.p, Q)
    uh = np.asarray(uh, dtype=np.float64)
    acc = 0.0
    for s in range(0, prob.ne, batch):
        el = np.arange(s, min(prob.ne, s + batch))
        Xe = element_vertices(prob.vertices, prob.nx, prob.ny, prob.nz, el)
        X, _ = trilinear(Xe, xi)
        _, detJ = geometry(prob.vertices, prob.nx, prob.ny, prob.nz, Q, el)
        uq = uh[dof_map(prob.nx, prob.ny, prob.nz, prob.p, el)] @ phi.T      # [e, nq]
        acc += np.sum(w[None, :] * detJ * (uq - u(X)) ** 2)
    return np.sqrt(acc)
