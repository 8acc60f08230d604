"""Jacobi- and Chebyshev-preconditioned CG, manufactured load vector and L2 error (oracle).

The paper has no solver section for this operator; these are the textbook algorithms:
preconditioned conjugate gradients (Hestenes-Stiefel, with a diagonal or a Chebyshev polynomial
preconditioner), started from zero, stopped when the recursive residual satisfies
||r||_2 <= rtol ||b||_2.
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


def pcg_prec(A, b, M, rtol=1e-10, maxit=10000):
    """The same preconditioned CG with a general (linear, SPD) preconditioner z = M(r)."""
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b)
    r = b.copy()
    nb = np.sqrt(b @ b)
    if nb == 0.0:
        return x, 0, [0.0]
    z = M(r)
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
        z = M(r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, maxit, hist


def chebyshev(A, dinv, r, k, lo, hi):
    """Chebyshev polynomial preconditioner: k steps of the Chebyshev semi-iteration for
    D^-1 A z = D^-1 r from z = 0 with the spectrum assumed in [lo, hi] (k - 1 products with A).
    The result is z = q(D^-1 A) D^-1 r with the residual polynomial
        1 - lam q(lam) = T_k((theta - lam) / delta) / T_k(theta / delta),
    theta = (hi + lo) / 2, delta = (hi - lo) / 2, T_k the Chebyshev polynomial of the first
    kind; the textbook three-term recurrence in the directions d_j:
        d_0 = D^-1 r / theta,  rho_0 = delta / theta,
        rho_j = 1 / (2 theta / delta - rho_{j-1}),
        d_j = rho_j rho_{j-1} d_{j-1} + (2 rho_j / delta) D^-1 (r - A z_j),  z_{j+1} = z_j + d_j."""
    r = np.asarray(r, dtype=np.float64)
    theta, delta = 0.5 * (hi + lo), 0.5 * (hi - lo)
    rho = delta / theta
    d = dinv * r / theta
    z = d.copy()
    for _ in range(1, k):
        rho_new = 1.0 / (2.0 * theta / delta - rho)
        d = rho_new * rho * d + (2.0 * rho_new / delta) * (dinv * (r - A(z)))
        rho = rho_new
        z = z + d
    return z


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
