"""1D quadrature rules and the 1D Lagrange basis (oracle; test infrastructure only).

Eq. (2) of the paper writes the tensor-product basis as ``B_abc,ijk = B1d_ai B1d_bj B1d_ck``:
everything in 3D is built from a 1D basis evaluated at 1D quadrature points.  The paper does not
fix the nodes or the rule; the readings used here (standard for H1 spectral elements) are

* trial/test nodes: the p+1 Gauss-Lobatto-Legendre (GLL) points of [0, 1];
* quadrature: the Q-point Gauss-Legendre (GL) rule on [0, 1], Q = p + 2 by default;
* ``B1d[q][d] = l_d(x_q)`` and ``G1d[q][d] = l_d'(x_q)`` with ``l_d`` the Lagrange polynomial of
  node d.

Everything is computed in float64 from the defining properties (Newton iteration on Legendre
polynomials; Lagrange products), with no tabulated constants.
"""
import numpy as np


def legendre(n, x):
    """Legendre polynomial P_n and its derivative at points x (Bonnet's recurrence).

    (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1};  P_n' = n (x P_n - P_{n-1}) / (x^2 - 1).
    The derivative formula is used only away from x = +-1.
    """
    x = np.asarray(x, dtype=np.float64)
    if n == 0:
        return np.ones_like(x), np.zeros_like(x)
    p_prev, p = np.ones_like(x), x.copy()
    for k in range(1, n):
        p_prev, p = p, ((2 * k + 1) * x * p - k * p_prev) / (k + 1)
    dp = n * (x * p - p_prev) / (x * x - 1.0)
    return p, dp


def legendre_d2(n, x):
    """P_n, P_n', P_n'' at x, the second derivative from Legendre's equation
    (1 - x^2) P'' - 2 x P' + n (n+1) P = 0 (valid away from x = +-1)."""
    p, dp = legendre(n, x)
    d2p = (2.0 * x * dp - n * (n + 1) * p) / (1.0 - x * x)
    return p, dp, d2p


def _newton(f, x0, iters=100):
    x = np.array(x0, dtype=np.float64)
    for _ in range(iters):
        val, der = f(x)
        dx = val / der
        x = x - dx
        if np.max(np.abs(dx)) < 1e-16:
            break
    return x


def gauss_legendre(q):
    """Q-point Gauss-Legendre rule mapped to [0, 1]: (points ascending, weights).

    Nodes are the roots of P_Q on [-1, 1] (Newton from Chebyshev-like guesses); weights are
    2 / ((1 - x^2) P_Q'(x)^2).  The map t = (x + 1) / 2 halves the weights.
    """
    if q < 1:
        raise ValueError("need at least one Gauss point")
    i = np.arange(q)
    guess = np.cos(np.pi * (i + 0.75) / (q + 0.5))
    x = _newton(lambda t: legendre(q, t), guess)
    _, dp = legendre(q, x)
    w = 2.0 / ((1.0 - x * x) * dp * dp)
    order = np.argsort(x)
    x, w = x[order], w[order]
    return (x + 1.0) / 2.0, w / 2.0


def gauss_lobatto(d):
    """The d Gauss-Lobatto-Legendre points on [0, 1] (ascending): the end points and the roots of
    P_{d-1}' (Newton on P' with P'' from Legendre's equation)."""
    if d < 2:
        raise ValueError("GLL needs at least two points")
    n = d - 1
    if n == 1:
        x = np.array([-1.0, 1.0])
    else:
        guess = np.cos(np.pi * np.arange(1, n) / n)
        def f(t):
            _, dp, d2p = legendre_d2(n, t)
            return dp, d2p
        interior = _newton(f, guess)
        x = np.concatenate(([-1.0], np.sort(interior), [1.0]))
    return (x + 1.0) / 2.0


def lagrange(nodes, x):
    """Lagrange basis of the given nodes at points x, by the product formulas.

    Returns (L, dL) with L[q, d] = l_d(x_q) = prod_{m != d} (x_q - t_m) / (t_d - t_m) and
    dL[q, d] = l_d'(x_q) = sum_{m != d} 1/(t_d - t_m) prod_{l != d, m} (x_q - t_l) / (t_d - t_l).
    """
    t = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(t)
    L = np.ones((len(x), n))
    dL = np.zeros((len(x), n))
    for d in range(n):
        for m in range(n):
            if m == d:
                continue
            L[:, d] *= (x - t[m]) / (t[d] - t[m])
        for m in range(n):
            if m == d:
                continue
            term = np.full(len(x), 1.0 / (t[d] - t[m]))
            for l in range(n):
                if l == d or l == m:
                    continue
                term *= (x - t[l]) / (t[d] - t[l])
            dL[:, d] += term
    return L, dL


def basis_1d(p, q):
    """(B1d, G1d, points, weights, nodes) for order p with a Q-point Gauss rule: B1d[q, d] =
    l_d(x_q), G1d[q, d] = l_d'(x_q) on the p+1 GLL nodes (the 1D matrices of Eq. (2))."""
    nodes = gauss_lobatto(p + 1)
    pts, wts = gauss_legendre(q)
    B, G = lagrange(nodes, pts)
    return B, G, pts, wts, nodes
