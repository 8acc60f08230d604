"""Pins for the oracle's CG, load vector and L2 error (CPU only): agreement with a dense direct
solve, the O(h^{p+1}) L2 convergence of the manufactured sine solution, and breakdown detection."""
import numpy as np
import pytest

from oracle import operator as op
from oracle import solve
from oracle.solve import pcg, load_vector, l2_error, u_exact
from oracle.mesh import boundary_mask, dof_coordinates
from oracle.element import DIFFUSION, MASS
from paper_2603_09038_gb300.inputs import perturbed_vertices, lognormal_coefficient


def _dirichlet_system(prob):
    m = boundary_mask(prob.nx, prob.ny, prob.nz, prob.p).astype(np.float64)
    keep = 1.0 - m
    A = op.assemble(prob, DIFFUSION)
    d = op.diagonal(prob, DIFFUSION) * keep + m
    return A, m, keep, d


def test_pcg_matches_dense_solve():
    n, p = 2, 2
    V = perturbed_vertices(n, n, n)
    prob = op.Problem(n, n, n, p, V, coeff=lognormal_coefficient(n ** 3, 1.0))
    A, m, keep, d = _dirichlet_system(prob)
    b = load_vector(prob) * keep
    Abc = op.constrained(lambda v: op.apply(prob, v, DIFFUSION), m)
    x, it, hist = pcg(Abc, b, d, rtol=1e-13)
    dense = (np.diag(keep) @ A.toarray() @ np.diag(keep)) + np.diag(m)
    xd = np.linalg.solve(dense, b)
    assert np.abs(x - xd).max() <= 1e-10 * np.abs(xd).max()
    assert hist[-1] <= 1e-13 and it <= prob.ndofs


@pytest.mark.parametrize("p,meshes", [(1, (8, 16)), (2, (4, 8)), (3, (4, 8))])
def test_l2_convergence_rate_p_plus_1(p, meshes):
    errs = []
    for n in meshes:
        prob = op.Problem(n, n, n, p, perturbed_vertices(n, n, n))
        A, m, keep, d = _dirichlet_system(prob)
        b = load_vector(prob) * keep
        x, _, _ = pcg(lambda v: keep * (A @ (keep * v)) + m * v, b, d, rtol=1e-12)
        errs.append(l2_error(prob, x))
    rate = np.log2(errs[0] / errs[1])
    assert abs(rate - (p + 1)) < 0.2, (errs, rate)


def test_l2_error_of_interpolant_and_of_exact_polynomial():
    """The L2 error routine is exact on the space: the error of a Q_p function's interpolant is 0,
    and the sine's nodal interpolant has the expected O(h^{p+1}) size."""
    n, p = 2, 2
    V = perturbed_vertices(n, n, n, amp=0.0)
    prob = op.Problem(n, n, n, p, V)
    X = dof_coordinates(V, n, n, n, p)
    poly = lambda Y: Y[..., 0] ** 2 * Y[..., 1] - Y[..., 2]
    assert l2_error(prob, poly(X), u=poly) < 1e-14
    e1 = l2_error(prob, u_exact(X))
    prob2 = op.Problem(2 * n, 2 * n, 2 * n, p, perturbed_vertices(2 * n, 2 * n, 2 * n, amp=0.0))
    e2 = l2_error(prob2, u_exact(dof_coordinates(prob2.vertices, 2 * n, 2 * n, 2 * n, p)))
    assert 2.5 < np.log2(e1 / e2) < 3.5


def test_load_vector_integrates_f():
    """1^T b = int f = 3 pi^2 (2/pi)^3 up to quadrature error, and the mass-matrix identity
    b = M f_h holds for f in the discrete space."""
    n, p = 4, 3
    prob = op.Problem(n, n, n, p, perturbed_vertices(n, n, n))
    b = load_vector(prob)
    exact = 3 * np.pi ** 2 * (2 / np.pi) ** 3
    assert abs(b.sum() - exact) < 1e-4 * exact
    X = dof_coordinates(prob.vertices, n, n, n, p)
    lin = lambda Y: 1.0 + Y[..., 0] - 2 * Y[..., 2]
    bl = load_vector(prob, f=lin)
    # on a trilinear mesh the physical linear function is an element of the trilinear image space
    np.testing.assert_allclose(bl, op.apply(prob, lin(X), MASS), atol=1e-14 * np.abs(bl).max())


def test_pcg_detects_indefinite_operator():
    n, p = 2, 1
    prob = op.Problem(n, n, n, p, perturbed_vertices(n, n, n))
    b = np.ones(prob.ndofs)
    with pytest.raises(ArithmeticError):
        pcg(lambda v: -op.apply(prob, v, MASS), b, np.ones(prob.ndofs), rtol=1e-10)


def _cheb_T(k, x):
    """T_k(x) by its closed forms (cos / cosh), independent of any recurrence."""
    x = np.asarray(x, dtype=np.float64)
    out = np.empty_like(x)
    inside = np.abs(x) <= 1.0
    out[inside] = np.cos(k * np.arccos(x[inside]))
    xo = x[~inside]
    out[~inside] = np.sign(xo) ** k * np.cosh(k * np.arccosh(np.abs(xo)))
    return out


@pytest.mark.parametrize("k", [1, 2, 3, 4, 7])
def test_chebyshev_matches_closed_form_polynomial(k):
    """On A = diag(lam), D = diag(d): z_i = q(lam_i / d_i) r_i / d_i with
    1 - mu q(mu) = T_k((theta - mu) / delta) / T_k(theta / delta) (pinned by the cos/cosh forms
    of T_k, not by the three-term recurrence the oracle uses)."""
    rng = np.random.default_rng(k)
    n = 50
    d = rng.uniform(0.5, 2.0, n)
    mu = np.concatenate([rng.uniform(0.01, 2.0, n - 2), [0.004, 2.0]])  # eigenvalues of D^-1 A
    lam = mu * d
    r = rng.standard_normal(n)
    lo, hi = 0.05, 2.0
    z = solve.chebyshev(lambda v: lam * v, 1.0 / d, r, k, lo, hi)
    theta, delta = (hi + lo) / 2, (hi - lo) / 2
    e = _cheb_T(k, (theta - mu) / delta) / _cheb_T(k, np.array([theta / delta]))[0]
    q = (1.0 - e) / mu
    np.testing.assert_allclose(z, q * r / d, rtol=1e-11, atol=1e-12)
    # positive on (0, hi]: an SPD preconditioner whenever hi bounds the spectrum
    assert np.all(q > 0)


def test_chebyshev_pcg_solves_and_beats_jacobi():
    """Chebyshev-PCG (degree 4, [lmax/30, lmax] with the exact lmax of D^-1 A_bc) reaches the
    dense solution and needs fewer iterations than Jacobi-PCG on the same system."""
    from oracle.mesh import boundary_mask
    from paper_2603_09038_gb300.inputs import perturbed_vertices
    n, p = 4, 3
    V = perturbed_vertices(n, n, n)
    prob = op.Problem(n, n, n, p, V)
    A = op.assemble(prob, DIFFUSION).toarray()
    m = boundary_mask(n, n, n, p).astype(np.float64)
    keep = 1.0 - m
    Abc = keep[:, None] * A * keep[None, :] + np.diag(m)
    dg = np.diag(Abc)
    dinv = keep / dg
    b = solve.load_vector(prob) * keep
    s = np.sqrt(dg)
    lmax = np.linalg.eigvalsh(Abc / s[:, None] / s[None, :]).max()
    Aop = lambda v: keep * (A @ (keep * v))
    xc, itc, _ = solve.pcg_prec(Aop, b, lambda r: solve.chebyshev(Aop, dinv, r, 4, lmax / 30, lmax),
                                rtol=1e-10)
    xj, itj, _ = solve.pcg(lambda v: Abc @ v, b, dg, rtol=1e-10)
    x = np.linalg.solve(Abc, b)
    assert np.abs(xc - x).max() <= 1e-8 * np.abs(x).max()
    assert itc * 2 < itj, (itc, itj)
