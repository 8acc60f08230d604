"""Pins of oracle/learned.py (CPU): the patch operator with exact local inverses equals the
symmetrically weighted additive Schwarz matrix assembled element by element; the local blocks
equal what probing the operator with unit vectors reads back; flexible CG with a fixed SPD
preconditioner produces the preconditioned-CG iterates; the patch operator is positively
homogeneous and its BF16 rounding bound covers an explicit BF16 evaluation; the Adam update
matches its closed forms."""
import numpy as np
import pytest

from oracle import learned as ol
from oracle import mlp as omlp
from oracle import operator as oop
from oracle.element import DIFFUSION
from oracle.mesh import boundary_mask, dof_map
from oracle.solve import pcg as oracle_pcg, load_vector
from paper_2603_09038_gb300.inputs import perturbed_vertices, lognormal_coefficient


def _prob(dims=(3, 3, 2), p=2, sigma=1.0):
    V = perturbed_vertices(*dims)
    c = lognormal_coefficient(int(np.prod(dims)), sigma)
    return oop.Problem(*dims, p, V, coeff=c)


def test_exact_local_inverses_give_weighted_additive_schwarz():
    prob = _prob()
    A = oop.assemble(prob, DIFFUSION)
    dmap, S, W = ol.patch_data(prob, DIFFUSION)
    Sp = np.where(S > 0, 1.0 / np.where(S > 0, S, 1.0), 0.0)        # pseudo-inverse of S
    inv = [np.linalg.inv(ol.local_block(prob, DIFFUSION, e, A)) for e in range(prob.ne)]

    def f_exact(Xn, elems):   # x -> S_e^+ A_ee^-1 S_e^+ x, element by element
        return np.stack([Sp[dmap[e]] * (inv[e] @ (Sp[dmap[e]] * x)) for x, e in zip(Xn, elems)])

    Mx = ol.additive_schwarz(prob, DIFFUSION)
    rng = np.random.default_rng(3)
    for _ in range(3):
        r = rng.standard_normal(prob.ndofs)
        z = ol.patch_apply(prob, DIFFUSION, f_exact, r)
        assert np.abs(z - Mx @ r).max() <= 1e-12 * np.abs(Mx @ r).max()
    mask = boundary_mask(prob.nx, prob.ny, prob.nz, prob.p) == 1
    Mi = Mx[~mask][:, ~mask]
    assert np.allclose(Mi, Mi.T, rtol=0, atol=1e-14 * np.abs(Mi).max())
    assert np.linalg.eigvalsh(Mi).min() > 0                            # SPD on the free dofs
    assert np.all(Mx[mask] == 0) and np.all(Mx[:, mask] == 0)


def test_local_block_equals_probing_the_operator():
    prob = _prob((4, 3, 3), 3)
    e = 1 + 4 * (1 + 3 * 1)                                             # interior element
    idx = dof_map(prob.nx, prob.ny, prob.nz, prob.p, [e])[0]
    Aee = ol.local_block(prob, DIFFUSION, e)
    probe = np.zeros_like(Aee)
    for a, g in enumerate(idx):
        u = np.zeros(prob.ndofs)
        u[g] = 1.0
        probe[:, a] = oop.apply(prob, u, DIFFUSION)[idx]
    assert np.abs(probe - Aee).max() <= 1e-13 * np.abs(Aee).max()
    # the target relation t = S^-1 A_ee^-1 S^-1 x, and t does not depend on the scale of x
    _, S, _ = ol.patch_data(prob, DIFFUSION)
    x = np.random.default_rng(1).standard_normal(len(idx))
    t = ol.local_target(prob, DIFFUSION, e, x)
    assert np.abs(S[idx] * (Aee @ (S[idx] * t)) - x).max() <= 1e-12 * np.abs(x).max()
    assert np.allclose(ol.local_target(prob, DIFFUSION, e, 3.0 * x), 3.0 * t, rtol=1e-13, atol=0)
    with pytest.raises(ValueError):
        ol.local_target(prob, DIFFUSION, 0, x)                          # touches the boundary


def test_fcg_with_fixed_spd_preconditioner_is_pcg():
    prob = _prob((4, 3, 3), 2)
    m = boundary_mask(prob.nx, prob.ny, prob.nz, prob.p).astype(np.float64)
    keep = 1.0 - m
    A = oop.assemble(prob, DIFFUSION)
    Abc = lambda v: keep * (A @ (keep * v)) + m * v
    d = oop.diagonal(prob, DIFFUSION) * keep + m
    b = load_vector(prob) * keep
    x_p, it_p, hist_p = oracle_pcg(Abc, b, d, rtol=1e-10)
    x_f, it_f, hist_f, _ = ol.fcg(Abc, lambda r: r / d, b, rtol=1e-10)
    assert it_f == it_p
    assert np.allclose(hist_f, hist_p, rtol=1e-6, atol=1e-14)
    assert np.abs(x_f - x_p).max() <= 1e-10 * np.abs(x_p).max()
    # a nonlinear (positively homogeneous) preconditioner still converges to the solution
    x_n, it_n, _, _ = ol.fcg(Abc, lambda r: r / d * (1.0 + 0.1 * np.tanh(r / (np.abs(r).max() + 1e-300))),
                             b, rtol=1e-10, maxit=2000)
    assert np.abs(x_n - x_p).max() <= 1e-7 * np.abs(x_p).max()


@pytest.mark.parametrize("width", [0, 16])
def test_patch_apply_homogeneous_and_bf16_bound(width):
    prob = _prob((3, 2, 3), 2)
    din = (prob.p + 1) ** 3
    rng = np.random.default_rng(5 + width)
    W = omlp.init_weights(din, width, 9)[:3] + (0.2 * rng.standard_normal((din, din)),)
    Wb = tuple(ol.bf16_round(w) for w in W)
    r = rng.standard_normal(prob.ndofs)
    z, zb = ol.patch_apply(prob, DIFFUSION, ol.network(Wb), r, bound=ol.network_rounding_bound(Wb))
    z2 = ol.patch_apply(prob, DIFFUSION, ol.network(Wb), 2.5 * r)
    assert np.allclose(z2, 2.5 * z, rtol=1e-13, atol=1e-300)
    # an explicit BF16 evaluation (rounded input and hidden activations) stays inside the bound
    W1, W2, W3, W0 = omlp._weights(Wb)

    def f_bf16(Xn, elems):
        a = ol.bf16_round(Xn)
        y = a @ W0
        if width:
            h = ol.bf16_round(omlp.relu(a @ W1))
            h = ol.bf16_round(omlp.relu(h @ W2))
            y = y + h @ W3
        return y
    zq = ol.patch_apply(prob, DIFFUSION, f_bf16, r)
    assert np.all(np.abs(zq - z) <= zb)
    assert np.abs(zq - z).max() > 0 and zb.max() <= 0.25 * np.abs(z).max()


def test_adam_closed_forms():
    rng = np.random.default_rng(2)
    w0, g1, g2 = rng.standard_normal(50), rng.standard_normal(50), rng.standard_normal(50)
    m0, v0 = np.zeros(50), np.zeros(50)
    lr, eps = 1e-3, 1e-8
    w1, m1, v1 = ol.adam_step(w0, g1, m0, v0, 1, lr)
    # first step: bias-corrected moments are g and g^2, so the step is lr * g / (|g| + eps)
    assert np.allclose(w1, w0 - lr * g1 / (np.abs(g1) + eps), rtol=1e-14, atol=0)
    w2, m2, v2 = ol.adam_step(w1, g2, m1, v1, 2, lr)
    mh = (0.9 * 0.1 * g1 + 0.1 * g2) / (1 - 0.81)
    vh = (0.999 * 0.001 * g1 ** 2 + 0.001 * g2 ** 2) / (1 - 0.999 ** 2)
    assert np.allclose(w2, w1 - lr * mh / (np.sqrt(vh) + eps), rtol=1e-13, atol=0)
    # a constant gradient moves every weight by lr per step
    w, m, v = w0.copy(), m0.copy(), v0.copy()
    for t in range(1, 6):
        w, m, v = ol.adam_step(w, np.full(50, 0.3), m, v, t, lr)
    assert np.allclose(w, w0 - 5 * lr, rtol=0, atol=1e-9)


def _lattice_perm(S, nx, ny, nz, p):
    """perm[i] = the variable-order space's true dof at the single-order mesh's dof i (matched by
    lattice coordinates)."""
    from oracle.quadrature import gauss_lobatto
    t = gauss_lobatto(p + 1)

    def coord(I, n):
        e = np.minimum(I // p, n - 1)
        return e + t[I - e * p]
    N = [nx * p + 1, ny * p + 1, nz * p + 1]
    K, J, I = np.meshgrid(np.arange(N[2]), np.arange(N[1]), np.arange(N[0]), indexing="ij")
    mc = np.stack([coord(I.reshape(-1), nx), coord(J.reshape(-1), ny), coord(K.reshape(-1), nz)], 1)
    key = {tuple(np.round(c, 9)): k for k, c in enumerate(S.true_lattice_coords())}
    return np.array([key[tuple(np.round(c, 9))] for c in mc])


def test_vspace_patch_operator_reduces_to_the_single_order_one():
    """With one order on every element the variable-order patch operator (the X numbering, the
    shared scaling (mult diag)^-1/2, the constrained-row mask) is patch_apply's, dof by dof."""
    from oracle.varorder import VarSpace
    dims, p = (3, 2, 3), 2
    prob = _prob(dims, p, sigma=1.0)
    S = VarSpace(*dims, np.full(int(np.prod(dims)), p, dtype=np.int32))
    perm = _lattice_perm(S, *dims, p)
    din = (p + 1) ** 3
    rng = np.random.default_rng(3)
    W = omlp.init_weights(din, 16, 3)
    W = (W[0], W[1], W[2], W[3] + 0.1 * rng.standard_normal(W[3].shape))
    r = rng.standard_normal(prob.ndofs)
    zs = ol.patch_apply(prob, DIFFUSION, ol.network(W), r)
    rv = np.zeros(S.ntrue)
    rv[perm] = r
    zv = ol.vspace_patch_apply(S, prob.vertices, DIFFUSION, {p: ol.network(W)}, rv,
                               coeff=prob.coeff)
    assert np.abs(zv[perm] - zs).max() <= 1e-12 * np.abs(zs).max()


def test_vspace_patch_operator_symmetric_for_a_symmetric_linear_map():
    """f(x) = x W0 with W0 symmetric per order: M = E^T F (sum_e R_e^T W0 R_e) F E is symmetric on
    a mixed-order space with constrained nodes (built column by column)."""
    from oracle.varorder import VarSpace
    from paper_2603_09038_gb300.inputs import block_orders
    dims = (2, 2, 2)
    orders = block_orders(*dims, block=1, orders=(1, 2, 3), seed=4)
    S = VarSpace(*dims, orders)
    V = perturbed_vertices(*dims, seed=5)
    rng = np.random.default_rng(6)
    nets = {}
    for p in np.unique(orders):
        d = (int(p) + 1) ** 3
        A = rng.standard_normal((d, d))
        W0 = A + A.T
        nets[int(p)] = (lambda W0_: (lambda Xn, el: Xn @ W0_))(W0)
    n = S.ntrue
    E, mats = S.prolongation(), S.element_matrices(V, DIFFUSION)
    M = np.stack([ol.vspace_patch_apply(S, V, DIFFUSION, nets, np.eye(n)[j], E=E, mats=mats)
                  for j in range(n)], 1)
    assert np.abs(M).max() > 0
    assert np.abs(M - M.T).max() <= 1e-11 * np.abs(M).max()
    interior = S.boundary_mask() == 0
    assert np.all(M[~interior] == 0.0) and np.all(M[:, ~interior] == 0.0)


def _mean_scaled_inverse(p, sigma, n=4):
    """Mean over the interior elements of an n^3 order-p mesh (log-normal coefficient sigma, its
    own seed) of the scaled local inverse S_e^-1 A_ee^-1 S_e^-1 (the map an exact patch network
    would realise)."""
    c = None if sigma == 0 else np.exp(sigma * np.random.default_rng(11).standard_normal(n ** 3))
    prob = oop.Problem(n, n, n, p, perturbed_vertices(n, n, n), coeff=c)
    A = oop.assemble(prob, DIFFUSION)
    _, S, _ = ol.patch_data(prob, DIFFUSION)
    d = (p + 1) ** 3
    acc, cnt = np.zeros((d, d)), 0
    for ez in range(1, n - 1):
        for ey in range(1, n - 1):
            for ex in range(1, n - 1):
                e = ex + n * (ey + n * ez)
                acc += np.stack([ol.local_target(prob, DIFFUSION, e, col, A=A, S=S)
                                 for col in np.eye(d)], 1)
                cnt += 1
    return acc / cnt


@pytest.mark.parametrize("sigma", [0.0, 2.0])
def test_vspace_patch_operator_beats_jacobi_with_exact_patch_maps(sigma):
    """Per-order maps set to the mean exact scaled local inverse of a single-order mesh: flexible
    CG with the variable-order patch operator needs fewer iterations than Jacobi on a mixed-order
    space, with a unit and a log-normal (sigma = 2) coefficient. This fails when the constrained
    rows also gather E r (that counts the residual of the true dofs they interpolate twice), and
    at sigma = 2 when a true dof's scaling leaves out the higher-order neighbours that read it
    through constrained nodes."""
    from oracle.varorder import VarSpace
    from paper_2603_09038_gb300.inputs import block_orders
    import scipy.sparse as sp
    n = 4
    orders = block_orders(n, n, n, block=2, orders=(2, 3), seed=7)
    assert len(set(orders.tolist())) == 2
    S = VarSpace(n, n, n, orders)
    V = perturbed_vertices(n, n, n)
    c = None if sigma == 0 else np.exp(sigma * np.random.default_rng(2).standard_normal(n ** 3))
    E, mats = S.prolongation(), S.element_matrices(V, DIFFUSION, c)
    A = S.assemble(V, DIFFUSION, coeff=c, sparse=True).tocsr()
    inner = (S.boundary_mask() == 0).astype(np.float64)
    Abc = (sp.diags(inner) @ A @ sp.diags(inner) + sp.diags(1.0 - inner)).tocsr()
    nets = {}
    for p in (2, 3):
        T = _mean_scaled_inverse(p, sigma)
        nets[p] = (lambda T_: (lambda Xn, el: Xn @ T_.T))(T)
    b = np.random.default_rng(5).uniform(-1, 1, S.ntrue) * inner
    diag = Abc.diagonal()
    _, it_j, _, _ = ol.fcg(Abc, lambda r: r / diag, b, rtol=1e-8)
    _, it_l, _, _ = ol.fcg(Abc, lambda r: ol.vspace_patch_apply(S, V, DIFFUSION, nets, r,
                                                                coeff=c, E=E, mats=mats),
                           b, rtol=1e-8)
    assert it_l < 0.85 * it_j, (it_l, it_j)
