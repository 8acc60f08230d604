"""Pins for the oracle's variable-order (minimum-rule) space and its operator (CPU only).

Each pin checks the oracle against something other than itself: a hand-derived numbering, the
dimension of the continuous piecewise-polynomial space by brute force, exact reproduction of
polynomials, closed-form energies, and the single-order case against the structured operator.
"""
import numpy as np
import pytest

from oracle import operator as op
from oracle.element import DIFFUSION, MASS
from oracle.quadrature import gauss_lobatto, lagrange
from oracle.varorder import VarSpace
from paper_2603_09038_gb300.inputs import block_orders, perturbed_vertices, uniform_vector


def _lattice(nx, ny, nz):
    """Unperturbed vertex lattice with unit spacing (element (ex, ey, ez) = [ex, ex+1] x ...)."""
    zs, ys, xs = np.meshgrid(np.arange(nz + 1.0), np.arange(ny + 1.0), np.arange(nx + 1.0),
                             indexing="ij")
    return np.stack([xs.reshape(-1), ys.reshape(-1), zs.reshape(-1)], axis=1)


def _node_coords(S):
    """Lattice coordinates of every E-vector row, computed from the element layout alone."""
    out = np.zeros((S.nlocal, 3))
    for e in range(S.ne):
        p = int(S.order[e])
        D = p + 1
        t = gauss_lobatto(D)
        ex, ey, ez = e % S.nx, (e // S.nx) % S.ny, e // (S.nx * S.ny)
        a = np.arange(D ** 3)
        i, j, k = a % D, (a // D) % D, a // (D * D)
        s = S.local_first[e]
        out[s:s + D ** 3] = np.stack([ex + t[i], ey + t[j], ez + t[k]], axis=1)
    return out


def test_hand_numbering_two_elements():
    """A 2 x 1 x 1 mesh of orders (1, 2), numbered by hand from the documented rule: 12 vertices,
    then the order-2 element's four x-edges, its y-edges and z-edges at x = 2, its x-normal face
    at x = 2, its two y-normal and two z-normal faces, and its cell.  The shared face and the
    edges on it take order 1 (no dofs): 26 true dofs = 8 + 27 - 9 constrained face nodes."""
    S = VarSpace(2, 1, 1, [1, 2])
    assert S.ntrue == 26 and S.nlocal == 35
    expect = [(1.5, 0, 0), (1.5, 1, 0), (1.5, 0, 1), (1.5, 1, 1),      # x-edges
              (2, 0.5, 0), (2, 0.5, 1),                                # y-edges
              (2, 0, 0.5), (2, 1, 0.5),                                # z-edges
              (2, 0.5, 0.5),                                           # x-normal face
              (1.5, 0, 0.5), (1.5, 1, 0.5),                            # y-normal faces
              (1.5, 0.5, 0), (1.5, 0.5, 1),                            # z-normal faces
              (1.5, 0.5, 0.5)]                                         # cell
    np.testing.assert_array_equal(S.true_lattice_coords()[12:], np.array(expect, dtype=float))
    # the order-2 element's node at the centre of the shared face is the mean of its 4 corners
    E = S.prolongation().toarray()
    a = 0 + 3 * (1 + 3 * 1)                    # (i, j, k) = (0, 1, 1) of element 1
    row = E[8 + a]
    corners = [1 + 3 * (0 + 2 * 0), 1 + 3 * (1 + 2 * 0), 1 + 3 * (0 + 2 * 1), 1 + 3 * (1 + 2 * 1)]
    np.testing.assert_allclose(row[corners], 0.25, rtol=0, atol=1e-15)
    others = np.setdiff1d(np.arange(row.size), corners)
    assert abs(row.sum() - 1.0) < 1e-15 and np.abs(row[others]).max() <= 1e-15


def _jump_matrix(S):
    """Rows: value jumps across every interior face at (P+2)^2 points, on the discontinuous
    local space (all elements' nodal values concatenated)."""
    P = int(S.order.max())
    pts = 0.5 - 0.5 * np.cos(np.pi * (np.arange(P + 2) + 0.5) / (P + 2))   # distinct, interior
    rows = []
    for e in range(S.ne):
        ex, ey, ez = e % S.nx, (e // S.nx) % S.ny, e // (S.nx * S.ny)
        c = [ex, ey, ez]
        n = [S.nx, S.ny, S.nz]
        for d in range(3):
            if c[d] + 1 >= n[d]:
                continue
            nb = c.copy()
            nb[d] += 1
            f = nb[0] + S.nx * (nb[1] + S.ny * nb[2])
            u, v = [a for a in range(3) if a != d]
            for s in pts:
                for t in pts:
                    r = np.zeros(S.nlocal)
                    for el, side in ((e, 1.0), (f, 0.0)):
                        p = int(S.order[el])
                        D = p + 1
                        L = [None] * 3
                        tq = gauss_lobatto(D)
                        L[d] = lagrange(tq, [side])[0][0]
                        L[u] = lagrange(tq, [s])[0][0]
                        L[v] = lagrange(tq, [t])[0][0]
                        phi = np.einsum('k,j,i->kji', L[2], L[1], L[0]).reshape(-1)
                        sgn = 1.0 if el == e else -1.0
                        r[S.local_first[el]:S.local_first[el] + D ** 3] += sgn * phi
                    rows.append(r)
    return np.array(rows)


@pytest.mark.parametrize("dims,orders", [
    ((2, 2, 2), [1, 2, 3, 2, 2, 1, 3, 2]),
    ((3, 2, 1), [2, 4, 2, 3, 1, 4]),
    ((2, 2, 2), [3] * 8),
    ((2, 1, 2), [8, 5, 7, 6]),
])
def test_dimension_equals_continuous_space(dims, orders):
    """Brute force: the continuous piecewise-Q_{p_e} functions are the null space of the face
    jumps on the discontinuous space; its dimension must equal the number of true dofs, E must
    have full column rank, and every E x must be continuous."""
    S = VarSpace(*dims, orders)
    J = _jump_matrix(S)
    sv = np.linalg.svd(J, compute_uv=False)
    rank = int((sv > 1e-10 * sv[0]).sum())
    assert S.nlocal - rank == S.ntrue
    E = S.prolongation().toarray()
    assert np.linalg.matrix_rank(E) == S.ntrue
    assert np.abs(J @ E).max() < 1e-12


@pytest.mark.parametrize("dims,orders", [((3, 2, 2), None), ((2, 2, 2), [2, 5, 3, 2, 4, 2, 6, 3])])
def test_polynomial_reproduction(dims, orders):
    """A global polynomial of degree <= the smallest order in each variable lies in the space:
    its values at the true-dof positions, prolonged, are its values at every element node."""
    nx, ny, nz = dims
    if orders is None:
        orders = block_orders(nx, ny, nz, block=1, orders=(2, 4, 6), seed=3)
    S = VarSpace(nx, ny, nz, orders)

    def u(X):
        x, y, z = X[:, 0], X[:, 1], X[:, 2]
        return (1 + x - 0.4 * x ** 2) * (2 - y + 0.3 * y ** 2) * (1 + 0.7 * z - 0.2 * z ** 2)

    E = S.prolongation()
    np.testing.assert_allclose(E @ u(S.true_lattice_coords()), u(_node_coords(S)),
                               rtol=0, atol=1e-12)


def test_polynomial_reproduction_high_orders():
    """Orders 5..8 reproduce a degree-5 polynomial in each variable exactly."""
    S = VarSpace(2, 2, 1, [5, 8, 7, 6])

    def u(X):
        x, y, z = X[:, 0], X[:, 1], X[:, 2]
        return (1 + x ** 5 - 0.3 * x ** 3) * (0.5 + y ** 4 - y ** 5 / 3) * (1 - z ** 5 + 2 * z)

    np.testing.assert_allclose(S.prolongation() @ u(S.true_lattice_coords()), u(_node_coords(S)),
                               rtol=0, atol=1e-11)


def test_energy_closed_forms():
    """Unit-spacing affine mesh [0,3] x [0,2] x [0,2], mixed orders: for u = x y,
    u^T K u = int |grad u|^2 = nz (nx ny^3 + ny nx^3) / 3 and u^T M u = int u^2 =
    nz nx^3 ny^3 / 9; constants are in the kernel of the diffusion operator."""
    nx, ny, nz = 3, 2, 2
    S = VarSpace(nx, ny, nz, block_orders(nx, ny, nz, block=1, orders=(1, 2, 3), seed=5))
    V = _lattice(nx, ny, nz)
    X = S.true_lattice_coords()
    uu = X[:, 0] * X[:, 1]
    K = S.assemble(V, DIFFUSION)
    M = S.assemble(V, MASS)
    assert abs(uu @ K @ uu - nz * (nx * ny ** 3 + ny * nx ** 3) / 3.0) < 1e-11
    assert abs(uu @ M @ uu - nz * nx ** 3 * ny ** 3 / 9.0) < 1e-10
    assert np.abs(K @ np.ones(S.ntrue)).max() < 1e-12
    assert np.abs(K - K.T).max() < 1e-13 and np.abs(M - M.T).max() < 1e-13
    assert np.linalg.eigvalsh(M).min() > 0


@pytest.mark.parametrize("p", [1, 2, 3])
def test_single_order_equals_structured_operator(p):
    """With one order everywhere P is a permutation and the operator is the structured one."""
    n = 2
    V = perturbed_vertices(n, n, n, seed=7)
    S = VarSpace(n, n, n, [p] * n ** 3)
    X = S.true_lattice_coords()
    # structured lattice index of each true dof from its position
    I = np.rint(X * p).astype(np.int64)
    N = n * p + 1
    perm = I[:, 0] + N * (I[:, 1] + N * I[:, 2])
    assert np.array_equal(np.sort(perm), np.arange(N ** 3))
    prob = op.Problem(n, n, n, p, V)
    for kind in (DIFFUSION, MASS):
        A = op.assemble(prob, kind).toarray()
        B = S.assemble(V, kind)
        assert np.abs(B - A[np.ix_(perm, perm)]).max() < 1e-13 * np.abs(A).max()


def test_boundary_mask_and_apply_match_assembly():
    nx, ny, nz = 2, 2, 3
    S = VarSpace(nx, ny, nz, block_orders(nx, ny, nz, block=1, orders=(2, 3, 4), seed=11))
    X = S.true_lattice_coords()
    m = S.boundary_mask()
    interior = (X[:, 0] > 0) & (X[:, 0] < nx) & (X[:, 1] > 0) & (X[:, 1] < ny) & \
               (X[:, 2] > 0) & (X[:, 2] < nz)
    np.testing.assert_array_equal(m, (~interior).astype(np.uint8))
    V = perturbed_vertices(nx, ny, nz, seed=2)
    x = uniform_vector(S.ntrue, seed=4)
    for kind in (DIFFUSION, MASS):
        np.testing.assert_allclose(S.apply(V, x, kind), S.assemble(V, kind) @ x, rtol=0,
                                   atol=1e-13 * np.abs(x).max() * 50)


def test_block_orders_layout():
    o = block_orders(16, 16, 8, block=8, orders=(2, 4, 6), seed=0).reshape(8, 16, 16)
    assert set(np.unique(o)) <= {2, 4, 6}
    for bz in range(1):
        for by in range(2):
            for bx in range(2):
                blk = o[bz * 8:(bz + 1) * 8, by * 8:(by + 1) * 8, bx * 8:(bx + 1) * 8]
                assert np.unique(blk).size == 1


def test_jacobi_diagonal_single_order_and_unconstrained_dofs():
    """One order: the structured operator's diagonal (permuted).  Mixed orders: the exact
    diagonal of the assembled E^T A E on every dof that each element reaches through at most one
    of its nodes, positive everywhere."""
    n, p = 2, 3
    V = perturbed_vertices(n, n, n, seed=7)
    S = VarSpace(n, n, n, [p] * n ** 3)
    I = np.rint(S.true_lattice_coords() * p).astype(np.int64)
    N = n * p + 1
    perm = I[:, 0] + N * (I[:, 1] + N * I[:, 2])
    prob = op.Problem(n, n, n, p, V)
    for kind in (DIFFUSION, MASS):
        np.testing.assert_allclose(S.jacobi_diagonal(V, kind), op.diagonal(prob, kind)[perm],
                                   rtol=1e-13, atol=0)
    nx, ny, nz = 3, 2, 2
    S = VarSpace(nx, ny, nz, block_orders(nx, ny, nz, block=1, orders=(1, 2, 4), seed=8))
    V = perturbed_vertices(nx, ny, nz, seed=3)
    E = S.prolongation().tocsc()
    single = np.ones(S.ntrue, dtype=bool)
    for i in range(S.ntrue):
        rows = E.indices[E.indptr[i]:E.indptr[i + 1]]
        elems = np.searchsorted(S.local_first, rows, side="right") - 1
        if np.unique(elems).size < elems.size:
            single[i] = False
    assert single.sum() > 0 and (~single).sum() > 0
    for kind in (DIFFUSION, MASS):
        d = S.jacobi_diagonal(V, kind)
        A = S.assemble(V, kind)
        assert np.all(d > 0)
        np.testing.assert_allclose(d[single], np.diag(A)[single], rtol=1e-12, atol=0)
