"""The learned element-patch preconditioner around the network, flexible CG and the Adam update
(oracle; TEST INFRASTRUCTURE).

The paper has no learned component; these are the definitions the library's extension uses,
written out plainly in FP64 (the network itself is oracle/mlp.py):

* Patch operator.  For a residual r (a vector of the operator's dofs)

      M(r) = sum_e R_e^T W_e S_e s_e f(x_e / s_e),   x_e = S_e W_e R_e r,   s_e = ||x_e||_2,

  with R_e the restriction to element e's D^3 dofs (the dof map), W_e = diag(mult^-1/2) on e
  (mult = number of elements sharing the dof; 0 on the boundary), S = diag(A)^-1/2 (0 on the
  boundary) and f the network (oracle/mlp.py) with BF16 weights.  Elements with s_e = 0 add
  nothing.  With f_e(x) = S_e^+ A_ee^-1 S_e^+ x (S^+ the pseudo-inverse, A_ee = R_e A R_e^T) it
  is the symmetrically weighted additive Schwarz operator sum_e R_e^T W_e A_ee^-1 W_e R_e.
* Local-solve targets.  A training pair of element e is x = S_e v, t = S_e^-1 A_ee^-1 v for a
  vector v of the element's dofs (A_ee from the assembled matrix), i.e.
  t = S_e^-1 A_ee^-1 S_e^-1 x; the library stores pairs scaled to ||t|| = 1.
* Flexible CG with one stored direction (Notay's FCG(1)), for a possibly nonlinear
  preconditioner M: r0 = b - A x0, z = M(r), p = z; then q = A p, alpha = (p.r)/(p.q),
  x += alpha p, r -= alpha q, z = M(r), beta = -(z.q)/(p.q), p = z + beta p.  With a fixed
  symmetric positive definite M it produces the preconditioned CG iterates.
* Adam (Kingma and Ba): m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
  w -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps), t the step number from 1.
"""
import numpy as np

from . import mlp
from . import operator as oop
from .mesh import boundary_mask, dof_map

U_BF16 = 2.0 ** -9      # unit roundoff of round-to-nearest BF16 (8 significand bits)
U_FP32 = 2.0 ** -24


def bf16_round(a):
    """Round-to-nearest-even of values (first rounded to float32) to bfloat16, as float64."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def patch_data(prob, kind):
    """(dof map [ne, D^3] int64, S = diag(A)^-1/2 and W = mult^-1/2, both 0 on the boundary)."""
    dmap = dof_map(prob.nx, prob.ny, prob.nz, prob.p)
    mask = boundary_mask(prob.nx, prob.ny, prob.nz, prob.p)
    mult = np.bincount(dmap.reshape(-1), minlength=prob.ndofs).astype(np.float64)
    diag = oop.diagonal(prob, kind)
    S = np.where(mask == 1, 0.0, 1.0 / np.sqrt(np.where(mask == 1, 1.0, diag)))
    W = np.where(mask == 1, 0.0, 1.0 / np.sqrt(mult))
    return dmap, S, W


def patch_apply(prob, kind, f, r, bound=None):
    """M(r) for an element map f(Xn, elems) -> Y on rows Xn = x_e / s_e ([ne, D^3]).
    bound: optional map giving per-row error bounds of f (same shape, >= 0); the second
    return value is then the element-wise bound sum_e |R_e^T W_e S_e| s_e bound_e."""
    dmap, S, W = patch_data(prob, kind)
    r = np.asarray(r, dtype=np.float64)
    F = (S * W)[dmap]                       # [ne, D^3] the diagonal of S_e W_e per element
    X = F * r[dmap]
    s = np.linalg.norm(X, axis=1)
    live = s > 0
    elems = np.nonzero(live)[0]
    Xn = X[live] / s[live, None]
    z = np.zeros(prob.ndofs)
    Y = f(Xn, elems)
    np.add.at(z, dmap[live].reshape(-1), (F[live] * s[live, None] * Y).reshape(-1))
    if bound is None:
        return z
    zb = np.zeros(prob.ndofs)
    np.add.at(zb, dmap[live].reshape(-1), (np.abs(F[live]) * s[live, None] *
                                           bound(Xn, elems)).reshape(-1))
    return z, zb


def vspace_patch_apply(space, vertices, kind, nets, r, coeff=None, E=None, bounds=None,
                       mats=None):
    """M(r) on a variable-order space (oracle/varorder.VarSpace) with one network per order:

        M(r) = E^T F sum_e R_e^T s_e f_p(e)(x_e / s_e),   x_e = R_e F E r,   s_e = ||x_e||_2,

    in the local numbering X: a row of E with a single stored weight (a node that is a true
    dof's node) is that true dof's row, shared by every element that reaches it; every other row
    (a constrained node of one element) is its own row.  R_e picks element e's rows; F = (mult
    diag)^-1/2 per X row, mult = the number of element rows mapped to it and diag = the space's
    Jacobi diagonal diag(E^T blockdiag(diag A_e) E) at its true dof (space.jacobi_diagonal: the
    higher-order neighbours that read the dof through constrained nodes count too), F = 0 on the
    rows that carry no patch unknown: the boundary true dofs and every constrained row (the true
    dofs it interpolates are unknowns of the elements that own them; gathering E r there too
    would count their residual twice).
    r is taken zero and the
    result is zeroed on the boundary true dofs, so that M = (1-m) M (1-m); elements with s_e = 0
    add nothing.  With one order everywhere this is
    patch_apply's operator.  nets: {order: f(Xn, elems) -> Y}; E: the prolongation with the
    sparsity to use (default: the space's own); bounds: optional {order: bound map} (as in
    patch_apply), the second return value then bounds |M_computed - M| element-wise; mats: the
    element matrices (space.element_matrices), when already computed."""
    E = (space.prolongation() if E is None else E).tocsr()
    nloc, ntrue = E.shape
    mask = space.boundary_mask() == 1
    nnz_row = np.diff(E.indptr)
    xrow = np.empty(nloc, dtype=np.int64)
    unit = nnz_row == 1
    xrow[unit] = E.indices[E.indptr[:-1][unit]]
    own = np.nonzero(~unit)[0]
    xrow[own] = ntrue + np.arange(own.size)
    nX = ntrue + own.size
    maskX = np.ones(nX, dtype=bool)
    maskX[:ntrue] = mask
    if mats is None:
        mats = space.element_matrices(vertices, kind, coeff)
    dloc = np.concatenate([np.diag(K) for K in mats])    # element diagonals, local row order
    mult = np.bincount(xrow, minlength=nX).astype(np.float64)
    diag = np.zeros(nX)
    diag[:ntrue] = E.multiply(E).T @ dloc               # sum_i E_ij^2 (A_e)_ii
    live_rows = (~maskX) & (mult > 0) & (diag > 0)
    F = np.zeros(nX)
    F[live_rows] = 1.0 / np.sqrt(mult[live_rows] * diag[live_rows])
    Fl = F[xrow]                                   # the scaling of every element row
    r_free = np.where(mask, 0.0, np.asarray(r, dtype=np.float64))
    x_loc = Fl * (E @ r_free)
    y_loc = np.zeros(nloc)
    yb_loc = np.zeros(nloc)
    first = space.local_first
    for p in np.unique(space.order):
        el = np.nonzero(space.order == p)[0]
        D3 = (int(p) + 1) ** 3
        rows = (first[el][:, None] + np.arange(D3)[None, :])          # [ne_p, D^3]
        X = x_loc[rows]
        s = np.linalg.norm(X, axis=1)
        live = s > 0
        if not np.any(live):
            continue
        Xn = X[live] / s[live, None]
        Y = nets[int(p)](Xn, el[live])
        y_loc[rows[live].reshape(-1)] = (Fl[rows[live]] * s[live, None] * Y).reshape(-1)
        if bounds is not None:
            yb_loc[rows[live].reshape(-1)] = (np.abs(Fl[rows[live]]) * s[live, None] *
                                              bounds[int(p)](Xn, el[live])).reshape(-1)
    z = E.T @ y_loc
    z[mask] = 0.0
    if bounds is None:
        return z
    zb = abs(E).T @ yb_loc
    zb[mask] = 0.0
    return z, zb


def network(W):
    """The network f of the patch operator: oracle/mlp.py's forward pass in FP64 with the given
    (BF16) weights, the same for every element."""
    return lambda Xn, elems: mlp.forward(W, Xn)[0]


def network_rounding_bound(W, slack=1.5):
    """Element-wise bound on |f_bf16(x) - f(x)|, where f_bf16 rounds its input and hidden
    activations to BF16 (unit roundoff 2^-9) and accumulates in FP32 (length-n sums within
    n 2^-24 of the sum of absolute terms), as the BF16 tensor-core kernels do; first-order
    propagation through the layers (ReLU is 1-Lipschitz), times a slack factor."""
    W1, W2, W3, W0 = [np.abs(np.asarray(w, dtype=np.float64)) for w in mlp._weights(W)]

    def bound(Xn, elems):
        A = np.abs(Xn)
        din = A.shape[1]
        ea = (U_BF16 + 4 * U_FP32) * A                        # input scaled, narrowed, rounded
        y_abs = A @ W0
        ey = ea @ W0 + din * U_FP32 * y_abs
        if W1.size:
            h1 = np.abs(mlp.relu(Xn @ mlp._weights(W)[0]))
            e1 = ea @ W1 + U_BF16 * h1 + din * U_FP32 * (A @ W1)
            h2 = np.abs(mlp.relu(mlp.relu(Xn @ mlp._weights(W)[0]) @ mlp._weights(W)[1]))
            w = W1.shape[1]
            e2 = e1 @ W2 + U_BF16 * h2 + w * U_FP32 * ((h1 + e1) @ W2)
            ey = ey + e2 @ W3 + w * U_FP32 * ((h2 + e2) @ W3)
        return slack * ey
    return bound


def local_block(prob, kind, e, A=None):
    """A_ee = R_e A R_e^T: the assembled matrix on element e's dofs ([D^3, D^3], dense)."""
    A = oop.assemble(prob, kind) if A is None else A
    idx = dof_map(prob.nx, prob.ny, prob.nz, prob.p, [e])[0]
    return A[idx][:, idx].toarray()


def local_target(prob, kind, e, x, A=None, S=None):
    """t = S_e^-1 A_ee^-1 S_e^-1 x for an element whose dofs are all interior (S_e > 0)."""
    if S is None:
        _, S, _ = patch_data(prob, kind)
    idx = dof_map(prob.nx, prob.ny, prob.nz, prob.p, [e])[0]
    Se = S[idx]
    if np.any(Se <= 0):
        raise ValueError("element %d touches the boundary" % e)
    return np.linalg.solve(local_block(prob, kind, e, A), np.asarray(x) / Se) / Se


def additive_schwarz(prob, kind):
    """Dense sum_e R_e^T W_e A_ee^-1 W_e R_e, assembled element by element (the value of the
    patch operator with the exact local inverses)."""
    A = oop.assemble(prob, kind)
    dmap, _, W = patch_data(prob, kind)
    Mx = np.zeros((prob.ndofs, prob.ndofs))
    for e in range(prob.ne):
        idx = dmap[e]
        Ainv = np.linalg.inv(A[idx][:, idx].toarray())
        Mx[np.ix_(idx, idx)] += W[idx][:, None] * Ainv * W[idx][None, :]
    return Mx


def fcg(A, M, b, rtol=1e-10, maxit=10000, x0=None):
    """Notay's flexible CG with one stored direction.  A: callable or matrix, M: callable
    (possibly nonlinear).  Stops when ||r|| <= rtol ||b||.  Returns (x, iterations, history of
    ||r|| / ||b||, the iterates)."""
    Aop = A if callable(A) else (lambda v: A @ v)
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - Aop(x)
    nb = np.linalg.norm(b)
    hist, xs = [np.linalg.norm(r) / nb if nb > 0 else 0.0], [x.copy()]
    if nb == 0.0:
        return x, 0, hist, xs
    z = M(r)
    p = z.copy()
    it = 0
    while it < maxit:
        q = Aop(p)
        pq = p @ q
        alpha = (p @ r) / pq
        x = x + alpha * p
        r = r - alpha * q
        it += 1
        hist.append(np.linalg.norm(r) / nb)
        xs.append(x.copy())
        if hist[-1] <= rtol:
            break
        z = M(r)
        beta = -(z @ q) / pq
        p = z + beta * p
    return x, it, hist, xs


def adam_step(w, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update at step t (from 1): returns (w, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v
