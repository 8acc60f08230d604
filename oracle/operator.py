"""Operator action, rows, diagonal and assembled matrix from element matrices (oracle).

``apply`` is the plain definition of Eq. (1) on one process (P = identity):
y = G^T (blockdiag_e K_e) G x = sum_e G_e^T K_e G_e x, with the element matrices of
``element.py``.  Accumulation order is fixed (elements in index order).
"""
import numpy as np

from .element import element_matrices, DIFFUSION, MASS  # noqa: F401
from .mesh import dof_map, ndofs, n_points


class Problem:
    """The inputs that define one operator: mesh size, vertices, order, rule and coefficient."""

    def __init__(self, nx, ny, nz, p, vertices, q1d=None, coeff=None):
        self.nx, self.ny, self.nz, self.p = int(nx), int(ny), int(nz), int(p)
        self.q1d = int(q1d) if q1d else self.p + 2
        self.vertices = np.asarray(vertices, dtype=np.float64).reshape(-1, 3)
        self.coeff = None if coeff is None else np.asarray(coeff, dtype=np.float64)
        self.ne = self.nx * self.ny * self.nz
        self.ndofs = ndofs(self.nx, self.ny, self.nz, self.p)

    def elem_mats(self, kind, elems=None):
        return element_matrices(self.vertices, self.nx, self.ny, self.nz, self.p, self.q1d,
                                self.coeff, kind, elems)

    def dof_map(self, elems=None):
        return dof_map(self.nx, self.ny, self.nz, self.p, elems)


def _batches(ne, batch):
    for s in range(0, ne, batch):
        yield np.arange(s, min(ne, s + batch))


def apply(prob, x, kind, batch=256):
    """y = sum_e G_e^T K_e G_e x for the whole vector x [ndofs]."""
    x = np.asarray(x, dtype=np.float64)
    y = np.zeros(prob.ndofs)
    for el in _batches(prob.ne, batch):
        K = prob.elem_mats(kind, el)
        gm = prob.dof_map(el)
        ye = np.einsum('eab,eb->ea', K, x[gm])
        np.add.at(y, gm, ye)
    return y


def elements_of_dof(prob, g):
    """Indices of the elements whose closure holds global dof g (1 to 8 of them)."""
    p = prob.p
    Nx, Ny = n_points(prob.nx, p), n_points(prob.ny, p)
    ix, iy, iz = g % Nx, (g // Nx) % Ny, g // (Nx * Ny)

    def cands(i, n):
        return [e for e in {(i - 1) // p, i // p} if 0 <= e < n and e * p <= i <= e * p + p]

    out = [ex + prob.nx * (ey + prob.ny * ez)
           for ez in cands(iz, prob.nz) for ey in cands(iy, prob.ny) for ex in cands(ix, prob.nx)]
    return sorted(out)


def apply_rows(prob, x, kind, rows):
    """Selected entries y[rows] of y = A x, each summed over the few elements that hold the dof
    (used to check a full-size apply one output at a time)."""
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros(len(rows))
    for n, g in enumerate(rows):
        els = np.array(elements_of_dof(prob, int(g)))
        K = prob.elem_mats(kind, els)
        gm = prob.dof_map(els)
        for t in range(len(els)):
            (a,) = np.nonzero(gm[t] == g)[0]
            out[n] += K[t, a, :] @ x[gm[t]]
    return out


def diagonal(prob, kind, batch=256):
    """diag(A) = sum_e G_e^T diag(K_e)."""
    d = np.zeros(prob.ndofs)
    for el in _batches(prob.ne, batch):
        K = prob.elem_mats(kind, el)
        np.add.at(d, prob.dof_map(el), np.einsum('eaa->ea', K))
    return d


def assemble(prob, kind):
    """Assembled global matrix as a scipy CSR matrix (tiny meshes)."""
    import scipy.sparse as sp
    K = prob.elem_mats(kind)
    gm = prob.dof_map()
    D3 = gm.shape[1]
    rows = np.repeat(gm, D3, axis=1).reshape(-1)
    cols = np.tile(gm, (1, D3)).reshape(-1)
    return sp.coo_matrix((K.reshape(-1), (rows, cols)), shape=(prob.ndofs, prob.ndofs)).tocsr()


def constrained(apply_fn, mask):
    """Essential-BC operator A_bc x = (1 - m) * A((1 - m) * x) + m * x (identity rows and
    columns on the Dirichlet set m); standard treatment, the paper is silent."""
    keep = 1.0 - np.asarray(mask, dtype=np.float64)

    def A_bc(x):
        return keep * apply_fn(keep * x) + (1.0 - keep) * x
    return A_bc
