"""Variable-order conforming H1 space on the structured hex mesh: the constraint operator P of
Eq. (1) under the minimum rule (oracle; TEST INFRASTRUCTURE, never imported by the library).

Eq. (1) writes the operator as ``A = P^T G^T B^T D B G P``; on one process with a single order
P is the identity.  With an order per element (Fig. 1's caption: P also carries constraints) the
global space must stay continuous, and the paper is silent on how.  Reading (minimum rule):

* every mesh entity (vertex, edge, face, cell) carries an order: a cell its element's order p_e,
  a face / edge the smallest order among the elements that contain it, a vertex none;
* the global ("true") dofs of an entity of order q are the values at the interior GLL_q nodes of
  the entity (vertex: 1 value, edge: q-1, face: (q-1)^2, cell: (q-1)^3);
* the function on an edge is the degree-q_e interpolant through its closure nodes (end vertices
  and its own dofs); on a face the Q_{q_f} interpolant through its (q_f+1)^2 closure nodes, whose
  boundary values are the bounding edges' functions there; on an element the Q_p interpolant
  through its (p+1)^3 GLL nodes, each node taking the value of the function of the entity whose
  relative interior holds it.  The traces then agree from both sides of every face and edge: the
  space is exactly the continuous piecewise-Q_{p_e} functions (a pin checks this dimension by
  brute force).

P = E maps true dofs to the E-vector (element-major, elements in index order e = ex + nx*(ey +
ny*ez), local node a = i + D*(j + D*k)); ``apply`` is y = E^T blockdiag(A_e) E x.

Numbering of the true dofs (the library's is the same and is documented with its entry points):
vertices lexicographic on the (nx+1)(ny+1)(nz+1) lattice; then the x-, y- and z-directed edges,
each family lexicographic on its own index box (x fastest), q_e - 1 dofs per edge in increasing
coordinate; then the x-, y- and z-normal faces likewise, (q_f - 1)^2 dofs per face with the
face's first in-plane axis fastest (x-normal: y, z; y-normal: x, z; z-normal: x, y); then the
cells, (p - 1)^3 dofs each, x fastest.  Edges and faces are parametrised along the global axes,
which every element of the structured mesh shares, so no orientation flips arise.
"""
import numpy as np
import scipy.sparse as sp

from .element import element_matrices
from .quadrature import gauss_lobatto, lagrange

BIG = 1 << 20


def _lagrange_at(nodes, x):
    """Lagrange basis of ``nodes`` at the single point x (the product formula; where x coincides
    with a node only up to the last bit -- GLL nodes of different orders meet at 0, 1/2 and 1 --
    the values differ from 0 and 1 by rounding)."""
    return lagrange(np.asarray(nodes, dtype=np.float64), [x])[0][0]


class VarSpace:
    """Minimum-rule variable-order H1 space of an nx x ny x nz structured hex mesh; ``order`` holds
    one order (1..8) per element, element index ex + nx*(ey + ny*ez)."""

    def __init__(self, nx, ny, nz, order):
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.order = np.asarray(order, dtype=np.int64).reshape(-1)
        if self.order.size != nx * ny * nz:
            raise ValueError("one order per element")
        if self.order.min() < 1 or self.order.max() > 8:
            raise ValueError("orders must be 1..8")
        self.ne = self.order.size
        P = self.order.reshape(nz, ny, nx)
        Pp = np.full((nz + 2, ny + 2, nx + 2), BIG, dtype=np.int64)
        Pp[1:-1, 1:-1, 1:-1] = P

        def win(z0, z1, y0, y1, x0, x1):
            return Pp[z0:Pp.shape[0] - z1, y0:Pp.shape[1] - y1, x0:Pp.shape[2] - x1]

        # entity orders: min over the elements that contain the entity (out-of-mesh cells = BIG)
        # x-edge (ix, iy, iz): cells (ix, iy-1|iy, iz-1|iz)      shape (nz+1, ny+1, nx)
        ex = np.minimum.reduce([win(c, 1 - c, b, 1 - b, 1, 1) for b in (0, 1) for c in (0, 1)])
        # y-edge (ix, iy, iz): cells (ix-1|ix, iy, iz-1|iz)      shape (nz+1, ny, nx+1)
        ey = np.minimum.reduce([win(c, 1 - c, 1, 1, a, 1 - a) for a in (0, 1) for c in (0, 1)])
        # z-edge (ix, iy, iz): cells (ix-1|ix, iy-1|iy, iz)      shape (nz, ny+1, nx+1)
        ez = np.minimum.reduce([win(1, 1, b, 1 - b, a, 1 - a) for a in (0, 1) for b in (0, 1)])
        # x-face (ix, iy, iz): cells (ix-1|ix, iy, iz)           shape (nz, ny, nx+1)
        fx = np.minimum.reduce([win(1, 1, 1, 1, a, 1 - a) for a in (0, 1)])
        fy = np.minimum.reduce([win(1, 1, b, 1 - b, 1, 1) for b in (0, 1)])
        fz = np.minimum.reduce([win(c, 1 - c, 1, 1, 1, 1) for c in (0, 1)])
        self.edge_order = [ex, ey, ez]
        self.face_order = [fx, fy, fz]
        for arr in self.edge_order + self.face_order:
            assert arr.max() < BIG

        nv = (nx + 1) * (ny + 1) * (nz + 1)
        self.nv = nv
        off = nv
        self.edge_first = []   # first true dof of every edge, per direction, [box shape]
        for q in self.edge_order:
            cnt = (q - 1).reshape(-1)
            first = off + np.concatenate([[0], np.cumsum(cnt)[:-1]])
            self.edge_first.append(first.reshape(q.shape))
            off += int(cnt.sum())
        self.face_first = []
        for q in self.face_order:
            cnt = ((q - 1) ** 2).reshape(-1)
            first = off + np.concatenate([[0], np.cumsum(cnt)[:-1]])
            self.face_first.append(first.reshape(q.shape))
            off += int(cnt.sum())
        cnt = (self.order - 1) ** 3
        self.cell_first = off + np.concatenate([[0], np.cumsum(cnt)[:-1]])
        off += int(cnt.sum())
        self.ntrue = off
        self.local_size = (self.order + 1) ** 3
        self.local_first = np.concatenate([[0], np.cumsum(self.local_size)[:-1]])
        self.nlocal = int(self.local_size.sum())

    # -- entity closures: sparse rows (dict col -> weight) of the closure nodes' values --------

    def _vertex(self, ix, iy, iz):
        return {ix + (self.nx + 1) * (iy + (self.ny + 1) * iz): 1.0}

    def _edge_closure(self, d, ix, iy, iz):
        """(q, rows): the q+1 closure node values of the d-directed edge at (ix, iy, iz)."""
        q = int(self.edge_order[d][iz, iy, ix])
        first = int(self.edge_first[d][iz, iy, ix])
        lo = [ix, iy, iz]
        hi = [ix, iy, iz]
        hi[d] += 1
        rows = [self._vertex(*lo)] + [{first + m - 1: 1.0} for m in range(1, q)] + \
               [self._vertex(*hi)]
        return q, rows

    def _face_closure(self, d, ix, iy, iz):
        """(q, rows): the (q+1)^2 closure node values of the d-normal face at (ix, iy, iz),
        first in-plane axis fastest."""
        q = int(self.face_order[d][iz, iy, ix])
        first = int(self.face_first[d][iz, iy, ix])
        u, v = [a for a in range(3) if a != d]          # in-plane axes, u fastest
        t = gauss_lobatto(q + 1)
        rows = [None] * ((q + 1) ** 2)
        for n in range(q + 1):
            for m in range(q + 1):
                if 0 < m < q and 0 < n < q:
                    rows[m + (q + 1) * n] = {first + (m - 1) + (q - 1) * (n - 1): 1.0}
                    continue
                # on the boundary: the function of a bounding edge (a corner lies on two; either)
                base = [ix, iy, iz]
                if m in (0, q):
                    base[u] += (m == q)
                    ed, coord = v, t[n]                 # edge runs along v
                else:
                    base[v] += (n == q)
                    ed, coord = u, t[m]                 # edge runs along u
                qe, erows = self._edge_closure(ed, *base)
                rows[m + (q + 1) * n] = _combine(_lagrange_at(gauss_lobatto(qe + 1), coord),
                                                 erows)
        return q, rows

    def prolongation(self):
        """E = G P as a scipy CSR matrix [nlocal, ntrue] (the element values of every true-dof
        vector); rows element-major, node a = i + D*(j + D*k)."""
        data, ri, ci = [], [], []
        for e in range(self.ne):
            p = int(self.order[e])
            D = p + 1
            ex, ey, ez = e % self.nx, (e // self.nx) % self.ny, e // (self.nx * self.ny)
            tp = gauss_lobatto(D)
            faces, edges = {}, {}
            for a in range(D ** 3):
                ijk = (a % D, (a // D) % D, a // (D * D))
                fixed = [c in (0, p) for c in ijk]
                pos = [ex + (ijk[0] == p), ey + (ijk[1] == p), ez + (ijk[2] == p)]
                cell = [ex, ey, ez]
                nb = sum(fixed)
                if nb == 3:
                    row = self._vertex(*pos)
                elif nb == 0:
                    i, j, k = ijk
                    row = {int(self.cell_first[e]) + (i - 1) + (p - 1) * ((j - 1) + (p - 1) * (k - 1)): 1.0}
                elif nb == 2:
                    d = fixed.index(False)
                    key = list(pos)
                    key[d] = cell[d]
                    key = (d, *key)
                    if key not in edges:
                        edges[key] = self._edge_closure(*key)
                    qe, erows = edges[key]
                    row = _combine(_lagrange_at(gauss_lobatto(qe + 1), tp[ijk[d]]), erows)
                else:
                    d = fixed.index(True)
                    key = list(cell)
                    key[d] = pos[d]
                    key = (d, *key)
                    if key not in faces:
                        faces[key] = self._face_closure(*key)
                    qf, frows = faces[key]
                    u, v = [x for x in range(3) if x != d]
                    tq = gauss_lobatto(qf + 1)
                    Lu = _lagrange_at(tq, tp[ijk[u]])
                    Lv = _lagrange_at(tq, tp[ijk[v]])
                    w = np.outer(Lv, Lu).reshape(-1)            # index m + (q+1) n
                    row = _combine(w, frows)
                r = int(self.local_first[e]) + a
                for c, val in row.items():
                    if val != 0.0:
                        ri.append(r)
                        ci.append(c)
                        data.append(val)
        return sp.csr_matrix((data, (ri, ci)), shape=(self.nlocal, self.ntrue))

    def true_lattice_coords(self):
        """Lattice coordinates [ntrue, 3] of the true dofs (element (ex, ey, ez) spans
        [ex, ex+1] x [ey, ey+1] x [ez, ez+1]; a node sits at its GLL point)."""
        X = np.zeros((self.ntrue, 3))
        nx, ny, nz = self.nx, self.ny, self.nz
        v = np.arange(self.nv)
        X[:self.nv] = np.stack([v % (nx + 1), (v // (nx + 1)) % (ny + 1),
                                v // ((nx + 1) * (ny + 1))], axis=1)
        for d in range(3):
            q = self.edge_order[d]
            for (iz, iy, ix), qe in np.ndenumerate(q):
                t = gauss_lobatto(qe + 1)
                for m in range(1, qe):
                    pt = np.array([ix, iy, iz], dtype=np.float64)
                    pt[d] += t[m]
                    X[self.edge_first[d][iz, iy, ix] + m - 1] = pt
            q = self.face_order[d]
            u, w = [a for a in range(3) if a != d]
            for (iz, iy, ix), qf in np.ndenumerate(q):
                t = gauss_lobatto(qf + 1)
                for n in range(1, qf):
                    for m in range(1, qf):
                        pt = np.array([ix, iy, iz], dtype=np.float64)
                        pt[u] += t[m]
                        pt[w] += t[n]
                        X[self.face_first[d][iz, iy, ix] + (m - 1) + (qf - 1) * (n - 1)] = pt
        for e in range(self.ne):
            p = int(self.order[e])
            t = gauss_lobatto(p + 1)
            ex, ey, ez = e % nx, (e // nx) % ny, e // (nx * ny)
            for k in range(1, p):
                for j in range(1, p):
                    for i in range(1, p):
                        X[self.cell_first[e] + (i - 1) + (p - 1) * ((j - 1) + (p - 1) * (k - 1))] = \
                            (ex + t[i], ey + t[j], ez + t[k])
        return X

    def boundary_mask(self):
        """1 for true dofs on the boundary of the domain (the Dirichlet set)."""
        X = self.true_lattice_coords()
        n = np.array([self.nx, self.ny, self.nz], dtype=np.float64)
        return (np.any(X == 0.0, axis=1) | np.any(X == n[None, :], axis=1)).astype(np.uint8)

    def element_matrices(self, vertices, kind, coeff=None):
        """List of dense element matrices [D_e^3, D_e^3] (element index order), each element at
        its own order with a p_e + 2 point Gauss rule."""
        mats = [None] * self.ne
        for p in np.unique(self.order):
            el = np.nonzero(self.order == p)[0]
            K = element_matrices(vertices, self.nx, self.ny, self.nz, int(p), int(p) + 2,
                                 coeff, kind, el)
            for t, e in enumerate(el):
                mats[e] = K[t]
        return mats

    def apply(self, vertices, x, kind, coeff=None, E=None):
        """y = E^T blockdiag(A_e) E x: Eq. (1) with the constraint operator P."""
        E = self.prolongation() if E is None else E
        u = E @ np.asarray(x, dtype=np.float64)
        v = np.zeros_like(u)
        for e, K in enumerate(self.element_matrices(vertices, kind, coeff)):
            s = int(self.local_first[e])
            n = K.shape[0]
            v[s:s + n] = K @ u[s:s + n]
        return E.T @ v

    def jacobi_diagonal(self, vertices, kind, coeff=None, E=None):
        """diag(E^T blockdiag(diag A_e) E) = sum_e sum_a E[a, i]^2 A_e[a, a]: the Jacobi diagonal
        of the variable-order operator (exact wherever no element reaches a dof through two of its
        nodes)."""
        E = self.prolongation() if E is None else E
        dloc = np.concatenate([np.diag(K) for K in self.element_matrices(vertices, kind, coeff)])
        return E.multiply(E).T @ dloc

    def assemble(self, vertices, kind, coeff=None, sparse=False, E=None):
        """E^T blockdiag(A_e) E: dense (tiny meshes), or a scipy CSR matrix with sparse=True."""
        E = self.prolongation() if E is None else E
        blocks = self.element_matrices(vertices, kind, coeff)
        A = sp.block_diag([sp.csr_matrix(b) for b in blocks], format="csr")
        K = (E.T @ A @ E).tocsr()
        return K if sparse else K.toarray()


def _combine(weights, rows):
    """sum_m weights[m] * rows[m] for sparse rows given as dicts."""
    out = {}
    for w, r in zip(weights, rows):
        if w == 0.0:
            continue
        for c, val in r.items():
            out[c] = out.get(c, 0.0) + w * val
    return out
