"""Structured hexahedral mesh topology: the element restriction G of Eq. (1) (oracle).

Fig. 1 / Eq. (1): G maps the rank-local dof vector (L-vector) to element dofs (E-vector); G^T is
the scatter-add back.  On one process P is the identity, so the L-vector is the global vector.

Readings (the paper is silent on the numbering):
* elements e = ex + nx*(ey + ny*ez), x fastest;
* element-local dofs a = i + D*(j + D*k), D = p + 1, x fastest;
* global dofs lexicographic on the (nx*p+1) x (ny*p+1) x (nz*p+1) point lattice, x fastest, so
  element (ex, ey, ez), local (i, j, k) -> (ex*p+i) + Nx*((ey*p+j) + Ny*(ez*p+k));
* mesh vertices lexicographic on the (nx+1) x (ny+1) x (nz+1) lattice, x fastest, and the eight
  element corners ordered v = a + 2b + 4c for the corner at offset (a, b, c).
"""
import numpy as np


def n_points(n, p):
    return n * p + 1


def ndofs(nx, ny, nz, p):
    return n_points(nx, p) * n_points(ny, p) * n_points(nz, p)


def _elem_coords(nx, ny, nz, elems):
    ne = nx * ny * nz
    e = np.arange(ne, dtype=np.int64) if elems is None else np.asarray(elems, dtype=np.int64)
    return e % nx, (e // nx) % ny, e // (nx * ny)


def _local_ijk(D):
    """(i, j, k) of every local index a = i + D*(j + D*k), in order of a."""
    a = np.arange(D ** 3)
    return a % D, (a // D) % D, a // (D * D)


def dof_map(nx, ny, nz, p, elems=None):
    """Element dof map ``map[e, a]`` (int64, [ne, D^3]): the index gather of G.
    ``elems`` restricts the result to the listed elements (rows in that order)."""
    D = p + 1
    Nx, Ny = n_points(nx, p), n_points(ny, p)
    ex, ey, ez = _elem_coords(nx, ny, nz, elems)
    i, j, k = _local_ijk(D)
    return ((ex[:, None] * p + i[None, :])
            + Nx * ((ey[:, None] * p + j[None, :]) + Ny * (ez[:, None] * p + k[None, :])))


def element_vertices(vertices, nx, ny, nz, elems=None):
    """Corner coordinates [ne, 8, 3] of the (listed) elements from the vertex array
    [(nx+1)(ny+1)(nz+1), 3]; corner v = a + 2b + 4c sits at lattice offset (a, b, c)."""
    V = np.asarray(vertices, dtype=np.float64).reshape(-1, 3)
    if V.shape[0] != (nx + 1) * (ny + 1) * (nz + 1):
        raise ValueError("vertex array does not match the mesh size")
    ex, ey, ez = _elem_coords(nx, ny, nz, elems)
    v = np.arange(8)
    a, b, c = v % 2, (v // 2) % 2, v // 4
    idx = (ex[:, None] + a) + (nx + 1) * ((ey[:, None] + b) + (ny + 1) * (ez[:, None] + c))
    return V[idx]


def boundary_mask(nx, ny, nz, p):
    """1 for dofs on the boundary of the lattice (the Dirichlet set), 0 elsewhere."""
    Nx, Ny, Nz = n_points(nx, p), n_points(ny, p), n_points(nz, p)
    m = np.zeros((Nz, Ny, Nx), dtype=np.uint8)
    m[0, :, :] = m[-1, :, :] = 1
    m[:, 0, :] = m[:, -1, :] = 1
    m[:, :, 0] = m[:, :, -1] = 1
    return m.reshape(-1)


def trilinear(Xe, xi):
    """Physical points and Jacobians of trilinear hexes at reference points.

    x(xi) = sum_v X_v N_v(xi) with N_v the product over the three axes of (1 - t) or t.
    Xe: [ne, 8, 3] corners; xi: [nq, 3] in [0, 1]^3.  Returns (x [ne, nq, 3],
    J [ne, nq, 3, 3]) with J[..., i, r] = d x_i / d xi_r.
    """
    Xe = np.asarray(Xe, dtype=np.float64)
    xi = np.atleast_2d(np.asarray(xi, dtype=np.float64))
    N = np.empty((xi.shape[0], 8))
    dN = np.empty((xi.shape[0], 8, 3))
    for v in range(8):
        a, b, c = v % 2, (v // 2) % 2, v // 4
        fa = xi[:, 0] if a else 1.0 - xi[:, 0]
        fb = xi[:, 1] if b else 1.0 - xi[:, 1]
        fc = xi[:, 2] if c else 1.0 - xi[:, 2]
        da, db, dc = (1.0 if a else -1.0), (1.0 if b else -1.0), (1.0 if c else -1.0)
        N[:, v] = fa * fb * fc
        dN[:, v, 0] = da * fb * fc
        dN[:, v, 1] = fa * db * fc
        dN[:, v, 2] = fa * fb * dc
    x = np.einsum('qv,evi->eqi', N, Xe)
    J = np.einsum('qvr,evi->eqir', dN, Xe)
    return x, J


def dof_coordinates(vertices, nx, ny, nz, p):
    """Physical coordinates [ndof, 3] of every nodal (GLL) dof: the trilinear image of the
    reference GLL lattice of an element that owns it."""
    from .quadrature import gauss_lobatto
    D = p + 1
    t = gauss_lobatto(D)
    i, j, k = _local_ijk(D)
    ref = np.stack([t[i], t[j], t[k]], axis=1)
    x, _ = trilinear(element_vertices(vertices, nx, ny, nz), ref)
    out = np.zeros((ndofs(nx, ny, nz, p), 3))
    out[dof_map(nx, ny, nz, p)] = x
    return out
