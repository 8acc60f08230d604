"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module holds no arithmetic of the method: it only draws the mesh vertices, vectors and
coefficients that both the CUDA path and the CPU oracle receive as data.

* ``perturbed_vertices``: the regular (nx+1) x (ny+1) x (nz+1) vertex lattice of the unit cube,
  x fastest, with every vertex not on the cube's boundary moved by h * U[-amp, amp] in each
  coordinate independently (h = 1/n along that axis), so the domain stays the unit cube;
* ``uniform_vector``: x ~ U[-1, 1];
* ``lognormal_coefficient``: one value per element, exp(sigma * Z), Z ~ N(0, 1);
* ``block_orders``: one polynomial order per element, constant on block^3-element blocks, each
  block's order drawn uniformly from a set.

Generators are ``numpy.random.default_rng(seed)`` (PCG64), so every input is reproducible.
"""
import numpy as np

MESH_SEED = 1234
COEFF_SEED = 42


def perturbed_vertices(nx, ny, nz, seed=MESH_SEED, amp=0.1):
    xs = np.linspace(0.0, 1.0, nx + 1)
    ys = np.linspace(0.0, 1.0, ny + 1)
    zs = np.linspace(0.0, 1.0, nz + 1)
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    V = np.stack([X.reshape(-1), Y.reshape(-1), Z.reshape(-1)], axis=1)
    if amp:
        rng = np.random.default_rng(seed)
        h = np.array([1.0 / nx, 1.0 / ny, 1.0 / nz])
        d = rng.uniform(-amp, amp, size=V.shape) * h[None, :]
        ix = np.arange((nx + 1) * (ny + 1) * (nz + 1))
        i, j, k = ix % (nx + 1), (ix // (nx + 1)) % (ny + 1), ix // ((nx + 1) * (ny + 1))
        interior = (i > 0) & (i < nx) & (j > 0) & (j < ny) & (k > 0) & (k < nz)
        V[interior] += d[interior]
    return np.ascontiguousarray(V)


def uniform_vector(n, seed):
    return np.random.default_rng(seed).uniform(-1.0, 1.0, size=int(n))


def lognormal_coefficient(ne, sigma=1.0, seed=COEFF_SEED):
    return np.exp(sigma * np.random.default_rng(seed).standard_normal(int(ne)))


# Elements per axis of the ~50 M dof order-sweep meshes (n^3 hexes, (n*p+1)^3 dofs).
ORDER_SWEEP_N = {1: 368, 2: 184, 3: 123, 4: 92, 5: 74, 6: 61, 7: 53, 8: 46}


def block_orders(nx, ny, nz, block=8, orders=(2, 4, 6), seed=7):
    """One polynomial order per element (index ex + nx*(ey + ny*ez)): the mesh is cut into
    block^3-element blocks (ragged at the far ends) and each block draws its order uniformly from
    ``orders``."""
    bx, by, bz = -(-nx // block), -(-ny // block), -(-nz // block)
    pick = np.random.default_rng(seed).integers(0, len(orders), size=bx * by * bz)
    o = np.asarray(orders, dtype=np.int32)[pick].reshape(bz, by, bx)
    ez, ey, ex = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return np.ascontiguousarray(o[ez // block, ey // block, ex // block].reshape(-1))
