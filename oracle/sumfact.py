"""Sum-factorised partial-assembly apply on the CPU (oracle; test infrastructure).

A second route to the same operator, following the paper's structure: D is precomputed at the
quadrature points (partial assembly, Section II-B), and B, G are applied on the fly as three
successive 1D contractions per direction (Eq. (2); the three-GEMM split of Section III-D).
It is used to cross-check ``operator.apply`` (brute force on tiny meshes) and as the timed CPU
baseline; it shares nothing with the CUDA path.

Quadrature data (standard forms; the paper is silent on the H1 specifics):
  diffusion  D_q = w_q c_e adj(J) adj(J)^T / det J   (symmetric 3x3)
  mass       M_q = w_q c_e det J
"""
import numpy as np

from .quadrature import basis_1d
from .element import geometry, DIFFUSION, MASS
from .mesh import dof_map


def qdata(prob, kind, elems=None):
    """[ne, Q, Q, Q, 3, 3] (diffusion) or [ne, Q, Q, Q] (mass), axes (qz, qy, qx)."""
    _, _, _, wts, _ = basis_1d(prob.p, prob.q1d)
    Q = prob.q1d
    J, detJ = geometry(prob.vertices, prob.nx, prob.ny, prob.nz, Q, elems)
    ne = J.shape[0]
    w = np.einsum('z,y,x->zyx', wts, wts, wts).reshape(-1)
    if prob.coeff is None:
        c = np.ones(ne)
    else:
        c = prob.coeff if elems is None else prob.coeff[np.asarray(elems)]
    s = w[None, :] * c[:, None]
    if kind == MASS:
        return (s * detJ).reshape(ne, Q, Q, Q)
    adj = np.linalg.inv(J) * detJ[..., None, None]                  # adj(J) = det J * J^{-1}
    Dq = np.einsum('eqrk,eqsk->eqrs', adj, adj) * (s / detJ)[..., None, None]
    return Dq.reshape(ne, Q, Q, Q, 3, 3)


def apply(prob, x, kind, batch=1024):
    """y = G^T B^T D B G x with B applied by 1D contractions (dims of X: [e, k, j, i])."""
    B, G, _, _, _ = basis_1d(prob.p, prob.q1d)
    D = prob.p + 1
    x = np.asarray(x, dtype=np.float64)
    y = np.zeros(prob.ndofs)
    for s in range(0, prob.ne, batch):
        el = np.arange(s, min(prob.ne, s + batch))
        gm = dof_map(prob.nx, prob.ny, prob.nz, prob.p, el)
        X = x[gm].reshape(len(el), D, D, D)                          # [e, k, j, i]
        if kind == MASS:
            M = qdata(prob, MASS, el)
            U = np.einsum('xi,ekji->ekjx', B, X)
            U = np.einsum('yj,ekjx->ekyx', B, U)
            U = np.einsum('zk,ekyx->ezyx', B, U)
            V = M * U
            V = np.einsum('zk,ezyx->ekyx', B, V)
            V = np.einsum('yj,ekyx->ekjx', B, V)
            Y = np.einsum('xi,ekjx->ekji', B, V)
        elif kind == DIFFUSION:
            Dq = qdata(prob, DIFFUSION, el)
            # reference gradient (d/dxi, d/deta, d/dzeta) at the quadrature points
            T_g = np.einsum('xi,ekji->ekjx', G, X)
            T_b = np.einsum('xi,ekji->ekjx', B, X)
            u0 = np.einsum('zk,ekyx->ezyx', B, np.einsum('yj,ekjx->ekyx', B, T_g))
            u1 = np.einsum('zk,ekyx->ezyx', B, np.einsum('yj,ekjx->ekyx', G, T_b))
            u2 = np.einsum('zk,ekyx->ezyx', G, np.einsum('yj,ekjx->ekyx', B, T_b))
            u = np.stack([u0, u1, u2], axis=-1)
            v = np.einsum('ezyxrs,ezyxs->ezyxr', Dq, u)
            # transposes: Y = sum_r (d/dxi_r)^T v_r
            W0 = np.einsum('yj,ekyx->ekjx', B, np.einsum('zk,ezyx->ekyx', B, v[..., 0]))
            W1 = np.einsum('yj,ekyx->ekjx', G, np.einsum('zk,ezyx->ekyx', B, v[..., 1]))
            W2 = np.einsum('yj,ekyx->ekjx', B, np.einsum('zk,ezyx->ekyx', G, v[..., 2]))
            Y = np.einsum('xi,ekjx->ekji', G, W0) + np.einsum('xi,ekjx->ekji', B, W1 + W2)
        else:
            raise ValueError(kind)
        np.add.at(y, gm, Y.reshape(len(el), -1))
    return y
