"""GPU parity of the paper's mixed H1 / L2 gradient and divergence pair (fe_mixed_apply through the
C ABI) against oracle/mixed.py's element matrices built by direct quadrature.

Small perturbed meshes whose element counts leave a ragged last thread block, every built
order pair, both blocks in one fused launch and each block alone: every output compared, relative
max-norm error <= 1e-12.  The benchmark's size (128^3 hexes, H1 order 4 / L2 order 3, 538 M
values): outputs of sampled elements (gradient) and sampled H1 dofs (divergence), each computed
by the oracle from the element matrices of the elements involved, plus adjointness
u . (G p) = p . (G^T u) at full size.
"""
import numpy as np
import pytest

from gpu_util import lib, torch_cuda, TOL
from oracle.mixed import MixedProblem, element_gradient_matrices
from oracle.mesh import dof_map
from paper_2603_09038_gb300.inputs import perturbed_vertices, uniform_vector

pytestmark = pytest.mark.gpu

PAIRS = [(4, 3), (2, 1), (3, 3)]


def _setup(dims, ph, pl, seed=1234):
    fe = lib()
    V = perturbed_vertices(*dims, seed=seed)
    mx = fe.fe_mixed_setup(*dims, ph, pl, V)
    return fe, mx, V


@pytest.mark.parametrize("ph,pl", PAIRS)
@pytest.mark.parametrize("dims", [(3, 2, 2), (2, 3, 4), (5, 4, 3), (1, 1, 1)])
def test_fused_pair_matches_oracle(dims, ph, pl):
    torch = torch_cuda()
    fe, mx, V = _setup(dims, ph, pl)
    try:
        nh, nl = fe.fe_mixed_sizes(mx)
        M = MixedProblem(*dims, V, ph, pl)
        assert (nh, nl) == (M.ndof_h, M.ndof_l)
        ph_ = uniform_vector(nh, seed=3)
        ul_ = uniform_vector(nl, seed=4)
        p = torch.from_numpy(ph_).cuda()
        u = torch.from_numpy(ul_).cuda()
        gp = torch.full((nl,), float("nan"), dtype=torch.float64, device="cuda")
        gtu = torch.full((nh,), float("nan"), dtype=torch.float64, device="cuda")
        ref_g, ref_d = M.gradient(ph_), M.divergence(ul_)
        fe.fe_mixed_apply(mx, p, u, gp, gtu)             # both blocks, one launch
        torch.cuda.synchronize()
        for got, ref in ((gp, ref_g), (gtu, ref_d)):
            g = got.cpu().numpy()
            assert np.abs(g - ref).max() <= TOL * np.abs(ref).max()
        gp2 = torch.full_like(gp, float("nan"))
        gtu2 = torch.full_like(gtu, float("nan"))
        fe.fe_mixed_apply(mx, p, None, gp2, None)        # each block alone
        fe.fe_mixed_apply(mx, None, u, None, gtu2)
        torch.cuda.synchronize()
        assert np.abs(gp2.cpu().numpy() - ref_g).max() <= TOL * np.abs(ref_g).max()
        assert np.abs(gtu2.cpu().numpy() - ref_d).max() <= TOL * np.abs(ref_d).max()
    finally:
        fe.fe_mixed_destroy(mx)


def test_constants_and_linear_pressures():
    """G 1 = 0 (constants have no gradient); for p = alpha . x the element sums of G p give
    alpha times the element volumes, alpha in total on the unit cube."""
    torch = torch_cuda()
    from oracle.mesh import dof_coordinates
    dims = (4, 3, 3)
    fe, mx, V = _setup(dims, 4, 3, seed=9)
    try:
        nh, nl = fe.fe_mixed_sizes(mx)
        gp = torch.empty(nl, dtype=torch.float64, device="cuda")
        fe.fe_mixed_apply(mx, torch.ones(nh, dtype=torch.float64, device="cuda"), None, gp, None)
        torch.cuda.synchronize()
        assert float(gp.abs().max()) <= 1e-14
        X = dof_coordinates(V, *dims, 4)
        alpha = np.array([0.7, -1.3, 2.1])
        fe.fe_mixed_apply(mx, torch.from_numpy(X @ alpha).cuda(), None, gp, None)
        torch.cuda.synchronize()
        tot = gp.cpu().numpy().reshape(-1, 3, 64).sum(axis=(0, 2))
        assert np.abs(tot - alpha).max() <= 1e-13
    finally:
        fe.fe_mixed_destroy(mx)


def test_errors():
    fe = lib()
    V = perturbed_vertices(2, 2, 2)
    with pytest.raises(fe.FEError) as e:
        fe.fe_mixed_setup(2, 2, 2, 5, 3, V)
    assert e.value.status == fe.FE_ERR_UNSUPPORTED
    bad = V.copy().reshape(-1, 3)
    bad[0], bad[1] = bad[1].copy(), bad[0].copy()        # swap two corners: inverted element
    with pytest.raises(fe.FEError) as e:
        fe.fe_mixed_setup(2, 2, 2, 4, 3, bad)
    assert e.value.status == fe.FE_ERR_ARG


def test_full_size_sampled_and_adjoint():
    """128^3 hexes (the size of the benchmark's mixed workload): 24 sampled elements' gradient
    values and 24 sampled H1 dofs' divergence values against the oracle, and adjointness."""
    torch = torch_cuda()
    n, ph, pl = 128, 4, 3
    fe, mx, V = _setup((n, n, n), ph, pl)
    try:
        nh, nl = fe.fe_mixed_sizes(mx)
        g = torch.Generator(device="cuda").manual_seed(2)
        p = torch.rand(nh, dtype=torch.float64, device="cuda", generator=g) * 2 - 1
        u = torch.rand(nl, dtype=torch.float64, device="cuda", generator=g) * 2 - 1
        gp = torch.empty(nl, dtype=torch.float64, device="cuda")
        gtu = torch.empty(nh, dtype=torch.float64, device="cuda")
        fe.fe_mixed_apply(mx, p, u, gp, gtu)
        torch.cuda.synchronize()
        # adjointness at full size (FP64 sums of 5e8 terms: relative 1e-12 of the absolute sums)
        lhs = float(torch.dot(u, gp))
        rhs = float(torch.dot(p, gtu))
        scale = float(torch.dot(u.abs(), gp.abs()))
        assert abs(lhs - rhs) <= 1e-11 * scale
        rng = np.random.default_rng(5)
        Dh, Dl = ph + 1, pl + 1
        ne = n ** 3
        elems = np.unique(np.concatenate([rng.choice(ne, 22, replace=False), [0, ne - 1]]))
        Ge = element_gradient_matrices(V, n, n, n, ph, pl, elems=elems)    # [s, 3, Dl^3, Dh^3]
        gm = dof_map(n, n, n, ph, elems)
        ph_s = p.cpu().numpy()[gm]                                          # [s, Dh^3]
        ref = np.einsum('ecab,eb->eca', Ge, ph_s).reshape(len(elems), -1)
        got = gp.view(ne, 3 * Dl ** 3)[torch.from_numpy(elems).cuda()].cpu().numpy()
        scale_g = float(gp.abs().max())
        assert np.abs(got - ref).max() <= TOL * scale_g
        # divergence at sampled H1 dofs: the sum over the elements containing each dof
        N = n * ph + 1
        un = u.cpu().numpy().reshape(ne, 3, Dl ** 3)
        scale_d = float(gtu.abs().max())
        gtu_h = gtu.cpu().numpy()
        for I, J, K in rng.integers(0, N, size=(24, 3)):
            gid = I + N * (J + N * K)
            exs = [e for e in {I // ph, (I - 1) // ph} if 0 <= e < n]
            eys = [e for e in {J // ph, (J - 1) // ph} if 0 <= e < n]
            ezs = [e for e in {K // ph, (K - 1) // ph} if 0 <= e < n]
            tot = 0.0
            for ez in ezs:
                for ey in eys:
                    for ex in exs:
                        e = ex + n * (ey + n * ez)
                        b = (I - ex * ph) + Dh * ((J - ey * ph) + Dh * (K - ez * ph))
                        Ge1 = element_gradient_matrices(V, n, n, n, ph, pl, elems=[e])[0]
                        tot += np.einsum('ca,ca->', Ge1[:, :, b], un[e])
            assert abs(gtu_h[gid] - tot) <= TOL * scale_d, (I, J, K)
    finally:
        fe.fe_mixed_destroy(mx)
