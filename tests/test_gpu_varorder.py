"""GPU parity of the variable-order (minimum-rule) space against the oracle, through the C ABI.

Small meshes: every entry of E x and of y = E^T blockdiag(A_e) E x against the oracle (several
element blocks per order, ragged block sizes, all orders 1..8 present somewhere).  The benchmark's
mixed-order workload (64^3 hexes, 8^3-element blocks of orders 2, 4, 6): properties that hold at
any size (partition of unity, constants in the kernel of the diffusion operator, volume, symmetry).
"""
import functools

import numpy as np
import pytest

from oracle.element import DIFFUSION, MASS
from oracle.solve import pcg as oracle_pcg
from oracle.varorder import VarSpace
from paper_2603_09038_gb300.inputs import (block_orders, lognormal_coefficient, perturbed_vertices,
                                           uniform_vector)
from tests.gpu_util import TOL, lib, rel_err, torch_cuda

pytestmark = pytest.mark.gpu

CASES = {
    "blocks_2_4_6": ((4, 4, 4), dict(block=2, orders=(2, 4, 6), seed=1), None),
    "ragged_1to5_sigma1": ((5, 4, 3), dict(block=1, orders=(1, 2, 3, 4, 5), seed=2), 1.0),
    "orders_6to8": ((2, 2, 1), dict(block=1, orders=(6, 7, 8), seed=3), None),
    "single_order_3": ((3, 3, 3), dict(block=4, orders=(3,), seed=0), None),
}


def _setup(name):
    dims, kw, sigma = CASES[name]
    ne = int(np.prod(dims))
    orders = block_orders(*dims, **kw)
    V = perturbed_vertices(*dims, seed=5)
    c = None if sigma is None else lognormal_coefficient(ne, sigma)
    return dims, orders, V, c


@functools.lru_cache(maxsize=None)
def _oracle(name):
    """(space, E) of a case, built once per session (the Python construction takes seconds)."""
    dims, orders, _, _ = _setup(name)
    S = VarSpace(*dims, orders)
    return S, S.prolongation()


@pytest.mark.parametrize("name", list(CASES))
def test_sizes_layout_and_mask(name):
    torch = torch_cuda()
    fe = lib()
    dims, orders, V, c = _setup(name)
    S, E = _oracle(name)
    # the library drops weights of magnitude <= 1e-13 (its documented rule); the oracle keeps
    # every computed weight: compare structure with that rule applied to the oracle's values
    E = E.tocsr(copy=True)
    E.data[np.abs(E.data) <= 1e-13] = 0.0
    E.eliminate_zeros()
    vs = fe.fe_vspace_setup(*dims, orders, V, c)
    try:
        ntrue, nlocal, nnz = fe.fe_vspace_sizes(vs)
        assert (ntrue, nlocal, nnz) == (S.ntrue, S.nlocal, E.nnz)
        # constrained rows: every row of E other than a single weight 1
        per_row = np.diff(E.indptr)
        single = (per_row == 1) & (np.abs(E.data[np.minimum(E.indptr[:-1], E.nnz - 1)] - 1.0) == 0)
        cons = ~single
        touched = np.unique(E[np.nonzero(cons)[0]].indices).size
        assert fe.fe_vspace_constraint_sizes(vs) == (int(cons.sum()), int(per_row[cons].sum()),
                                                     touched)
        first = fe.fe_vspace_layout(vs, S.ne)
        # groups of ascending order, elements ascending within each
        key = sorted(range(S.ne), key=lambda e: (S.order[e], e))
        expect = np.zeros(S.ne, dtype=np.int64)
        off = 0
        for e in key:
            expect[e] = off
            off += int(S.order[e] + 1) ** 3
        np.testing.assert_array_equal(first, expect)
        m = torch.zeros(ntrue, dtype=torch.uint8, device="cuda")
        fe.fe_vspace_boundary_mask(vs, m)
        np.testing.assert_array_equal(m.cpu().numpy(), S.boundary_mask())
    finally:
        fe.fe_vspace_destroy(vs)


@pytest.mark.parametrize("name", list(CASES))
def test_prolongation_matches_oracle(name):
    torch = torch_cuda()
    fe = lib()
    dims, orders, V, c = _setup(name)
    S, E = _oracle(name)
    vs = fe.fe_vspace_setup(*dims, orders, V, c)
    try:
        x = uniform_vector(S.ntrue, seed=21)
        ref = E @ x
        dx = torch.from_numpy(x).cuda()
        de = torch.empty(S.nlocal, dtype=torch.float64, device="cuda")
        fe.fe_vspace_prolong(vs, dx, de)
        got = de.cpu().numpy()
        first = fe.fe_vspace_layout(vs, S.ne)
        perm = np.concatenate([first[e] + np.arange(int(S.local_size[e])) for e in range(S.ne)])
        assert rel_err(got[perm], ref) <= 1e-14
    finally:
        fe.fe_vspace_destroy(vs)


@pytest.mark.parametrize("name", list(CASES))
def test_apply_matches_oracle(name):
    """Both FP64-accurate variants (FP64 and float-float) against the oracle's E^T A E x."""
    torch = torch_cuda()
    fe = lib()
    dims, orders, V, c = _setup(name)
    S, E = _oracle(name)
    x = uniform_vector(S.ntrue, seed=22)
    refs = {kind: S.apply(V, x, kind, coeff=c, E=E) for kind in (DIFFUSION, MASS)}
    vs = fe.fe_vspace_setup(*dims, orders, V, c)
    try:
        dx = torch.from_numpy(x).cuda()
        dy = torch.empty(S.ntrue, dtype=torch.float64, device="cuda")
        for variant in ("f64", "f32x2"):
            fe.fe_vspace_set_variant(vs, variant)
            for kind, op in ((DIFFUSION, fe.FE_DIFFUSION), (MASS, fe.FE_MASS)):
                fe.fe_vspace_apply(vs, op, dx, dy)
                assert rel_err(dy.cpu().numpy(), refs[kind]) <= TOL, (kind, variant)
    finally:
        fe.fe_vspace_destroy(vs)


@pytest.mark.parametrize("name", list(CASES))
def test_diagonal_matches_oracle(name):
    """fe_vspace_diagonal against diag(E^T blockdiag(diag A_e) E), from FP64 and float-pair data."""
    torch = torch_cuda()
    fe = lib()
    dims, orders, V, c = _setup(name)
    S, E = _oracle(name)
    vs = fe.fe_vspace_setup(*dims, orders, V, c)
    try:
        d = torch.empty(S.ntrue, dtype=torch.float64, device="cuda")
        for variant in ("f64", "f32x2"):
            fe.fe_vspace_set_variant(vs, variant)
            for kind, op in ((DIFFUSION, fe.FE_DIFFUSION), (MASS, fe.FE_MASS)):
                fe.fe_vspace_diagonal(vs, op, d)
                ref = S.jacobi_diagonal(V, kind, coeff=c, E=E)
                assert rel_err(d.cpu().numpy(), ref) <= TOL, (kind, variant)
    finally:
        fe.fe_vspace_destroy(vs)


@pytest.mark.parametrize("name", ["blocks_2_4_6", "ragged_1to5_sigma1"])
def test_pcg_matches_oracle(name):
    """Jacobi-PCG on the variable-order space against the oracle's PCG on the same constrained
    system (x = 0 start, homogeneous essential conditions, the same Jacobi diagonal): the same
    iteration count (+-1), iterates that agree to the tolerance, and the true residual."""
    torch = torch_cuda()
    fe = lib()
    dims, orders, V, c = _setup(name)
    S, E = _oracle(name)
    K = S.assemble(V, DIFFUSION, coeff=c, sparse=True, E=E)
    m = S.boundary_mask().astype(bool)
    free = (~m).astype(np.float64)
    d = S.jacobi_diagonal(V, DIFFUSION, coeff=c, E=E)
    b = uniform_vector(S.ntrue, seed=31)
    rtol = 1e-10
    xo, it_o, _ = oracle_pcg(lambda v: free * (K @ (free * v)) + m * v, free * b,
                             np.where(m, 1.0, d), rtol=rtol, maxit=5000)
    vs = fe.fe_vspace_setup(*dims, orders, V, c)
    try:
        for variant in ("f64", "f32x2"):
            fe.fe_vspace_set_variant(vs, variant)
            db = torch.from_numpy(b).cuda()
            dx = torch.empty_like(db)
            st, stats = fe.fe_vspace_pcg(vs, fe.FE_DIFFUSION, db, dx, rtol, 5000)
            assert st == fe.FE_OK, fe.fe_last_error()
            assert abs(stats["iters"] - it_o) <= 1, (stats["iters"], it_o)
            assert stats["true_rel_resid"] <= 2 * rtol
            x = dx.cpu().numpy()
            assert np.abs(x - xo).max() <= 1e-7 * np.abs(xo).max()
            assert np.all(x[m] == 0.0)
    finally:
        fe.fe_vspace_destroy(vs)


def test_argument_errors():
    fe = lib()
    torch_cuda()
    V = perturbed_vertices(2, 2, 2)
    for bad in ([0] + [2] * 7, [9] + [2] * 7):
        with pytest.raises(fe.FEError) as ei:
            fe.fe_vspace_setup(2, 2, 2, bad, V)
        assert ei.value.status == fe.FE_ERR_ARG
    with pytest.raises(fe.FEError):
        fe.fe_vspace_setup(2, 2, 2, [2] * 8, V, ops=0)
    vs = fe.fe_vspace_setup(2, 2, 2, [2] * 8, V, ops=fe.FE_MASS)
    try:
        import torch
        x = torch.zeros(fe.fe_vspace_sizes(vs)[0], dtype=torch.float64, device="cuda")
        with pytest.raises(fe.FEError) as ei:
            fe.fe_vspace_apply(vs, fe.FE_DIFFUSION, x, torch.empty_like(x))
        assert ei.value.status == fe.FE_ERR_ARG
        with pytest.raises(fe.FEError) as ei:
            fe.fe_vspace_pcg(vs, fe.FE_DIFFUSION, x, torch.empty_like(x), 1e-8, 10)
        assert ei.value.status == fe.FE_ERR_ARG
        st, stats = fe.fe_vspace_pcg(vs, fe.FE_MASS, x, torch.empty_like(x), 1e-8, 10)
        assert st == fe.FE_OK and stats["iters"] == 0        # b = 0: x = 0 at once
    finally:
        fe.fe_vspace_destroy(vs)


def test_benchmark_workload_properties():
    """64^3 hexes, 8^3-element blocks of orders 2, 4, 6, perturbed unit cube (the launch
    configuration the benchmark times): E 1 = 1 on every node, A 1 = 0 for diffusion,
    1^T M 1 = volume 1, and x^T A y = y^T A x for both operators."""
    torch = torch_cuda()
    fe = lib()
    n = 64
    orders = block_orders(n, n, n, block=8, orders=(2, 4, 6), seed=7)
    V = perturbed_vertices(n, n, n)
    vs = fe.fe_vspace_setup(n, n, n, orders, V)
    try:
        fe.fe_vspace_set_variant(vs, "f32x2")
        ntrue, nlocal, _ = fe.fe_vspace_sizes(vs)
        one = torch.ones(ntrue, dtype=torch.float64, device="cuda")
        e = torch.empty(nlocal, dtype=torch.float64, device="cuda")
        fe.fe_vspace_prolong(vs, one, e)
        assert float((e - 1).abs().max()) <= 1e-14
        y = torch.empty_like(one)
        fe.fe_vspace_apply(vs, fe.FE_MASS, one, y)
        assert abs(float(y.sum()) - 1.0) <= 1e-12
        fe.fe_vspace_apply(vs, fe.FE_DIFFUSION, one, y)
        x = torch.from_numpy(uniform_vector(ntrue, seed=1)).cuda()
        ax = torch.empty_like(x)
        fe.fe_vspace_apply(vs, fe.FE_DIFFUSION, x, ax)
        assert float(y.abs().max()) <= 1e-12 * float(ax.abs().max())
        z = torch.from_numpy(uniform_vector(ntrue, seed=2)).cuda()
        az = torch.empty_like(z)
        for op in (fe.FE_DIFFUSION, fe.FE_MASS):
            fe.fe_vspace_apply(vs, op, x, ax)
            fe.fe_vspace_apply(vs, op, z, az)
            a, b = float(torch.dot(z, ax)), float(torch.dot(x, az))
            assert abs(a - b) <= 1e-12 * float(ax.abs().sum()), op
    finally:
        fe.fe_vspace_destroy(vs)


@pytest.mark.parametrize("variant", ["f64", "f32x2"])
@pytest.mark.parametrize("name", list(CASES))
def test_persistent_launch_equals_per_order_launches(name, variant):
    """One persistent launch over all orders (the default) and one fused launch per order give
    the same y = E^T blockdiag(A_e) E x (up to the order of the atomic adds), for both
    operators; the 64^3 workload's block mix is covered by the first case's orders 2, 4, 6."""
    torch = torch_cuda()
    fe = lib()
    dims, orders, V, c = _setup(name)
    vs = fe.fe_vspace_setup(*dims, orders, V, c)
    try:
        fe.fe_vspace_set_variant(vs, variant)
        ntrue, _, _ = fe.fe_vspace_sizes(vs)
        x = torch.from_numpy(uniform_vector(ntrue, seed=17)).cuda()
        for op in (fe.FE_DIFFUSION, fe.FE_MASS):
            y1 = torch.empty_like(x)
            y0 = torch.empty_like(x)
            fe.fe_vspace_set_persistent(vs, 1)
            fe.fe_vspace_apply(vs, op, x, y1)
            fe.fe_vspace_set_persistent(vs, 0)
            fe.fe_vspace_apply(vs, op, x, y0)
            torch.cuda.synchronize()
            err = float((y1 - y0).abs().max()) / float(y0.abs().max())
            assert err <= 1e-13, (op, err)
        fe.fe_vspace_set_persistent(vs, 1)
    finally:
        fe.fe_vspace_destroy(vs)


@pytest.mark.parametrize("persistent", [1, 0])
def test_batched_apply_and_pcg_match_single(persistent):
    """fe_vspace_apply_batched against one fe_vspace_apply per right-hand side; and
    fe_vspace_pcg_batched (lockstep, graph-replayed iteration batches) against fe_vspace_pcg per
    system: the same iteration counts (+-1) and iterates, true residuals within the tolerance."""
    torch = torch_cuda()
    fe = lib()
    dims, orders, V, c = _setup("blocks_2_4_6")
    vs = fe.fe_vspace_setup(*dims, orders, V, c)
    try:
        fe.fe_vspace_set_persistent(vs, persistent)
        fe.fe_vspace_set_variant(vs, "f32x2")
        n, _, _ = fe.fe_vspace_sizes(vs)
        nr = 3
        X = torch.from_numpy(np.stack([uniform_vector(n, seed=30 + j) for j in range(nr)])).cuda()
        Y = torch.empty_like(X)
        fe.fe_vspace_apply_batched(vs, fe.FE_DIFFUSION, nr, X, n, Y, n)
        y1 = torch.empty(n, dtype=torch.float64, device="cuda")
        for j in range(nr):
            fe.fe_vspace_apply(vs, fe.FE_DIFFUSION, X[j].contiguous(), y1)
            torch.cuda.synchronize()
            assert float((Y[j] - y1).abs().max()) <= 1e-13 * float(y1.abs().max())
        B = X.clone()
        Xs = torch.empty_like(B)
        rtol = 1e-9
        st, stats = fe.fe_vspace_pcg_batched(vs, fe.FE_DIFFUSION, nr, B, n, Xs, n, rtol, 5000)
        assert st == fe.FE_OK, fe.fe_last_error()
        for j in range(nr):
            x1 = torch.empty(n, dtype=torch.float64, device="cuda")
            st1, s1 = fe.fe_vspace_pcg(vs, fe.FE_DIFFUSION, B[j].contiguous(), x1, rtol, 5000)
            assert st1 == fe.FE_OK
            assert abs(stats[j]["iters"] - s1["iters"]) <= 1
            assert stats[j]["true_rel_resid"] <= 10 * rtol
            assert float((Xs[j] - x1).abs().max()) <= 1e-7 * float(x1.abs().max())
    finally:
        fe.fe_vspace_destroy(vs)


def _unpack(w, din, width):
    n1, n2 = din * width, width * width
    n3 = n1 + n2 + width * din
    return (w[:n1].reshape(din, width), w[n1:n1 + n2].reshape(width, width),
            w[n1 + n2:n3].reshape(width, din), w[n3:].reshape(din, din))


def test_learned_preconditioner_on_the_variable_order_space():
    """One network per order (orders 2, 4, 6: widths 64, 64 and the linear map for order 6, which
    runs the unfused GEMM path), copied from single-order handles: fe_vspace_lpc_apply against
    the oracle's variable-order patch operator element by element within its BF16 rounding
    bound; flexible CG with it reaches the FP64 residual and the Jacobi-PCG solution; the error
    paths (an order missing, a network of another order, an order the space lacks)."""
    from oracle import learned as ol
    from tests.gpu_util import gpu_problem
    torch = torch_cuda()
    fe = lib()
    name = "blocks_2_4_6"
    dims, orders, V, c = _setup(name)
    S, E = _oracle(name)
    E = E.tocsr(copy=True)
    E.data[np.abs(E.data) <= 1e-13] = 0.0   # the library's documented sparsity rule
    E.eliminate_zeros()
    vs = fe.fe_vspace_setup(*dims, orders, V, c)
    rng = np.random.default_rng(21)
    nets, bounds = {}, {}
    try:
        ntrue, _, _ = fe.fe_vspace_sizes(vs)
        b = torch.from_numpy(uniform_vector(ntrue, seed=8)).cuda()
        x = torch.empty_like(b)
        for p, width in ((2, 64), (4, 64), (6, 0)):
            if p == 6:   # not every order attached yet
                with pytest.raises(fe.FEError) as e:
                    fe.fe_vspace_fcg(vs, fe.FE_DIFFUSION, b, x, 1e-8, 10)
                assert e.value.status == fe.FE_ERR_UNSUPPORTED
            with gpu_problem(3, 3, 3, p) as (_, mesh, pa, _V, _c):
                lpc = fe.fe_lpc_create(pa, fe.FE_DIFFUSION, width, 10 + p)
                try:
                    din = (p + 1) ** 3
                    w = fe.fe_lpc_weights(lpc)
                    w[-din * din:] = 0.1 * rng.standard_normal(din * din)
                    fe.fe_lpc_weights(lpc, w)
                    with pytest.raises(fe.FEError) as e:      # a network of another order
                        fe.fe_vspace_set_learned(vs, fe.FE_DIFFUSION, 2 if p != 2 else 4, lpc)
                    assert e.value.status == fe.FE_ERR_ARG
                    fe.fe_vspace_set_learned(vs, fe.FE_DIFFUSION, p, lpc)
                    Wb = tuple(ol.bf16_round(a) for a in _unpack(w, din, width))
                    nets[p] = ol.network(Wb)
                    bounds[p] = ol.network_rounding_bound(Wb)
                finally:
                    fe.fe_lpc_destroy(lpc)
        with pytest.raises(fe.FEError) as e:                  # no element of order 3 here
            fe.fe_vspace_set_learned(vs, fe.FE_DIFFUSION, 3, None)
        assert e.value.status == fe.FE_ERR_ARG
        r = torch.from_numpy(np.random.default_rng(4).standard_normal(ntrue)).cuda()
        z = torch.full_like(r, float("nan"))
        fe.fe_vspace_lpc_apply(vs, r, z)
        torch.cuda.synchronize()
        zg = z.cpu().numpy()
        zr, zb = ol.vspace_patch_apply(S, V, DIFFUSION, nets, r.cpu().numpy(), coeff=c, E=E,
                                       bounds=bounds)
        assert np.abs(zr).max() > 0
        assert np.all(np.abs(zg - zr) <= zb + 1e-13 * np.abs(zr).max())
        st, sf = fe.fe_vspace_fcg(vs, fe.FE_DIFFUSION, b, x, 1e-8, 5000)
        assert st == fe.FE_OK, fe.fe_last_error()
        assert sf["true_rel_resid"] <= 1e-8
        xj = torch.empty_like(b)
        st, sj = fe.fe_vspace_pcg(vs, fe.FE_DIFFUSION, b, xj, 1e-8, 5000)
        assert st == fe.FE_OK
        assert (x - xj).abs().max().item() <= 1e-6 * xj.abs().max().item()
    finally:
        fe.fe_vspace_destroy(vs)
