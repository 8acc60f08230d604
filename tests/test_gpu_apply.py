"""GPU parity of the fused PA apply (through the C ABI) against the CPU oracle.

Small meshes: every output element compared with the oracle's element-matrix apply, for every
order 1..8, both operators and every arithmetic variant, on meshes whose element count spans
several thread blocks and leaves a ragged last block.  Full-size meshes (the ~50 M dof order
sweep and the 64^3 p=3 Poisson mesh, in the launch configuration the benchmark times): sampled
outputs, each computed one by one by the oracle, plus invariants that hold at any size.
Bound: relative max-norm error <= 1e-12.
"""
import numpy as np
import pytest

from gpu_util import gpu_problem, rel_err, torch_cuda, TOL
from oracle import operator as oop
from oracle.element import DIFFUSION, MASS
from paper_2603_09038_gb300.inputs import uniform_vector, ORDER_SWEEP_N

pytestmark = pytest.mark.gpu

VARIANTS = ["f64", "f32x2", "dmma"]
OPS = [(1, DIFFUSION), (2, MASS)]      # (FE_DIFFUSION / FE_MASS code, oracle kind)


def _apply(fe, pa, op, variant, xh):
    torch = torch_cuda()
    x = torch.from_numpy(xh).cuda()
    y = torch.full_like(x, float("nan"))
    fe.fe_apply(pa, op, variant, x, y)
    torch.cuda.synchronize()
    return y.cpu().numpy()


@pytest.mark.parametrize("variant", VARIANTS)
def test_config1_parity_ten_applies(variant):
    """4^3 hexes, p=2, Q=4, +-0.1h perturbation, c=1, x ~ U[-1,1] with seeds 0..9."""
    n, p = 4, 2
    with gpu_problem(n, n, n, p) as (fe, mesh, pa, V, c):
        fe.fe_pa_set_variant(pa, variant)
        prob = oop.Problem(n, n, n, p, V)
        for op, kind in OPS:
            for seed in range(10):
                xh = uniform_vector(prob.ndofs, seed)
                assert rel_err(_apply(fe, pa, op, variant, xh), oop.apply(prob, xh, kind)) <= TOL


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("p", range(1, 9))
def test_all_orders_ragged_blocks(variant, p):
    dims = (5, 4, 7) if p <= 3 else (3, 2, 5)
    with gpu_problem(*dims, p, sigma=1.0) as (fe, mesh, pa, V, c):
        fe.fe_pa_set_variant(pa, variant)
        prob = oop.Problem(*dims, p, V, coeff=c)
        xh = uniform_vector(prob.ndofs, seed=p)
        for op, kind in OPS:
            assert rel_err(_apply(fe, pa, op, variant, xh), oop.apply(prob, xh, kind)) <= TOL


@pytest.mark.parametrize("variant", VARIANTS)
def test_single_element_and_switching_back(variant):
    with gpu_problem(1, 1, 1, 4, sigma=1.0) as (fe, mesh, pa, V, c):
        prob = oop.Problem(1, 1, 1, 4, V, coeff=c)
        xh = uniform_vector(prob.ndofs, seed=3)
        fe.fe_pa_set_variant(pa, variant)
        for op, kind in OPS:
            assert rel_err(_apply(fe, pa, op, variant, xh), oop.apply(prob, xh, kind)) <= TOL
        fe.fe_pa_set_variant(pa, "f64")      # back to exact FP64 data
        for op, kind in OPS:
            assert rel_err(_apply(fe, pa, op, "f64", xh), oop.apply(prob, xh, kind)) <= 1e-14


def _sampled_rows(ndofs, rng, k=64):
    rows = rng.choice(ndofs, size=k, replace=False)
    return np.unique(np.concatenate([rows, [0, ndofs - 1, ndofs // 2]]))


def _full_size_check(n, p, variants, sigma=1.0):
    """FP64: sampled outputs against the oracle (computed one by one); every other variant: every
    output against the FP64 result, plus the same sampled outputs against the oracle."""
    torch = torch_cuda()
    with gpu_problem(n, n, n, p, sigma=sigma) as (fe, mesh, pa, V, c):
        ndofs, ne, _ = fe.fe_mesh_sizes(mesh)
        prob = oop.Problem(n, n, n, p, V, coeff=c)
        rng = np.random.default_rng(p)
        rows = _sampled_rows(ndofs, rng)
        trows = torch.from_numpy(rows).cuda()
        xh = uniform_vector(ndofs, seed=p)
        x = torch.from_numpy(xh).cuda()
        y = torch.empty_like(x)
        ones = torch.ones_like(x)
        yref = {}
        for variant in ["f64"] + [v for v in variants if v != "f64"]:
            fe.fe_pa_set_variant(pa, variant)
            for op, kind in OPS:
                fe.fe_apply(pa, op, variant, x, y)
                torch.cuda.synchronize()
                scale = float(y.abs().max())
                ref = oop.apply_rows(prob, xh, kind, rows)
                assert np.abs(y[trows].cpu().numpy() - ref).max() <= TOL * scale, (variant, kind)
                if variant == "f64":
                    yref[kind] = y.clone()
                else:
                    full = float((y - yref[kind]).abs().max()) / float(yref[kind].abs().max())
                    assert full <= TOL, (variant, kind, full)
                # invariants at full size: A 1 = 0; 1^T M 1 = sum_e c_e vol_e (unit cube if c=1)
                fe.fe_apply(pa, op, variant, ones, y)
                torch.cuda.synchronize()
                if kind == DIFFUSION:
                    assert float(y.abs().max()) <= TOL * scale
                else:
                    total = float(y.sum())
                    if c is None:
                        assert abs(total - 1.0) <= 1e-11
                    else:
                        assert c.min() <= total <= c.max()


@pytest.mark.parametrize("p", range(1, 9))
def test_order_sweep_full_size_sampled(p):
    """The ~50 M dof order-sweep meshes with a log-normal (sigma = 1) coefficient."""
    _full_size_check(ORDER_SWEEP_N[p], p, VARIANTS)


def test_poisson_mesh_full_size_sampled():
    """64^3 hexes, p = 3 (7.19 M dofs), c = 1: the benchmark's workload."""
    _full_size_check(64, 3, VARIANTS, sigma=None)


@pytest.mark.parametrize("p", [1, 2, 3, 5, 8])
def test_diagonal_matches_oracle(p):
    torch = torch_cuda()
    dims = (3, 2, 4)
    with gpu_problem(*dims, p, sigma=1.0) as (fe, mesh, pa, V, c):
        prob = oop.Problem(*dims, p, V, coeff=c)
        d = torch.empty(prob.ndofs, dtype=torch.float64, device="cuda")
        for op, kind in OPS:
            fe.fe_assemble_diagonal(pa, op, d)
            torch.cuda.synchronize()
            assert rel_err(d.cpu().numpy(), oop.diagonal(prob, kind)) <= TOL


@pytest.mark.parametrize("p", [1, 3, 6])
def test_load_vector_matches_oracle(p):
    from oracle.solve import load_vector
    torch = torch_cuda()
    dims = (3, 4, 2)
    with gpu_problem(*dims, p) as (fe, mesh, pa, V, c):
        prob = oop.Problem(*dims, p, V)
        b = torch.empty(prob.ndofs, dtype=torch.float64, device="cuda")
        fe.fe_load_vector_sine(pa, b)
        torch.cuda.synchronize()
        assert rel_err(b.cpu().numpy(), load_vector(prob)) <= TOL


def test_dof_map_and_mask_match_oracle():
    from oracle.mesh import dof_map, boundary_mask
    torch = torch_cuda()
    dims, p = (3, 4, 2), 3
    with gpu_problem(*dims, p) as (fe, mesh, pa, V, c):
        ndofs, ne, _ = fe.fe_mesh_sizes(mesh)
        m = torch.empty((ne, (p + 1) ** 3), dtype=torch.int32, device="cuda")
        fe.fe_mesh_dof_map(mesh, m)
        mask = torch.empty(ndofs, dtype=torch.uint8, device="cuda")
        fe.fe_mesh_boundary_mask(mesh, mask)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(m.cpu().numpy(), dof_map(*dims, p))
        np.testing.assert_array_equal(mask.cpu().numpy(), boundary_mask(*dims, p))


def test_errors_are_status_codes():
    from paper_2603_09038_gb300.inputs import perturbed_vertices
    torch = torch_cuda()
    fe = __import__("gpu_util").lib()
    V = perturbed_vertices(1, 1, 1, amp=0.0)
    V[[0, 1]] = V[[1, 0]]                       # inverted element
    mesh = fe.fe_mesh_setup(1, 1, 1, 2, V)
    try:
        with pytest.raises(fe.FEError) as ei:
            fe.fe_pa_setup(mesh, 0, None, fe.FE_DIFFUSION)
        assert ei.value.status == fe.FE_ERR_ARG and "det J" in str(ei.value)
        with pytest.raises(fe.FEError) as ei:
            fe.fe_pa_setup(mesh, 3, None, fe.FE_DIFFUSION)
        assert ei.value.status == fe.FE_ERR_UNSUPPORTED
    finally:
        fe.fe_mesh_destroy(mesh)
    with gpu_problem(2, 2, 2, 2, ops=1) as (fe, mesh, pa, V, c):
        x = torch.zeros(5 ** 3, dtype=torch.float64, device="cuda")
        y = torch.zeros_like(x)
        with pytest.raises(fe.FEError) as ei:
            fe.fe_apply(pa, fe.FE_MASS, "f64", x, y)       # mass was not set up
        assert ei.value.status == fe.FE_ERR_ARG
        with pytest.raises(fe.FEError) as ei:
            fe.fe_apply(pa, fe.FE_DIFFUSION, "f32x2", x, y)  # data still FP64-encoded
        assert ei.value.status == fe.FE_ERR_ARG


@pytest.mark.parametrize("variant", ["f64", "f32x2", "f32"])
def test_batched_apply_matches_single_applies(variant):
    """fe_apply_batched over 5 right-hand sides (padded leading dimension) equals 5 single
    applies (same kernel arithmetic; only the atomic order may differ)."""
    torch = torch_cuda()
    dims, p = (5, 4, 3), 3
    with gpu_problem(*dims, p, sigma=1.0) as (fe, mesh, pa, V, c):
        nd, _, _ = fe.fe_mesh_sizes(mesh)
        fe.fe_pa_set_variant(pa, variant)
        nr, ld = 5, nd + 7
        X = torch.rand(nr, ld, dtype=torch.float64, device="cuda") * 2 - 1
        Y = torch.full((nr, ld), 7.0, dtype=torch.float64, device="cuda")
        for op in (fe.FE_DIFFUSION, fe.FE_MASS):
            fe.fe_apply_batched(pa, op, variant, nr, X, ld, Y, ld)
            y1 = torch.empty(nd, dtype=torch.float64, device="cuda")
            for r in range(nr):
                fe.fe_apply(pa, op, variant, X[r, :nd].contiguous(), y1)
                torch.cuda.synchronize()
                ref = y1.cpu().numpy()
                got = Y[r, :nd].cpu().numpy()
                tol = 1e-6 if variant == "f32" else TOL
                assert np.abs(got - ref).max() <= tol * np.abs(ref).max()
        with pytest.raises(fe.FEError):
            fe.fe_apply_batched(pa, fe.FE_DIFFUSION, variant, 2, X, nd - 1, Y, ld)


@pytest.mark.parametrize("nrhs", [1, 3])
def test_autotune_selects_fastest_accurate_variant(nrhs):
    torch = torch_cuda()
    with gpu_problem(12, 12, 12, 3, sigma=1.0) as (fe, mesh, pa, V, c):
        best, ms = fe.fe_pa_autotune(pa, fe.FE_DIFFUSION, nrhs, 3)
        assert best in ("f64", "f32x2", "dmma")
        assert "f32" not in ms and ("dmma" in ms) == (nrhs == 1)
        assert ms[best] == min(ms.values())
        assert fe.fe_pa_get_variant(pa) == fe.VARIANTS[best]
        n, _, _ = fe.fe_mesh_sizes(mesh)
        x = torch.rand(n, dtype=torch.float64, device="cuda") * 2 - 1
        y, y64 = torch.empty_like(x), torch.empty_like(x)
        fe.fe_apply_diffusion(pa, x, y)
        fe.fe_pa_set_variant(pa, "f64")
        fe.fe_apply(pa, fe.FE_DIFFUSION, "f64", x, y64)
        torch.cuda.synchronize()
        assert (y - y64).abs().max().item() <= TOL * y64.abs().max().item()
        for bad in ((0, 3), (65, 3), (1, 0)):
            with pytest.raises(fe.FEError):
                fe.fe_pa_autotune(pa, fe.FE_DIFFUSION, *bad)


@pytest.mark.parametrize("variant", ["f64", "f32x2"])
@pytest.mark.parametrize("p", [1, 3, 5, 8])
def test_every_launch_shape_matches_oracle(variant, p):
    """Each built launch shape (threads and elements per block, the autotuner's candidates) of
    the FP64 and float-float kernels against the oracle, on meshes with a ragged last block."""
    dims = (5, 4, 7) if p <= 3 else (3, 2, 5)
    with gpu_problem(*dims, p, sigma=1.0) as (fe, mesh, pa, V, c):
        fe.fe_pa_set_variant(pa, variant)
        prob = oop.Problem(*dims, p, V, coeff=c)
        xh = uniform_vector(prob.ndofs, seed=p + 20)
        _, nshapes, _, _ = fe.fe_pa_get_shape(pa, 1, variant)
        assert nshapes >= 2
        # defaults: the float-float smaller-block shape where it measured faster
        sel_d = fe.fe_pa_get_shape(pa, fe.FE_DIFFUSION, variant)[0]
        sel_m = fe.fe_pa_get_shape(pa, fe.FE_MASS, variant)[0]
        if variant == "f32x2":
            assert (sel_d, sel_m) == (1 if p <= 2 else 0, 1 if p <= 4 or p == 8 else 0)
        else:
            assert (sel_d, sel_m) == (0, 0)
        geoms = set()
        for k in range(nshapes):
            for op, kind in OPS:
                fe.fe_pa_set_shape(pa, op, variant, k)
                sel, _, nt, ne = fe.fe_pa_get_shape(pa, op, variant)
                assert sel == k and nt >= 32 and ne >= 1
                geoms.add((op, nt, ne))
                err = rel_err(_apply(fe, pa, op, variant, xh), oop.apply(prob, xh, kind))
                assert err <= TOL, (variant, p, k, kind, err)
        assert len(geoms) > 2                                  # the shapes really differ
        with pytest.raises(fe.FEError):
            fe.fe_pa_set_shape(pa, 1, variant, nshapes)
