"""GPU Jacobi-PCG (fe_pcg through the C ABI) against the oracle's CG, the manufactured
O(h^{p+1}) convergence on the 64^3 p = 3 Poisson problem, and the failure paths (made on the
host: NaN in b, an indefinite operator, maxit)."""
import numpy as np
import pytest

from gpu_util import gpu_problem, torch_cuda
from oracle import operator as oop
from oracle.element import DIFFUSION
from oracle.mesh import boundary_mask
from oracle.solve import pcg as oracle_pcg, load_vector, l2_error

pytestmark = pytest.mark.gpu


def _oracle_solve(prob, b, rtol):
    m = boundary_mask(prob.nx, prob.ny, prob.nz, prob.p).astype(np.float64)
    keep = 1.0 - m
    A = oop.assemble(prob, DIFFUSION)
    d = oop.diagonal(prob, DIFFUSION) * keep + m
    return oracle_pcg(lambda v: keep * (A @ (keep * v)) + m * v, b * keep, d, rtol=rtol)


@pytest.mark.parametrize("variant", ["f64", "f32x2"])
@pytest.mark.parametrize("dims,p", [((4, 4, 4), 2), ((6, 5, 4), 3), ((3, 3, 3), 6)])
def test_pcg_matches_oracle_cg(variant, dims, p):
    torch = torch_cuda()
    with gpu_problem(*dims, p, sigma=1.0) as (fe, mesh, pa, V, c):
        prob = oop.Problem(*dims, p, V, coeff=c)
        b = torch.empty(prob.ndofs, dtype=torch.float64, device="cuda")
        fe.fe_load_vector_sine(pa, b)
        x = torch.empty_like(b)
        rtol = 1e-10
        fe.fe_pa_set_variant(pa, variant)
        st, stats = fe.fe_pcg(pa, fe.FE_DIFFUSION, fe.FE_PC_JACOBI, b, x, rtol, 5000)
        assert st == fe.FE_OK, fe.fe_last_error()
        assert stats["rel_resid"] <= rtol and stats["true_rel_resid"] <= 10 * rtol
        xr, it, hist = _oracle_solve(prob, load_vector(prob), rtol)
        assert abs(stats["iters"] - it) <= 1, (stats["iters"], it)
        xg = x.cpu().numpy()
        assert np.abs(xg - xr).max() <= 1e-8 * np.abs(xr).max()
        assert np.all(xg[boundary_mask(*dims, p) == 1] == 0.0)


@pytest.mark.parametrize("pinned", [True, False])
def test_pcg_host_buffers_match_device_solve(pinned):
    """fe_pcg_host (host b in, host x out, copies inside the call) gives the device call's
    iteration count and x (to rounding: the scatter's FP64 atomics make the order of the sums,
    and so the last bits, vary from solve to solve), with pinned torch tensors and with pageable
    numpy arrays; the oracle's CG pins the answer as for fe_pcg."""
    torch = torch_cuda()
    dims, p = (5, 4, 4), 3
    with gpu_problem(*dims, p, sigma=1.0) as (fe, mesh, pa, V, c):
        prob = oop.Problem(*dims, p, V, coeff=c)
        b = torch.empty(prob.ndofs, dtype=torch.float64, device="cuda")
        fe.fe_load_vector_sine(pa, b)
        x = torch.empty_like(b)
        st, ref = fe.fe_pcg(pa, fe.FE_DIFFUSION, fe.FE_PC_JACOBI, b, x, 1e-10, 5000)
        assert st == fe.FE_OK
        if pinned:
            hb = b.cpu().pin_memory()
            hx = torch.full((prob.ndofs,), float("nan"), dtype=torch.float64).pin_memory()
        else:
            hb = b.cpu().numpy().copy()
            hx = np.full(prob.ndofs, np.nan)
        st, stats = fe.fe_pcg_host(pa, fe.FE_DIFFUSION, fe.FE_PC_JACOBI, hb, hx, 1e-10, 5000)
        assert st == fe.FE_OK, fe.fe_last_error()
        got = hx.numpy() if pinned else hx
        assert stats["iters"] == ref["iters"]
        xd = x.cpu().numpy()
        assert np.abs(got - xd).max() <= 1e-9 * np.abs(xd).max()
        xr, it, _ = _oracle_solve(prob, load_vector(prob), 1e-10)
        assert np.abs(got - xr).max() <= 1e-8 * np.abs(xr).max()
        # not converged: the last iterate still comes back
        hx2 = np.full(prob.ndofs, np.nan)
        st, stats = fe.fe_pcg_host(pa, fe.FE_DIFFUSION, fe.FE_PC_JACOBI, b.cpu().numpy(), hx2,
                                   1e-12, 2)
        assert st == fe.FE_ERR_NOT_CONVERGED and stats["iters"] == 2
        assert np.all(np.isfinite(hx2))
        with pytest.raises(ValueError):                 # a device tensor is not a host buffer
            fe.fe_pcg_host(pa, fe.FE_DIFFUSION, fe.FE_PC_JACOBI, b, hx2, 1e-10, 10)
        with pytest.raises(fe.FEError) as e:            # bad operator: host_x left untouched
            hx3 = np.full(prob.ndofs, 7.0)
            fe.fe_pcg_host(pa, 99, fe.FE_PC_JACOBI, b.cpu().numpy(), hx3, 1e-10, 10)
        assert e.value.status == fe.FE_ERR_ARG and np.all(hx3 == 7.0)


def test_pcg_failure_paths():
    torch = torch_cuda()
    with gpu_problem(3, 3, 3, 2) as (fe, mesh, pa, V, c):
        n, _, _ = fe.fe_mesh_sizes(mesh)
        b = torch.empty(n, dtype=torch.float64, device="cuda")
        fe.fe_load_vector_sine(pa, b)
        x = torch.empty_like(b)
        st, stats = fe.fe_pcg(pa, fe.FE_DIFFUSION, fe.FE_PC_JACOBI, b, x, 1e-12, 1)
        assert st == fe.FE_ERR_NOT_CONVERGED and stats["iters"] == 1
        b2 = b.clone()
        b2[n // 2] = float("nan")                 # an interior dof
        st, _ = fe.fe_pcg(pa, fe.FE_DIFFUSION, fe.FE_PC_JACOBI, b2, x, 1e-10, 100)
        assert st == fe.FE_ERR_NAN
        zero = torch.zeros_like(b)
        st, stats = fe.fe_pcg(pa, fe.FE_DIFFUSION, fe.FE_PC_JACOBI, zero, x, 1e-10, 100)
        assert st == fe.FE_OK and stats["iters"] == 0 and float(x.abs().max()) == 0.0
    neg = -np.ones(27)                             # negative coefficient: -K is not SPD
    with gpu_problem(3, 3, 3, 2, coeff=neg) as (fe, mesh, pa, V, c):
        n, _, _ = fe.fe_mesh_sizes(mesh)
        b = torch.empty(n, dtype=torch.float64, device="cuda")
        fe.fe_load_vector_sine(pa, b)
        x = torch.empty_like(b)
        st, _ = fe.fe_pcg(pa, fe.FE_DIFFUSION, fe.FE_PC_NONE, b, x, 1e-10, 100)
        assert st == fe.FE_ERR_BREAKDOWN
        st, _ = fe.fe_pcg(pa, fe.FE_DIFFUSION, fe.FE_PC_JACOBI, b, x, 1e-10, 100)
        assert st == fe.FE_ERR_BREAKDOWN


def test_poisson_64_cubed_p3_convergence():
    """64^3 hexes p=3 (7.19 M dofs): Jacobi-PCG to 1e-10; the L2 error against the exact sine
    falls like h^{p+1} from 16^3 to 32^3 to 64^3 (rate 4 +- 0.2)."""
    torch = torch_cuda()
    errs = []
    for n in (16, 32, 64):
        with gpu_problem(n, n, n, 3) as (fe, mesh, pa, V, c):
            nd, _, _ = fe.fe_mesh_sizes(mesh)
            b = torch.empty(nd, dtype=torch.float64, device="cuda")
            fe.fe_load_vector_sine(pa, b)
            x = torch.empty_like(b)
            st, stats = fe.fe_pcg(pa, fe.FE_DIFFUSION, fe.FE_PC_JACOBI, b, x, 1e-10, 20000)
            assert st == fe.FE_OK and stats["true_rel_resid"] <= 1e-9
            errs.append(l2_error(oop.Problem(n, n, n, 3, V), x.cpu().numpy()))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(rates - 4.0) < 0.2), (errs, rates)


def test_f32_apply_is_fp32_accurate():
    """The FP32 inner operator of iterative refinement: relative error ~1e-6, not FP64."""
    from oracle import operator as oop2
    from paper_2603_09038_gb300.inputs import uniform_vector
    torch = torch_cuda()
    with gpu_problem(5, 4, 3, 3, sigma=1.0) as (fe, mesh, pa, V, c):
        prob = oop2.Problem(5, 4, 3, 3, V, coeff=c)
        fe.fe_pa_set_variant(pa, "f32")
        xh = uniform_vector(prob.ndofs, 1)
        x = torch.from_numpy(xh).cuda()
        y = torch.empty_like(x)
        for op, kind in ((fe.FE_DIFFUSION, DIFFUSION), (fe.FE_MASS, "mass")):
            fe.fe_apply(pa, op, "f32", x, y)
            torch.cuda.synchronize()
            ref = oop2.apply(prob, xh, kind)
            err = np.abs(y.cpu().numpy() - ref).max() / np.abs(ref).max()
            assert 1e-9 < err < 1e-5, err


@pytest.mark.parametrize("hi", ["f64", "f32x2"])
@pytest.mark.parametrize("dims,p", [((6, 5, 4), 3), ((4, 4, 4), 5)])
def test_iterative_refinement_reaches_fp64_residual(hi, dims, p):
    torch = torch_cuda()
    with gpu_problem(*dims, p, sigma=1.0) as (fe, mesh, pa, V, c):
        prob = oop.Problem(*dims, p, V, coeff=c)
        b = torch.empty(prob.ndofs, dtype=torch.float64, device="cuda")
        fe.fe_load_vector_sine(pa, b)
        x = torch.empty_like(b)
        fe.fe_pa_set_variant(pa, hi)
        rtol = 1e-10
        st, stats = fe.fe_pcg_ir(pa, fe.FE_DIFFUSION, fe.FE_PC_JACOBI, b, x, rtol, 5000, 1e-4)
        assert st == fe.FE_OK, fe.fe_last_error()
        assert stats["true_rel_resid"] <= rtol and stats["outer_iters"] >= 2
        xr, it, hist = _oracle_solve(prob, load_vector(prob), 1e-12)
        assert np.abs(x.cpu().numpy() - xr).max() <= 1e-8 * np.abs(xr).max()


def test_iterative_refinement_on_the_poisson_workload():
    """64^3 hexes p=3: fe_pcg_ir to 1e-8 gives the same answer as fe_pcg (both FP64-accurate
    residuals <= 1e-8) and a true residual checked by the oracle's own apply on sampled rows."""
    torch = torch_cuda()
    with gpu_problem(64, 64, 64, 3) as (fe, mesh, pa, V, c):
        nd, _, _ = fe.fe_mesh_sizes(mesh)
        b = torch.empty(nd, dtype=torch.float64, device="cuda")
        fe.fe_load_vector_sine(pa, b)
        x1 = torch.empty_like(b)
        x2 = torch.empty_like(b)
        st1, s1 = fe.fe_pcg(pa, fe.FE_DIFFUSION, fe.FE_PC_JACOBI, b, x1, 1e-8, 20000)
        st2, s2 = fe.fe_pcg_ir(pa, fe.FE_DIFFUSION, fe.FE_PC_JACOBI, b, x2, 1e-8, 20000)
        assert st1 == fe.FE_OK and st2 == fe.FE_OK
        assert s2["true_rel_resid"] <= 1e-8
        d = float((x1 - x2).abs().max() / x1.abs().max())
        assert d < 1e-6, d


def _bc_system(prob):
    m = boundary_mask(prob.nx, prob.ny, prob.nz, prob.p).astype(np.float64)
    keep = 1.0 - m
    A = oop.assemble(prob, DIFFUSION).toarray()
    Abc = keep[:, None] * A * keep[None, :] + np.diag(m)
    return A, Abc, keep


def test_chebyshev_pcg_matches_oracle_and_estimate_bounds():
    """fe_pcg_chebyshev with the oracle's exact lambda_max: the same iteration count as the
    oracle's Chebyshev-PCG (same polynomial), the dense solution; fe_estimate_lmax is a lower
    bound within 15 % of the exact value after 20 power steps."""
    from oracle.solve import pcg_prec, chebyshev
    torch = torch_cuda()
    dims, p = (5, 4, 4), 3
    with gpu_problem(*dims, p, sigma=1.0) as (fe, mesh, pa, V, c):
        prob = oop.Problem(*dims, p, V, coeff=c)
        A, Abc, keep = _bc_system(prob)
        dg = np.diag(Abc)
        s = np.sqrt(dg)
        lmax = float(np.linalg.eigvalsh(Abc / s[:, None] / s[None, :]).max())
        est = fe.fe_estimate_lmax(pa, fe.FE_DIFFUSION, 20)
        assert 0.85 * lmax <= est <= lmax * (1 + 1e-10), (est, lmax)
        b = torch.empty(prob.ndofs, dtype=torch.float64, device="cuda")
        fe.fe_load_vector_sine(pa, b)
        x = torch.empty_like(b)
        for variant in ("f64", "f32x2"):
            fe.fe_pa_set_variant(pa, variant)
            st, stats = fe.fe_pcg_chebyshev(pa, fe.FE_DIFFUSION, b, x, 1e-10, 2000, degree=4,
                                            lmax=lmax, lmin_ratio=30.0)
            assert st == fe.FE_OK, fe.fe_last_error()
            assert stats["rel_resid"] <= 1e-10 and stats["true_rel_resid"] <= 1e-9
            bh = b.cpu().numpy() * keep
            Aop = lambda v: keep * (A @ (keep * v))
            xo, ito, _ = pcg_prec(Aop, bh, lambda r: chebyshev(Aop, keep / dg, r, 4, lmax / 30, lmax),
                                  rtol=1e-10)
            assert abs(stats["iters"] - ito) <= 1, (stats["iters"], ito)
            xr = np.linalg.solve(Abc, bh)
            assert np.abs(x.cpu().numpy() - xr).max() <= 1e-8 * np.abs(xr).max()


def test_pcg_chebyshev_default_beats_jacobi_iterations():
    torch = torch_cuda()
    n, p = 12, 3
    with gpu_problem(n, n, n, p, ops=1) as (fe, mesh, pa, V, c):
        fe.fe_pa_set_variant(pa, "f32x2")
        nd, _, _ = fe.fe_mesh_sizes(mesh)
        b = torch.empty(nd, dtype=torch.float64, device="cuda")
        fe.fe_load_vector_sine(pa, b)
        xj, xc = torch.empty_like(b), torch.empty_like(b)
        st, sj = fe.fe_pcg(pa, fe.FE_DIFFUSION, fe.FE_PC_JACOBI, b, xj, 1e-8, 5000)
        assert st == fe.FE_OK
        st, sc = fe.fe_pcg(pa, fe.FE_DIFFUSION, fe.FE_PC_CHEBYSHEV, b, xc, 1e-8, 5000)
        assert st == fe.FE_OK, fe.fe_last_error()
        assert sc["true_rel_resid"] <= 1e-7
        assert 2 * sc["iters"] < sj["iters"], (sc, sj)
        d = (xc - xj).abs().max().item() / xj.abs().max().item()
        assert d <= 1e-6


def test_chebyshev_argument_errors():
    torch = torch_cuda()
    with gpu_problem(3, 3, 3, 2) as (fe, mesh, pa, V, c):
        n, _, _ = fe.fe_mesh_sizes(mesh)
        b = torch.ones(n, dtype=torch.float64, device="cuda")
        x = torch.empty_like(b)
        for kw in ({"degree": 33}, {"degree": -1}, {"lmin_ratio": 1.0}, {"lmax": -1.0}):
            with pytest.raises(fe.FEError) as e:
                fe.fe_pcg_chebyshev(pa, fe.FE_DIFFUSION, b, x, 1e-8, 10, **kw)
            assert e.value.status == fe.FE_ERR_ARG
        with pytest.raises(fe.FEError):
            fe.fe_pcg_ir(pa, fe.FE_DIFFUSION, fe.FE_PC_CHEBYSHEV, b, x, 1e-8, 10)
        with pytest.raises(fe.FEError):
            fe.fe_estimate_lmax(pa, fe.FE_DIFFUSION, -1)


@pytest.mark.parametrize("variant,maxit", [("f32x2", 5000), ("f64", 5000), ("dmma", 5000), ("f32x2", 21)])
def test_pcg_graph_replay_matches_eager(variant, maxit):
    """Iteration batches replayed as CUDA graphs give the same solve as kernel-by-kernel launches
    (atomics may change the last bits, so iterations within 1 and solutions within 1e-10), and
    stop at maxit exactly when it is not a multiple of the batch."""
    torch = torch_cuda()
    with gpu_problem(8, 8, 8, 3, sigma=1.0, ops=1) as (fe, mesh, pa, V, c):
        fe.fe_pa_set_variant(pa, variant)
        nd, _, _ = fe.fe_mesh_sizes(mesh)
        b = torch.empty(nd, dtype=torch.float64, device="cuda")
        fe.fe_load_vector_sine(pa, b)
        xg, xe = torch.empty_like(b), torch.empty_like(b)
        fe.fe_pcg_set_graphs(pa, 1)
        st_g, sg = fe.fe_pcg(pa, fe.FE_DIFFUSION, fe.FE_PC_JACOBI, b, xg, 1e-10, maxit)
        fe.fe_pcg_set_graphs(pa, 0)
        st_e, se = fe.fe_pcg(pa, fe.FE_DIFFUSION, fe.FE_PC_JACOBI, b, xe, 1e-10, maxit)
        assert st_g == st_e
        if maxit == 21:
            assert st_g == fe.FE_ERR_NOT_CONVERGED and sg["iters"] == se["iters"] == 21
        else:
            assert st_g == fe.FE_OK and abs(sg["iters"] - se["iters"]) <= 1
        assert sg["launches"] == se["launches"] or maxit != 21
        d = (xg - xe).abs().max().item() / xe.abs().max().item()
        assert d <= 1e-10 if maxit != 21 else d <= 1e-12


@pytest.mark.parametrize("variant", ["f32x2", "f64", "dmma"])
def test_pcg_batched_matches_single_solves(variant):
    """fe_pcg_batched on 5 right-hand sides (padded leading dimensions, one zero system) gives each
    system the solve fe_pcg gives it alone: iterations within 1, solutions within 1e-9."""
    torch = torch_cuda()
    dims, p = (6, 5, 4), 3
    with gpu_problem(*dims, p, sigma=1.0, ops=1) as (fe, mesh, pa, V, c):
        fe.fe_pa_set_variant(pa, variant)
        n, _, _ = fe.fe_mesh_sizes(mesh)
        nr, ld = 5, n + 7
        rng = np.random.default_rng(3)
        Bh = np.zeros((nr, ld))
        sine = torch.empty(n, dtype=torch.float64, device="cuda")
        fe.fe_load_vector_sine(pa, sine)
        Bh[0, :n] = sine.cpu().numpy()
        Bh[1, :n] = rng.standard_normal(n)
        Bh[2, :n] = 0.0                       # converges at once
        Bh[3, :n] = 3.0 * sine.cpu().numpy() + rng.uniform(-1, 1, n)
        Bh[4, :n] = rng.uniform(0, 1, n)
        B = torch.from_numpy(Bh.reshape(-1)).cuda()
        X = torch.full((nr * ld,), 7.0, dtype=torch.float64, device="cuda")
        st, stats = fe.fe_pcg_batched(pa, fe.FE_DIFFUSION, fe.FE_PC_JACOBI, nr, B, ld, X, ld,
                                      1e-10, 5000)
        assert st == fe.FE_OK, fe.fe_last_error()
        assert stats[2]["iters"] == 0
        Xh = X.cpu().numpy().reshape(nr, ld)
        assert np.all(Xh[2, :n] == 0.0)
        assert np.all(Xh[:, n:] == 7.0)       # padding untouched
        x1 = torch.empty(n, dtype=torch.float64, device="cuda")
        for j in (0, 1, 3, 4):
            b1 = torch.from_numpy(np.ascontiguousarray(Bh[j, :n])).cuda()
            st1, s1 = fe.fe_pcg(pa, fe.FE_DIFFUSION, fe.FE_PC_JACOBI, b1, x1, 1e-10, 5000)
            assert st1 == fe.FE_OK
            assert abs(stats[j]["iters"] - s1["iters"]) <= 1, (j, stats[j], s1)
            assert stats[j]["rel_resid"] <= 1e-10 and stats[j]["true_rel_resid"] <= 1e-9
            ref = x1.cpu().numpy()
            assert np.abs(Xh[j, :n] - ref).max() <= 1e-9 * np.abs(ref).max()


def test_pcg_batched_failure_is_per_system():
    torch = torch_cuda()
    with gpu_problem(4, 4, 4, 2, ops=1) as (fe, mesh, pa, V, c):
        n, _, _ = fe.fe_mesh_sizes(mesh)
        sine = torch.empty(n, dtype=torch.float64, device="cuda")
        fe.fe_load_vector_sine(pa, sine)
        B = torch.stack([sine, sine.clone(), sine.clone()]).reshape(-1).contiguous()
        B[n + n // 2] = float("nan")          # an interior dof of system 1
        X = torch.empty_like(B)
        st, stats = fe.fe_pcg_batched(pa, fe.FE_DIFFUSION, fe.FE_PC_JACOBI, 3, B, n, X, n, 1e-10, 500)
        assert st == fe.FE_ERR_NAN
        assert stats[0]["rel_resid"] <= 1e-10 and stats[2]["rel_resid"] <= 1e-10
        assert stats[0]["iters"] == stats[2]["iters"] > 0
        st, stats = fe.fe_pcg_batched(pa, fe.FE_DIFFUSION, fe.FE_PC_JACOBI, 1, sine, n, X, n, 1e-12, 3)
        assert st == fe.FE_ERR_NOT_CONVERGED and stats[0]["iters"] == 3
        for args in ((0, n, n), (2, n - 1, n), (2, n, n - 1)):
            with pytest.raises(fe.FEError):
                fe.fe_pcg_batched(pa, fe.FE_DIFFUSION, fe.FE_PC_JACOBI, args[0], B, args[1], X,
                                  args[2], 1e-8, 10)
        with pytest.raises(fe.FEError):
            fe.fe_pcg_batched(pa, fe.FE_DIFFUSION, fe.FE_PC_CHEBYSHEV, 1, sine, n, X, n, 1e-8, 10)


def test_chebyshev_degree_one_is_scaled_jacobi():
    """Degree 1 gives z = D^-1 r / theta: a constant multiple of Jacobi, which leaves the CG
    iterates unchanged, so iterations and solution equal Jacobi-PCG's."""
    torch = torch_cuda()
    with gpu_problem(6, 6, 6, 3, sigma=1.0, ops=1) as (fe, mesh, pa, V, c):
        n, _, _ = fe.fe_mesh_sizes(mesh)
        b = torch.empty(n, dtype=torch.float64, device="cuda")
        fe.fe_load_vector_sine(pa, b)
        xj, xc = torch.empty_like(b), torch.empty_like(b)
        st, sj = fe.fe_pcg(pa, fe.FE_DIFFUSION, fe.FE_PC_JACOBI, b, xj, 1e-10, 5000)
        st2, sc = fe.fe_pcg_chebyshev(pa, fe.FE_DIFFUSION, b, xc, 1e-10, 5000, degree=1,
                                      lmax=3.0, lmin_ratio=7.0)
        assert st == st2 == fe.FE_OK
        assert abs(sj["iters"] - sc["iters"]) <= 1
        d = (xc - xj).abs().max().item() / xj.abs().max().item()
        assert d <= 1e-9


def test_refinement_on_the_mixed_precision_configuration():
    """96^3 hexes, p = 4 (57 M dofs), sine load: the refinement (FP32 inner PCG, FP64 outer
    residual) reaches the FP64 residual 1e-8; its residual on sampled rows, computed by the
    oracle's own apply, is within the global bound |r_i| <= ||r||_2 <= 1e-8 ||b||_2; and it agrees
    with the float-float Jacobi-PCG answer."""
    torch = torch_cuda()
    n, p = 96, 4
    with gpu_problem(n, n, n, p, ops=1) as (fe, mesh, pa, V, c):
        nd, _, _ = fe.fe_mesh_sizes(mesh)
        b = torch.empty(nd, dtype=torch.float64, device="cuda")
        fe.fe_load_vector_sine(pa, b)
        x = torch.empty_like(b)
        st, stats = fe.fe_pcg_ir(pa, fe.FE_DIFFUSION, fe.FE_PC_JACOBI, b, x, 1e-8, 20000)
        assert st == fe.FE_OK and stats["true_rel_resid"] <= 1e-8, fe.fe_last_error()
        mask = boundary_mask(n, n, n, p)
        rng = np.random.default_rng(9)
        rows = rng.choice(np.nonzero(mask == 0)[0], 40, replace=False)
        prob = oop.Problem(n, n, n, p, V)
        xh, bh = x.cpu().numpy(), b.cpu().numpy()
        r_rows = bh[rows] - oop.apply_rows(prob, xh, DIFFUSION, rows)
        bn = float(np.linalg.norm(bh * (1 - mask)))
        assert np.abs(r_rows).max() <= 1e-8 * bn
        fe.fe_pa_set_variant(pa, "f32x2")
        xf = torch.empty_like(b)
        st, sf = fe.fe_pcg(pa, fe.FE_DIFFUSION, fe.FE_PC_JACOBI, b, xf, 1e-8, 20000)
        assert st == fe.FE_OK
        assert float((x - xf).abs().max()) <= 1e-6 * float(xf.abs().max())
