"""Magnitude range of the FP64-accurate arithmetic, and the FP64 residuals of the solvers.

The float-float variant (FE_VARIANT_F32X2) keeps its values as pairs of floats, whose exponent
range is far narrower than FP64's.  Its kernels scale every thread block's inputs and every
element's quadrature data by powers of two; these tests put the inputs, the coefficient and the
right-hand side at magnitudes well outside the float range (2^+-100, 1e+-30, and vectors whose
entries span 1e-30..1e30) and compare with the oracle at the same 1e-12 bound as at O(1)
magnitudes.  They also check that every solver's reported true residual is the FP64 one (it
matches the oracle's residual of the returned iterate), and that the solvers refuse the plain
FP32 arithmetic, which is not FP64-accurate.
"""
import numpy as np
import pytest

from gpu_util import gpu_problem, rel_err, torch_cuda, TOL
from oracle import operator as oop
from oracle.element import DIFFUSION, MASS
from oracle.mesh import boundary_mask
from oracle.solve import pcg as oracle_pcg, load_vector
from paper_2603_09038_gb300.inputs import uniform_vector, lognormal_coefficient

pytestmark = pytest.mark.gpu

DIMS, P = (4, 3, 5), 3
SCALES = [2.0 ** 100, 2.0 ** -100, 1e30, 1e-30]


def _apply(fe, pa, op, variant, xh):
    torch = torch_cuda()
    x = torch.from_numpy(xh).cuda()
    y = torch.full_like(x, float("nan"))
    fe.fe_apply(pa, op, variant, x, y)
    torch.cuda.synchronize()
    return y.cpu().numpy()


@pytest.mark.parametrize("cscale", [1.0] + SCALES)
@pytest.mark.parametrize("xscale", [1.0] + SCALES)
def test_apply_at_extreme_magnitudes(xscale, cscale):
    c = lognormal_coefficient(int(np.prod(DIMS)), 1.0) * cscale
    with gpu_problem(*DIMS, P, coeff=c) as (fe, mesh, pa, V, _):
        prob = oop.Problem(*DIMS, P, V, coeff=c)
        xh = uniform_vector(prob.ndofs, seed=5) * xscale
        for variant in ("f64", "f32x2"):
            fe.fe_pa_set_variant(pa, variant)
            for op, kind in ((fe.FE_DIFFUSION, DIFFUSION), (fe.FE_MASS, MASS)):
                ref = oop.apply(prob, xh, kind)
                assert np.isfinite(ref).all() and np.abs(ref).max() > 0
                err = rel_err(_apply(fe, pa, op, variant, xh), ref)
                assert err <= TOL, (variant, kind, xscale, cscale, err)


def test_apply_on_a_vector_spanning_sixty_decades():
    """Entries log-uniform in [1e-30, 1e30] with random signs: the float-float apply, whose block
    scale follows the largest entry, still meets the relative max-norm bound."""
    rng = np.random.default_rng(11)
    with gpu_problem(*DIMS, P, sigma=1.0) as (fe, mesh, pa, V, c):
        prob = oop.Problem(*DIMS, P, V, coeff=c)
        xh = rng.choice([-1.0, 1.0], prob.ndofs) * 10.0 ** rng.uniform(-30, 30, prob.ndofs)
        for variant in ("f64", "f32x2"):
            fe.fe_pa_set_variant(pa, variant)
            for op, kind in ((fe.FE_DIFFUSION, DIFFUSION), (fe.FE_MASS, MASS)):
                err = rel_err(_apply(fe, pa, op, variant, xh), oop.apply(prob, xh, kind))
                assert err <= TOL, (variant, kind, err)


def _oracle_solve(prob, b, rtol):
    m = boundary_mask(prob.nx, prob.ny, prob.nz, prob.p).astype(np.float64)
    keep = 1.0 - m
    A = oop.assemble(prob, DIFFUSION)
    d = oop.diagonal(prob, DIFFUSION) * keep + m
    return oracle_pcg(lambda v: keep * (A @ (keep * v)) + m * v, b * keep, d, rtol=rtol), A, keep


@pytest.mark.parametrize("bscale,cscale", [(1e-30, 1.0), (1e30, 1.0), (1e-30, 1e-30),
                                           (2.0 ** -100, 2.0 ** 100)])
def test_pcg_at_extreme_magnitudes(bscale, cscale):
    """Jacobi-PCG (float-float and FP64 iterations) on b scaled far outside the float range (the
    residual falls a further 1e-10 below it): the oracle CG's iterate, scaled, to 1e-8."""
    torch = torch_cuda()
    c = lognormal_coefficient(int(np.prod(DIMS)), 1.0) * cscale
    with gpu_problem(*DIMS, P, coeff=c) as (fe, mesh, pa, V, _):
        prob = oop.Problem(*DIMS, P, V, coeff=c)
        bh = load_vector(prob) * bscale
        b = torch.from_numpy(bh).cuda()
        rtol = 1e-10
        (xr, it, _), A, keep = _oracle_solve(prob, bh, rtol)
        for variant in ("f64", "f32x2"):
            fe.fe_pa_set_variant(pa, variant)
            x = torch.empty_like(b)
            st, stats = fe.fe_pcg(pa, fe.FE_DIFFUSION, fe.FE_PC_JACOBI, b, x, rtol, 5000)
            assert st == fe.FE_OK, fe.fe_last_error()
            assert abs(stats["iters"] - it) <= 1, (variant, stats["iters"], it)
            assert stats["true_rel_resid"] <= 10 * rtol
            xg = x.cpu().numpy()
            assert np.abs(xg - xr).max() <= 1e-8 * np.abs(xr).max(), variant


@pytest.mark.parametrize("bscale,cscale", [(1e-30, 1.0), (1e-30, 1e-30), (1e30, 2.0 ** -100)])
def test_iterative_refinement_at_extreme_magnitudes(bscale, cscale):
    """Mixed-precision refinement: the FP32 inner solves see power-of-two scaled right-hand
    sides and data, so b at 1e-30 (and a residual a further 1e-10 below) still converges."""
    torch = torch_cuda()
    c = lognormal_coefficient(int(np.prod(DIMS)), 1.0) * cscale
    with gpu_problem(*DIMS, P, coeff=c) as (fe, mesh, pa, V, _):
        prob = oop.Problem(*DIMS, P, V, coeff=c)
        bh = load_vector(prob) * bscale
        b = torch.from_numpy(bh).cuda()
        x = torch.empty_like(b)
        rtol = 1e-10
        st, stats = fe.fe_pcg_ir(pa, fe.FE_DIFFUSION, fe.FE_PC_JACOBI, b, x, rtol, 5000, 1e-4)
        assert st == fe.FE_OK, fe.fe_last_error()
        assert stats["true_rel_resid"] <= rtol and stats["outer_iters"] >= 2
        (xr, _, _), _, _ = _oracle_solve(prob, bh, 1e-12)
        assert np.abs(x.cpu().numpy() - xr).max() <= 1e-8 * np.abs(xr).max()


@pytest.mark.parametrize("variant", ["f64", "f32x2"])
def test_reported_true_residual_is_the_fp64_one(variant):
    """fe_pcg's true_rel_resid equals the oracle's ||(1-m)(b - A x)|| / ||(1-m) b|| of the
    returned x (FP64 assembled matrix), whatever arithmetic iterated.  A residual near 1e-10 of
    ||b|| carries a relative rounding error near 1e-16 / 1e-10 in either computation."""
    torch = torch_cuda()
    with gpu_problem(*DIMS, P, sigma=1.0) as (fe, mesh, pa, V, c):
        prob = oop.Problem(*DIMS, P, V, coeff=c)
        bh = load_vector(prob)
        b = torch.from_numpy(bh).cuda()
        x = torch.empty_like(b)
        fe.fe_pa_set_variant(pa, variant)
        st, stats = fe.fe_pcg(pa, fe.FE_DIFFUSION, fe.FE_PC_JACOBI, b, x, 1e-10, 5000)
        assert st == fe.FE_OK
        m = boundary_mask(*DIMS, P).astype(np.float64)
        keep = 1.0 - m
        A = oop.assemble(prob, DIFFUSION)
        xg = x.cpu().numpy()
        rel = np.linalg.norm(keep * (bh - A @ xg)) / np.linalg.norm(keep * bh)
        assert abs(stats["true_rel_resid"] - rel) <= 1e-3 * rel + 1e-15, (stats, rel)


def test_solvers_refuse_the_fp32_variant():
    torch = torch_cuda()
    with gpu_problem(3, 3, 3, 2, ops=1) as (fe, mesh, pa, V, c):
        n, _, _ = fe.fe_mesh_sizes(mesh)
        b = torch.ones(n, dtype=torch.float64, device="cuda")
        x = torch.empty_like(b)
        fe.fe_pa_set_variant(pa, "f32")
        for pc in (fe.FE_PC_JACOBI, fe.FE_PC_CHEBYSHEV):
            with pytest.raises(fe.FEError) as ei:
                fe.fe_pcg(pa, fe.FE_DIFFUSION, pc, b, x, 1e-8, 10)
            assert ei.value.status == fe.FE_ERR_UNSUPPORTED
        # the refinement does not iterate with the handle's variant: it works from any of them
        st, stats = fe.fe_pcg_ir(pa, fe.FE_DIFFUSION, fe.FE_PC_JACOBI, b, x, 1e-8, 2000)
        assert st == fe.FE_OK and stats["true_rel_resid"] <= 1e-8
