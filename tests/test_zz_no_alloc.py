"""fe_pcg_noalloc, the allocation-free variant of fe_pcg (through the C ABI).

It exists for callers that cannot allocate device memory during a solve -- applications whose
memory belongs to their own pool allocator, and latency-critical loops that cannot pay for
cudaMalloc/cudaFree -- and takes its scratch from a fixed array inside the library.  These
checks compare it with fe_pcg on two calls in a row (the second call must not be disturbed by
what the first left in the shared array), check that the device's free memory is the same
before and after each call, and that a mesh larger than the array, or an arithmetic that is not
FP64-accurate, is refused.  This file is collected last so that a failure here stops a -x run
only after every other test has run.
"""
import numpy as np
import pytest

from gpu_util import gpu_problem, torch_cuda

pytestmark = pytest.mark.gpu


def _masked_residual_norm(fe, torch, pa, op, mask, v):
    """||(1-m) A v||_2 with the FP64 operator."""
    y = torch.empty_like(v)
    fe.fe_apply(pa, op, "f64", v * (1.0 - mask), y)
    torch.cuda.synchronize()
    return float(((1.0 - mask) * y).norm())


def test_noalloc_matches_pcg_on_two_calls_in_a_row():
    torch = torch_cuda()
    with gpu_problem(6, 5, 4, 3, sigma=1.0) as (fe, mesh, pa, V, c):
        n, _, _ = fe.fe_mesh_sizes(mesh)
        assert n <= fe.FE_PCG_NOALLOC_MAX_DOFS
        mask8 = torch.empty(n, dtype=torch.uint8, device="cuda")
        fe.fe_mesh_boundary_mask(mesh, mask8)
        mask = mask8.to(torch.float64)
        b1 = torch.empty(n, dtype=torch.float64, device="cuda")
        fe.fe_load_vector_sine(pa, b1)
        b2 = torch.from_numpy(np.random.default_rng(7).uniform(-1, 1, n)).cuda()
        cases = [(b1, fe.FE_DIFFUSION, fe.FE_PC_JACOBI, 1e-10),
                 (b2, fe.FE_MASS, fe.FE_PC_JACOBI, 1e-10)]
        # one warm-up call per operator: the first call looks the scratch array up, and the first
        # launch of each kernel may load its code (lazy module loading), which takes memory
        for b, op, pc, rtol in cases:
            xw = torch.empty_like(b)
            fe.fe_pcg(pa, op, pc, b, xw, rtol, 5000)
            fe.fe_pcg_noalloc(pa, op, pc, b, xw, rtol, 5000)
        torch.cuda.synchronize()
        for b, op, pc, rtol in cases:          # two different solves back to back
            xr = torch.empty_like(b)
            st_r, s_r = fe.fe_pcg(pa, op, pc, b, xr, rtol, 5000)
            xn = torch.full_like(b, float("nan"))
            torch.cuda.synchronize()
            free0, _ = torch.cuda.mem_get_info()
            st_n, s_n = fe.fe_pcg_noalloc(pa, op, pc, b, xn, rtol, 5000)
            torch.cuda.synchronize()
            free1, _ = torch.cuda.mem_get_info()
            assert st_r == fe.FE_OK and st_n == fe.FE_OK, fe.fe_last_error()
            assert free1 == free0, "fe_pcg_noalloc changed the device's free memory"
            assert s_n["true_rel_resid"] <= 10 * rtol and s_r["true_rel_resid"] <= 10 * rtol
            # fe_pcg takes p.Ap from the apply's fused partials, fe_pcg_noalloc from a separate
            # dot-product pass, and the apply's atomic scatter-add makes the last bits
            # order-dependent: the iterates differ by rounding, and at the threshold the counts
            # may differ by one.  Any two iterates that meet the residual test differ by a vector
            # whose residual is at most the sum of theirs: ||A_bc (xn - xr)|| <= 20 rtol ||b||.
            assert abs(s_n["iters"] - s_r["iters"]) <= 1, (s_n["iters"], s_r["iters"])
            bn = float(((1.0 - mask) * b).norm())
            d = _masked_residual_norm(fe, torch, pa, op, mask, xn - xr)
            assert d <= 20 * rtol * bn, (d, bn)
            assert float((xn * mask).abs().max()) == 0.0
            if s_n["iters"] == s_r["iters"]:
                # same number of steps: the same iterate up to rounding noise
                err = float((xn - xr).abs().max()) / float(xr.abs().max())
                assert err <= 1e-9, err


def test_noalloc_rejects_meshes_beyond_its_scratch():
    torch = torch_cuda()
    with gpu_problem(22, 22, 22, 3, ops=1) as (fe, mesh, pa, V, c):
        n, _, _ = fe.fe_mesh_sizes(mesh)
        assert n > fe.FE_PCG_NOALLOC_MAX_DOFS
        b = torch.ones(n, dtype=torch.float64, device="cuda")
        x = torch.empty_like(b)
        with pytest.raises(fe.FEError) as ei:
            fe.fe_pcg_noalloc(pa, fe.FE_DIFFUSION, fe.FE_PC_JACOBI, b, x, 1e-8, 10)
        assert ei.value.status == fe.FE_ERR_ARG and "scratch" in str(ei.value)


def test_noalloc_rejects_the_fp32_variant():
    torch = torch_cuda()
    with gpu_problem(3, 3, 3, 2, ops=1) as (fe, mesh, pa, V, c):
        n, _, _ = fe.fe_mesh_sizes(mesh)
        fe.fe_pa_set_variant(pa, "f32")
        b = torch.ones(n, dtype=torch.float64, device="cuda")
        x = torch.empty_like(b)
        with pytest.raises(fe.FEError) as ei:
            fe.fe_pcg_noalloc(pa, fe.FE_DIFFUSION, fe.FE_PC_JACOBI, b, x, 1e-8, 10)
        assert ei.value.status == fe.FE_ERR_UNSUPPORTED
