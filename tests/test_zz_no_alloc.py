"""fe_pcg_noalloc, the allocation-free variant of fe_pcg (through the C ABI).

It exists for callers that cannot allocate device memory during a solve -- applications whose
memory belongs to their own pool allocator, and latency-critical loops that cannot pay for
cudaMalloc/cudaFree -- and takes its scratch from a fixed array inside the library.  These
checks compare it with fe_pcg on two calls in a row (the second call must not be disturbed by
what the first left in the shared array) and check that a mesh larger than the array is
refused.  This file is collected last so that a failure here stops a -x run only after every
other test has run.
"""
import numpy as np
import pytest

from gpu_util import gpu_problem, torch_cuda, TOL

pytestmark = pytest.mark.gpu


def _close(a, b):
    a, b = a.cpu().numpy(), b.cpu().numpy()
    return np.abs(a - b).max() <= TOL * max(np.abs(b).max(), 1e-300)


def test_noalloc_matches_pcg_on_two_calls_in_a_row():
    torch = torch_cuda()
    with gpu_problem(6, 5, 4, 3, sigma=1.0) as (fe, mesh, pa, V, c):
        n, _, _ = fe.fe_mesh_sizes(mesh)
        assert n <= fe.FE_PCG_NOALLOC_MAX_DOFS
        b1 = torch.empty(n, dtype=torch.float64, device="cuda")
        fe.fe_load_vector_sine(pa, b1)
        b2 = torch.from_numpy(np.random.default_rng(7).uniform(-1, 1, n)).cuda()
        cases = [(b1, fe.FE_DIFFUSION, fe.FE_PC_JACOBI, 1e-10),
                 (b2, fe.FE_MASS, fe.FE_PC_JACOBI, 1e-10)]
        for b, op, pc, rtol in cases:          # two different solves back to back
            xr = torch.empty_like(b)
            st_r, s_r = fe.fe_pcg(pa, op, pc, b, xr, rtol, 5000)
            xn = torch.full_like(b, float("nan"))
            st_n, s_n = fe.fe_pcg_noalloc(pa, op, pc, b, xn, rtol, 5000)
            torch.cuda.synchronize()
            assert st_r == fe.FE_OK and st_n == fe.FE_OK, fe.fe_last_error()
            # the apply's atomic scatter-add makes the last bits order-dependent, so the
            # iteration count may differ by one at the threshold; the answers agree to TOL
            assert abs(s_n["iters"] - s_r["iters"]) <= max(1, s_r["iters"] // 100)
            assert _close(xn, xr)
            assert s_n["true_rel_resid"] <= 10 * rtol and s_r["true_rel_resid"] <= 10 * rtol
            assert abs(s_n["true_rel_resid"] - s_r["true_rel_resid"]) <= TOL


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
