"""GPU learned patch preconditioner and flexible CG through the C ABI.

* The BF16 tensor-core forward and backward passes (fe_lpc_loss_grad) against the FP64 oracle
  (oracle/mlp.py, itself pinned by finite differences) on ragged shapes; the tolerance covers
  the BF16 rounding of the activations and of the back-propagated signals (unit roundoff 2^-8 per
  rounding, a few roundings deep, relative Frobenius error <= 3e-2) and is far below the O(1)
  error of a transposed or dropped term.
* The patch apply z = sum_e R_e^T W_e S_e s_e f(x_e / s_e), x_e = S_e W_e R_e r, S = diag(A)^(-1/2),
  against oracle/learned.py element by element within its BF16 rounding bound, on the fused
  inference kernel and on the unfused GEMM path (a width whose weights exceed shared memory).
* The training pairs against the oracle's local solves with the assembled A_ee; one Adam step
  against the oracle's update; FCG's iterates against the oracle's FCG(1).
* Flexible CG: with Jacobi it equals PCG (iterations, solution vs the oracle's dense solve); with
  zero weights it falls back to Jacobi; trained, it reaches the same FP64 residual as Jacobi-PCG
  in fewer iterations.
"""
import numpy as np
import pytest

from gpu_util import gpu_problem, torch_cuda
from oracle import learned as ol
from oracle import mlp as omlp
from oracle import operator as oop
from oracle.element import DIFFUSION
from oracle.mesh import boundary_mask

pytestmark = pytest.mark.gpu


bf16_round = ol.bf16_round


def unpack(w, din, width):
    n1, n2 = din * width, width * width
    n3 = n1 + n2 + width * din
    return (w[:n1].reshape(din, width), w[n1:n1 + n2].reshape(width, width),
            w[n1 + n2:n3].reshape(width, din), w[n3:].reshape(din, din))


def rel_fro(a, b):
    return float(np.linalg.norm(np.asarray(a) - b) / np.linalg.norm(b))


@pytest.mark.parametrize("p,width,batch", [(2, 40, 200), (3, 64, 130), (1, 16, 77), (2, 0, 90)])
def test_loss_grad_matches_oracle(p, width, batch):
    with gpu_problem(2, 2, 2, p) as (fe, mesh, pa, V, c):
        din = (p + 1) ** 3
        lpc = fe.fe_lpc_create(pa, fe.FE_DIFFUSION, width, 7)
        try:
            assert fe.fe_lpc_nparams(lpc) == 2 * din * width + width * width + din * din
            rng = np.random.default_rng(11 + p)
            W = omlp.init_weights(din, width, 5 + p)[:3] + (0.2 * rng.standard_normal((din, din)),)
            fe.fe_lpc_weights(lpc, np.concatenate([w.reshape(-1) for w in W]))
            got = fe.fe_lpc_weights(lpc)
            assert np.array_equal(got, np.concatenate([w.reshape(-1) for w in W]).astype(np.float32))
            X = rng.standard_normal((batch, din)).astype(np.float32)
            T = rng.standard_normal((batch, din)).astype(np.float32)
            loss, Y, g = fe.fe_lpc_loss_grad(lpc, X, T)
            Wb = tuple(bf16_round(w) for w in unpack(got, din, width))
            Yr, _ = omlp.forward(Wb, bf16_round(X))
            Lr, G = omlp.grad(Wb, bf16_round(X), T)
            assert rel_fro(Y, Yr) <= 3e-2
            assert abs(loss - Lr) <= 3e-2 * Lr
            for gg, gr in zip(unpack(g.astype(np.float64), din, width), G):
                if gr.size:
                    assert rel_fro(gg, gr) <= 3e-2
        finally:
            fe.fe_lpc_destroy(lpc)


@pytest.mark.parametrize("dims,p,width", [((4, 3, 3), 2, 32), ((5, 3, 2), 3, 256),
                                          ((3, 3, 4), 1, 64), ((2, 3, 3), 4, 512),
                                          ((4, 4, 3), 3, 0), ((3, 2, 3), 4, 0)])
def test_patch_apply_matches_oracle(dims, p, width):
    """z = M(r) from the fused kernel (or the unfused GEMM path for widths whose weights exceed
    shared memory) against oracle/learned.py's patch operator in FP64 with the same BF16 weights,
    element by element within the oracle's bound on the BF16 rounding of the inputs and hidden
    activations and the FP32 accumulation."""
    torch = torch_cuda()
    with gpu_problem(*dims, p, sigma=1.0) as (fe, mesh, pa, V, c):
        prob = oop.Problem(*dims, p, V, coeff=c)
        n, ne, _ = fe.fe_mesh_sizes(mesh)
        din = (p + 1) ** 3
        lpc = fe.fe_lpc_create(pa, fe.FE_DIFFUSION, width, 3)
        try:
            w = fe.fe_lpc_weights(lpc)
            w[-din * din:] = 0.1 * np.random.default_rng(8).standard_normal(din * din)
            fe.fe_lpc_weights(lpc, w)
            r = torch.from_numpy(np.random.default_rng(4).standard_normal(n)).cuda()
            z = torch.empty_like(r)
            fe.fe_lpc_apply(lpc, r, z)
            z2 = torch.empty_like(r)
            fe.fe_lpc_apply(lpc, 2.0 * r, z2)
            torch.cuda.synchronize()
            zg, z2g = z.cpu().numpy(), z2.cpu().numpy()
            Wb = tuple(ol.bf16_round(x) for x in unpack(w, din, width))
            zr, zb = ol.patch_apply(prob, DIFFUSION, ol.network(Wb), r.cpu().numpy(),
                                    bound=ol.network_rounding_bound(Wb))
            assert np.all(np.abs(zg - zr) <= zb + 1e-13 * np.abs(zr).max())
            assert rel_fro(zg, zr) <= 3e-2
            assert np.all(zg[boundary_mask(*dims, p) == 1] == 0.0)
            # positively homogeneous: M(2r) = 2 M(r) up to the order of the atomic adds
            assert np.abs(z2g - 2.0 * zg).max() <= 1e-12 * np.abs(zg).max()
        finally:
            fe.fe_lpc_destroy(lpc)


@pytest.mark.parametrize("dims,p,width", [((9, 8, 7), 1, 64), ((5, 4, 3), 2, 128),
                                          ((6, 5, 4), 3, 128), ((5, 5, 6), 3, 0),
                                          ((3, 4, 3), 4, 64), ((4, 3, 3), 4, 128),
                                          ((50, 50, 50), 1, 128), ((9, 8, 7), 1, 256),
                                          ((6, 5, 4), 3, 256), ((30, 30, 30), 2, 256)])
def test_inference_kernels_match_oracle(dims, p, width):
    """Every inference kernel built for (order, width) -- tcgen05 (128-element tiles, FP32
    accumulators in tensor memory; at width 256 and D^3 >= 27 the hidden activations in tensor
    memory too), the mma.sync fused kernel, the unfused GEMM path -- against oracle/learned.py's
    patch operator element by element within its BF16 rounding bound. The meshes leave a ragged
    last 128-element tile; at 50^3 (p = 1) and 30^3 (p = 2, width 256) the persistent tcgen05
    grid takes several tiles per CTA. No tcgen05 launch may give up a wait."""
    torch = torch_cuda()
    with gpu_problem(*dims, p, sigma=1.0) as (fe, mesh, pa, V, c):
        prob = oop.Problem(*dims, p, V, coeff=c)
        n, ne, _ = fe.fe_mesh_sizes(mesh)
        din = (p + 1) ** 3
        lpc = fe.fe_lpc_create(pa, fe.FE_DIFFUSION, width, 3)
        try:
            w = fe.fe_lpc_weights(lpc)
            w[-din * din:] = 0.1 * np.random.default_rng(8).standard_normal(din * din)
            fe.fe_lpc_weights(lpc, w)
            default = fe.fe_lpc_get_kernel(lpc)[0]       # the fastest built one
            assert default in (fe.FE_LPC_KERNEL_MMA_SYNC, fe.FE_LPC_KERNEL_TCGEN05)
            r = torch.from_numpy(np.random.default_rng(4).standard_normal(n)).cuda()
            Wb = tuple(ol.bf16_round(x) for x in unpack(w, din, width))
            zr, zb = ol.patch_apply(prob, DIFFUSION, ol.network(Wb), r.cpu().numpy(),
                                    bound=ol.network_rounding_bound(Wb))
            tested = []
            for k in (fe.FE_LPC_KERNEL_TCGEN05, fe.FE_LPC_KERNEL_MMA_SYNC, fe.FE_LPC_KERNEL_GEMM):
                try:
                    fe.fe_lpc_set_kernel(lpc, k)
                except fe.FEError as e:
                    assert e.status == fe.FE_ERR_UNSUPPORTED and k == fe.FE_LPC_KERNEL_MMA_SYNC
                    continue
                z = torch.full_like(r, float("nan"))
                fe.fe_lpc_apply(lpc, r, z)
                torch.cuda.synchronize()
                zg = z.cpu().numpy()
                assert np.all(np.abs(zg - zr) <= zb + 1e-13 * np.abs(zr).max()), k
                assert rel_fro(zg, zr) <= 3e-2
                assert np.all(zg[boundary_mask(*dims, p) == 1] == 0.0)
                tested.append(k)
            assert fe.FE_LPC_KERNEL_TCGEN05 in tested and fe.FE_LPC_KERNEL_GEMM in tested
            assert fe.fe_lpc_get_kernel(lpc)[1] == 0
        finally:
            fe.fe_lpc_destroy(lpc)


def test_tcgen05_kernel_selection_errors_and_fp32_solve():
    """Kernel choice errors (unknown id; tcgen05 asked for a width it is not built for); the
    FP32-vector tcgen05 kernel inside fe_fcg_ir reaches the FP64 residual like the mma.sync one."""
    torch = torch_cuda()
    with gpu_problem(6, 6, 5, 2, sigma=1.0) as (fe, mesh, pa, V, c):
        n, _, _ = fe.fe_mesh_sizes(mesh)
        lpc = fe.fe_lpc_create(pa, fe.FE_DIFFUSION, 48, 1)       # width 48: no tcgen05 kernel
        try:
            with pytest.raises(fe.FEError) as e:
                fe.fe_lpc_set_kernel(lpc, fe.FE_LPC_KERNEL_TCGEN05)
            assert e.value.status == fe.FE_ERR_UNSUPPORTED
            with pytest.raises(fe.FEError) as e:
                fe.fe_lpc_set_kernel(lpc, 7)
            assert e.value.status == fe.FE_ERR_ARG
            assert fe.fe_lpc_get_kernel(lpc)[0] != fe.FE_LPC_KERNEL_TCGEN05
        finally:
            fe.fe_lpc_destroy(lpc)
    with gpu_problem(16, 16, 16, 3, ops=1) as (fe, mesh, pa, V, c):
        fe.fe_pa_set_variant(pa, "f32x2")
        n, _, _ = fe.fe_mesh_sizes(mesh)
        lpc = fe.fe_lpc_create(pa, fe.FE_DIFFUSION, 0, 4)
        try:
            fe.fe_lpc_fit_linear(lpc)
            b = torch.empty(n, dtype=torch.float64, device="cuda")
            fe.fe_load_vector_sine(pa, b)
            res = {}
            for k in (fe.FE_LPC_KERNEL_MMA_SYNC, fe.FE_LPC_KERNEL_TCGEN05):
                fe.fe_lpc_set_kernel(lpc, k)
                x = torch.empty_like(b)
                st, stats = fe.fe_fcg_ir(pa, fe.FE_DIFFUSION, lpc, b, x, 1e-8, 20000)
                assert st == fe.FE_OK, (k, fe.fe_last_error())
                assert stats["true_rel_resid"] <= 1e-8
                res[k] = x.cpu().numpy()
            xt, xm = res[fe.FE_LPC_KERNEL_TCGEN05], res[fe.FE_LPC_KERNEL_MMA_SYNC]
            assert np.abs(xt - xm).max() <= 1e-6 * np.abs(xm).max()
            assert fe.fe_lpc_get_kernel(lpc)[1] == 0
        finally:
            fe.fe_lpc_destroy(lpc)


@pytest.mark.parametrize("variant", ["f64", "f32x2"])
@pytest.mark.parametrize("dims,p", [((5, 5, 5), 2), ((4, 5, 4), 3), ((4, 4, 4), 1),
                                    ((3, 3, 4), 5)])
def test_training_pairs_are_the_oracle_local_solves(variant, dims, p):
    """Every generated pair (x, t) of element e satisfies t = S_e^-1 A_ee^-1 S_e^-1 x with A_ee the
    block of the oracle's assembled matrix and S = diag(A)^-1/2, element by element (the
    library probes A_ee with applies and factors it by FP64 Cholesky); ||t|| = 1; the pairs
    cover the three kinds (normal v, A_ee u, residual snapshots) for every sampled element."""
    with gpu_problem(*dims, p, sigma=1.0) as (fe, mesh, pa, V, c):
        fe.fe_pa_set_variant(pa, variant)
        prob = oop.Problem(*dims, p, V, coeff=c)
        din = (p + 1) ** 3
        lpc = fe.fe_lpc_create(pa, fe.FE_DIFFUSION, 0, 5)
        try:
            reps = 6
            el, X, T = fe.fe_lpc_sample_pairs(lpc, din, reps, 1 << 14)
            assert len(el) > 0 and len(el) % reps == 0
            interior = [ex + dims[0] * (ey + dims[1] * ez) for ez in range(1, dims[2] - 1)
                        for ey in range(1, dims[1] - 1) for ex in range(1, dims[0] - 1)]
            assert sorted(set(el.tolist())) == sorted(interior)
            A = oop.assemble(prob, DIFFUSION)
            _, S, _ = ol.patch_data(prob, DIFFUSION)
            nonzero = 0
            for e, x, t in zip(el, X, T):
                if not np.any(x):       # a residual snapshot the short run never reached
                    assert not np.any(t)
                    continue
                nonzero += 1
                tr = ol.local_target(prob, DIFFUSION, int(e), x, A=A, S=S)
                assert abs(np.linalg.norm(t) - 1.0) <= 1e-12
                assert np.abs(t - tr).max() <= 1e-9, (e, np.abs(t - tr).max())
            assert nonzero >= 2 * len(el) // 3
        finally:
            fe.fe_lpc_destroy(lpc)


def test_adam_step_matches_oracle():
    """Two fe_lpc_adam_step calls from a fresh handle against oracle/learned.py's Adam update with
    the gradients the library's own backward pass returns for the same batches (FP32 update
    arithmetic: ~1e-7 of the weights, well below the step lr)."""
    with gpu_problem(2, 2, 2, 2) as (fe, mesh, pa, V, c):
        din, width, lr = 27, 32, 1e-3
        lpc = fe.fe_lpc_create(pa, fe.FE_DIFFUSION, width, 7)
        try:
            rng = np.random.default_rng(21)
            w = fe.fe_lpc_weights(lpc).astype(np.float64)
            m = np.zeros_like(w)
            v = np.zeros_like(w)
            for t in (1, 2):
                X = rng.standard_normal((100, din)).astype(np.float32)
                T = rng.standard_normal((100, din)).astype(np.float32)
                _, _, g = fe.fe_lpc_loss_grad(lpc, X, T)
                fe.fe_lpc_adam_step(lpc, X, T, lr)
                w, m, v = ol.adam_step(w, g.astype(np.float64), m, v, t, lr)
                got = fe.fe_lpc_weights(lpc).astype(np.float64)
                assert np.abs(got - w).max() <= 1e-6 * np.abs(w).max() + 1e-3 * lr, t
                assert np.abs(got - fe.fe_lpc_weights(lpc)).max() == 0
        finally:
            fe.fe_lpc_destroy(lpc)


def test_fcg_iterates_match_oracle_fcg():
    """fe_fcg with Jacobi, stopped after k = 1..6 iterations, against oracle/learned.py's FCG(1)
    with the oracle's own Jacobi diagonal on the oracle's assembled constrained operator."""
    torch = torch_cuda()
    dims, p = (4, 4, 3), 2
    with gpu_problem(*dims, p, sigma=1.0) as (fe, mesh, pa, V, c):
        prob = oop.Problem(*dims, p, V, coeff=c)
        m = boundary_mask(*dims, p).astype(np.float64)
        keep = 1.0 - m
        A = oop.assemble(prob, DIFFUSION)
        d = oop.diagonal(prob, DIFFUSION) * keep + m
        bh = np.random.default_rng(6).standard_normal(prob.ndofs) * keep
        _, _, _, xs = ol.fcg(lambda u: keep * (A @ (keep * u)) + m * u, lambda r: r / d, bh,
                             rtol=0.0, maxit=6)
        b = torch.from_numpy(bh).cuda()
        x = torch.empty_like(b)
        for k in range(1, 7):
            st, s = fe.fe_fcg(pa, fe.FE_DIFFUSION, None, b, x, 1e-30, k)
            assert st == fe.FE_ERR_NOT_CONVERGED and s["iters"] == k
            xr = xs[k]
            assert np.abs(x.cpu().numpy() - xr).max() <= 1e-11 * np.abs(xr).max(), k


def _dense_solve(prob, b):
    m = boundary_mask(prob.nx, prob.ny, prob.nz, prob.p).astype(np.float64)
    keep = 1.0 - m
    A = oop.assemble(prob, DIFFUSION).toarray()
    Abc = keep[:, None] * A * keep[None, :] + np.diag(m)
    return np.linalg.solve(Abc, b * keep)


def test_fcg_jacobi_equals_pcg_and_oracle():
    torch = torch_cuda()
    dims, p = (5, 4, 4), 3
    with gpu_problem(*dims, p, sigma=1.0) as (fe, mesh, pa, V, c):
        prob = oop.Problem(*dims, p, V, coeff=c)
        b = torch.empty(prob.ndofs, dtype=torch.float64, device="cuda")
        fe.fe_load_vector_sine(pa, b)
        x1, x2 = torch.empty_like(b), torch.empty_like(b)
        st, s1 = fe.fe_pcg(pa, fe.FE_DIFFUSION, fe.FE_PC_JACOBI, b, x1, 1e-10, 5000)
        assert st == fe.FE_OK
        st, s2 = fe.fe_fcg(pa, fe.FE_DIFFUSION, None, b, x2, 1e-10, 5000)
        assert st == fe.FE_OK, fe.fe_last_error()
        assert abs(s1["iters"] - s2["iters"]) <= 2, (s1["iters"], s2["iters"])
        assert s2["rel_resid"] <= 1e-10 and s2["true_rel_resid"] <= 1e-9
        assert s2["outer_iters"] == 1
        xr = _dense_solve(prob, b.cpu().numpy())
        xg = x2.cpu().numpy()
        assert np.abs(xg - xr).max() <= 1e-8 * np.abs(xr).max()


def test_fcg_zero_network_falls_back_to_jacobi():
    torch = torch_cuda()
    with gpu_problem(4, 4, 4, 2) as (fe, mesh, pa, V, c):
        n, _, _ = fe.fe_mesh_sizes(mesh)
        b = torch.empty(n, dtype=torch.float64, device="cuda")
        fe.fe_load_vector_sine(pa, b)
        x = torch.empty_like(b)
        lpc = fe.fe_lpc_create(pa, fe.FE_DIFFUSION, 16, 1)
        try:
            fe.fe_lpc_weights(lpc, np.zeros(fe.fe_lpc_nparams(lpc), dtype=np.float32))
            st, s = fe.fe_fcg(pa, fe.FE_DIFFUSION, lpc, b, x, 1e-10, 2000)
            assert st == fe.FE_OK, fe.fe_last_error()
            assert s["outer_iters"] == 2 and s["true_rel_resid"] <= 1e-9
            st, sj = fe.fe_fcg(pa, fe.FE_DIFFUSION, None, b, x, 1e-10, 2000)
            assert abs(s["iters"] - sj["iters"]) <= 2
        finally:
            fe.fe_lpc_destroy(lpc)


def test_fcg_chebyshev_fallback_hands_over():
    """With the Chebyshev fallback a zero network (z.r = 0 at once) hands x = 0 over to
    Chebyshev-PCG on the residual equation, which is then exactly fe_pcg_chebyshev on b: the
    same iterations and the same solution."""
    torch = torch_cuda()
    with gpu_problem(4, 4, 4, 2) as (fe, mesh, pa, V, c):
        n, _, _ = fe.fe_mesh_sizes(mesh)
        b = torch.empty(n, dtype=torch.float64, device="cuda")
        fe.fe_load_vector_sine(pa, b)
        x = torch.empty_like(b)
        xc = torch.empty_like(b)
        lpc = fe.fe_lpc_create(pa, fe.FE_DIFFUSION, 16, 1)
        try:
            fe.fe_lpc_weights(lpc, np.zeros(fe.fe_lpc_nparams(lpc), dtype=np.float32))
            fe.fe_lpc_set_fallback(lpc, fe.FE_PC_CHEBYSHEV)
            st, s = fe.fe_fcg(pa, fe.FE_DIFFUSION, lpc, b, x, 1e-10, 2000)
            assert st == fe.FE_OK, fe.fe_last_error()
            assert s["outer_iters"] == 2 and s["true_rel_resid"] <= 1e-9
            st, sc = fe.fe_pcg_chebyshev(pa, fe.FE_DIFFUSION, b, xc, 1e-10, 2000)
            assert st == fe.FE_OK
            assert s["iters"] == sc["iters"]
            assert float((x - xc).abs().max()) <= 1e-13 * float(xc.abs().max())
            with pytest.raises(fe.FEError) as e:
                fe.fe_lpc_set_fallback(lpc, 7)
            assert e.value.status == fe.FE_ERR_ARG
        finally:
            fe.fe_lpc_destroy(lpc)


def test_fcg_chebyshev_fallback_after_a_stall():
    """An untrained network of width 64 on a log-normal coefficient: whether or not FCG gives it
    up (stall or breakdown rule), the solve with the Chebyshev hand-over reaches the tolerance on
    the true residual."""
    torch = torch_cuda()
    with gpu_problem(6, 6, 6, 3, sigma=2.0) as (fe, mesh, pa, V, c):
        n, _, _ = fe.fe_mesh_sizes(mesh)
        b = torch.empty(n, dtype=torch.float64, device="cuda")
        fe.fe_load_vector_sine(pa, b)
        x = torch.empty_like(b)
        lpc = fe.fe_lpc_create(pa, fe.FE_DIFFUSION, 64, 3)
        try:
            fe.fe_lpc_set_fallback(lpc, fe.FE_PC_CHEBYSHEV)
            st, s = fe.fe_fcg(pa, fe.FE_DIFFUSION, lpc, b, x, 1e-9, 5000)
            assert st == fe.FE_OK, fe.fe_last_error()
            assert s["true_rel_resid"] <= 2e-9
        finally:
            fe.fe_lpc_destroy(lpc)


def test_pcg_learned_is_fcg_with_the_attached_preconditioner():
    """fe_pcg(pc = FE_PC_LEARNED) runs fe_fcg with the preconditioner attached by
    fe_pa_set_learned; without one (or after detaching, or destroying it) it is an argument
    error."""
    torch = torch_cuda()
    with gpu_problem(4, 4, 4, 2) as (fe, mesh, pa, V, c):
        n = fe.fe_mesh_ndofs(mesh)
        assert n == fe.fe_mesh_sizes(mesh)[0]
        b = torch.empty(n, dtype=torch.float64, device="cuda")
        fe.fe_load_vector_sine(pa, b)
        x1 = torch.empty_like(b)
        x2 = torch.empty_like(b)
        with pytest.raises(fe.FEError) as e:
            fe.fe_pcg(pa, fe.FE_DIFFUSION, fe.FE_PC_LEARNED, b, x1, 1e-10, 2000)
        assert e.value.status == fe.FE_ERR_ARG
        lpc = fe.fe_lpc_create(pa, fe.FE_DIFFUSION, 16, 1)
        try:
            # a zero network: z = 0 exactly, so both solves take the same (Jacobi) path
            fe.fe_lpc_weights(lpc, np.zeros(fe.fe_lpc_nparams(lpc), dtype=np.float32))
            fe.fe_pa_set_learned(pa, lpc)
            st1, s1 = fe.fe_pcg(pa, fe.FE_DIFFUSION, fe.FE_PC_LEARNED, b, x1, 1e-10, 2000)
            st2, s2 = fe.fe_fcg(pa, fe.FE_DIFFUSION, lpc, b, x2, 1e-10, 2000)
            assert st1 == st2 == fe.FE_OK, fe.fe_last_error()
            assert abs(s1["iters"] - s2["iters"]) <= 1
            assert s1["outer_iters"] == s2["outer_iters"] == 2
            assert s1["true_rel_resid"] <= 1e-9
            assert float((x1 - x2).abs().max()) <= 1e-7 * float(x2.abs().max())
            fe.fe_pa_set_learned(pa, None)
            with pytest.raises(fe.FEError):
                fe.fe_pcg(pa, fe.FE_DIFFUSION, fe.FE_PC_LEARNED, b, x1, 1e-10, 2000)
            fe.fe_pa_set_learned(pa, lpc)
        finally:
            fe.fe_lpc_destroy(lpc)
        with pytest.raises(fe.FEError):    # destroying the preconditioner detached it
            fe.fe_pcg(pa, fe.FE_DIFFUSION, fe.FE_PC_LEARNED, b, x1, 1e-10, 2000)


def test_checkpoint_roundtrip_and_resume(tmp_path):
    """fe_lpc_save / fe_lpc_load: the weights come back exactly; training resumed from the
    checkpoint follows the uninterrupted run (same batches: the batch draw depends on the seed and
    the Adam step count); a checkpoint of another shape is refused."""
    torch = torch_cuda()
    with gpu_problem(4, 4, 4, 2) as (fe, mesh, pa, V, c):
        path = str(tmp_path / "lpc.bin")
        a = fe.fe_lpc_create(pa, fe.FE_DIFFUSION, 64, 5)
        b = fe.fe_lpc_create(pa, fe.FE_DIFFUSION, 64, 5)
        other = fe.fe_lpc_create(pa, fe.FE_DIFFUSION, 128, 5)
        try:
            n = fe.fe_lpc_nparams(a)
            fe.fe_lpc_train(a, 30, 256, 1e-3)
            fe.fe_lpc_save(a, path)
            assert fe.fe_lpc_checkpoint_info(path) == (27, 64, n, 30)
            wa = fe.fe_lpc_weights(a)            # one argument: read
            fe.fe_lpc_load(b, path)
            np.testing.assert_array_equal(wa, fe.fe_lpc_weights(b))
            fe.fe_lpc_train(a, 30, 256, 1e-3)
            fe.fe_lpc_train(b, 30, 256, 1e-3)
            wa, wb = fe.fe_lpc_weights(a), fe.fe_lpc_weights(b)
            assert np.abs(wa - wb).max() <= 1e-3 * np.abs(wa).max()
            with pytest.raises(fe.FEError) as e:
                fe.fe_lpc_load(other, path)
            assert e.value.status == fe.FE_ERR_ARG
        finally:
            fe.fe_lpc_destroy(a)
            fe.fe_lpc_destroy(b)
            fe.fe_lpc_destroy(other)


@pytest.mark.parametrize("p", [5, 6])
def test_high_order_learned_preconditioner(p):
    """Orders above 4: the patch blocks are factored by panels in shared memory and the network
    runs on the unfused GEMM path; the fitted linear map inside FCG reaches the FP64 residual."""
    torch = torch_cuda()
    with gpu_problem(4, 4, 4, p, sigma=1.0, ops=1) as (fe, mesh, pa, V, c):
        nd, _, _ = fe.fe_mesh_sizes(mesh)
        b = torch.empty(nd, dtype=torch.float64, device="cuda")
        fe.fe_load_vector_sine(pa, b)
        x = torch.empty_like(b)
        lpc = fe.fe_lpc_create(pa, fe.FE_DIFFUSION, 0, 2)
        try:
            fe.fe_lpc_fit_linear(lpc, 1e-6, 16)
            st, s = fe.fe_fcg(pa, fe.FE_DIFFUSION, lpc, b, x, 1e-9, 3000)
            assert st == fe.FE_OK, fe.fe_last_error()
            assert s["true_rel_resid"] <= 2e-9
        finally:
            fe.fe_lpc_destroy(lpc)


def test_lpc_argument_errors():
    torch = torch_cuda()
    with gpu_problem(2, 2, 2, 2, ops=1) as (fe, mesh, pa, V, c):
        with pytest.raises(fe.FEError):
            fe.fe_lpc_create(pa, fe.FE_DIFFUSION, 4, 0)
        with pytest.raises(fe.FEError):
            fe.fe_lpc_create(pa, fe.FE_MASS, 32, 0)      # operator not set up
        lpc = fe.fe_lpc_create(pa, fe.FE_DIFFUSION, 32, 0)
        try:
            with pytest.raises(fe.FEError) as e:           # fewer than 3 elements per axis
                fe.fe_lpc_train(lpc, 1, 64, 1e-3)
            assert e.value.status == fe.FE_ERR_ARG
            with gpu_problem(3, 3, 3, 2) as (fe2, mesh2, pa2, V2, c2):
                n, _, _ = fe.fe_mesh_sizes(mesh2)
                b = torch.ones(n, dtype=torch.float64, device="cuda")
                x = torch.empty_like(b)
                with pytest.raises(fe.FEError):            # built for another handle
                    fe.fe_fcg(pa2, fe.FE_DIFFUSION, lpc, b, x, 1e-8, 10)
        finally:
            fe.fe_lpc_destroy(lpc)


@pytest.mark.parametrize("n,p,sigma,width", [(16, 2, None, 128), (16, 3, None, 128),
                                             (16, 3, 1.0, 128), (16, 3, None, 0),
                                             (16, 3, 1.0, 0), (16, 2, 1.0, 0)])
def test_trained_fcg_beats_jacobi_iterations(n, p, sigma, width):
    """The gain test: trained on the operator's own patch solves, FCG reaches the same FP64
    residual as Jacobi-PCG in fewer iterations, and the two solutions agree (Poisson, and a
    log-normal coefficient with sigma = 1)."""
    torch = torch_cuda()
    with gpu_problem(n, n, n, p, sigma=sigma, ops=1) as (fe, mesh, pa, V, c):
        fe.fe_pa_set_variant(pa, "f32x2")
        nd, _, _ = fe.fe_mesh_sizes(mesh)
        b = torch.empty(nd, dtype=torch.float64, device="cuda")
        fe.fe_load_vector_sine(pa, b)
        xj, xl = torch.empty_like(b), torch.empty_like(b)
        st, sj = fe.fe_pcg(pa, fe.FE_DIFFUSION, fe.FE_PC_JACOBI, b, xj, 1e-8, 20000)
        assert st == fe.FE_OK
        lpc = fe.fe_lpc_create(pa, fe.FE_DIFFUSION, width, 2)
        try:
            l0 = fe.fe_lpc_train(lpc, 1, 1024, 1e-3)
            l1 = fe.fe_lpc_train(lpc, 2000, 1024, 1e-3)
            assert l1 < 0.5 * l0, (l0, l1)
            st, sl = fe.fe_fcg(pa, fe.FE_DIFFUSION, lpc, b, xl, 1e-8, 20000)
            assert st == fe.FE_OK, fe.fe_last_error()
            assert sl["true_rel_resid"] <= 1e-7
            assert sl["outer_iters"] == 1, sl             # no fallback needed
            assert sl["iters"] < sj["iters"], (sl, sj)
            d = (xl - xj).abs().max().item() / xj.abs().max().item()
            assert d <= 1e-6
        finally:
            fe.fe_lpc_destroy(lpc)


@pytest.mark.parametrize("width,sigma", [(0, None), (128, None), (0, 1.0), (256, None)])
def test_fcg_ir_learned_mixed_precision(width, sigma):
    """Mixed-precision refinement around the FP32 learned-FCG inner solve reaches the
    FP64-accurate 1e-8 residual and the Jacobi-PCG solution."""
    torch = torch_cuda()
    n, p = 16, 3
    with gpu_problem(n, n, n, p, sigma=sigma, ops=1) as (fe, mesh, pa, V, c):
        fe.fe_pa_set_variant(pa, "f32x2")
        nd, _, _ = fe.fe_mesh_sizes(mesh)
        b = torch.empty(nd, dtype=torch.float64, device="cuda")
        fe.fe_load_vector_sine(pa, b)
        xj, xi = torch.empty_like(b), torch.empty_like(b)
        st, sj = fe.fe_pcg(pa, fe.FE_DIFFUSION, fe.FE_PC_JACOBI, b, xj, 1e-8, 20000)
        assert st == fe.FE_OK
        lpc = fe.fe_lpc_create(pa, fe.FE_DIFFUSION, width, 4)
        try:
            fe.fe_lpc_train(lpc, 2000, 1024, 1e-3)
            st, si = fe.fe_fcg_ir(pa, fe.FE_DIFFUSION, lpc, b, xi, 1e-8, 20000)
            assert st == fe.FE_OK, fe.fe_last_error()
            assert si["true_rel_resid"] <= 1e-8 and si["outer_iters"] >= 2
            assert fe.fe_pa_get_variant(pa) == fe.VARIANTS["f32x2"]   # handle's variant kept
            d = (xi - xj).abs().max().item() / xj.abs().max().item()
            assert d <= 1e-6
        finally:
            fe.fe_lpc_destroy(lpc)


def test_fcg_ir_rejects_unsupported_width():
    """Order 4 (D^3 = 125) at width 256 has no FP32 fused kernel: its weights do not fit in
    shared memory beside a tcgen05 tile, and the mma.sync kernel is not built for it."""
    torch = torch_cuda()
    with gpu_problem(3, 3, 3, 4, ops=1) as (fe, mesh, pa, V, c):
        nd, _, _ = fe.fe_mesh_sizes(mesh)
        b = torch.ones(nd, dtype=torch.float64, device="cuda")
        x = torch.empty_like(b)
        lpc = fe.fe_lpc_create(pa, fe.FE_DIFFUSION, 256, 4)
        try:
            with pytest.raises(fe.FEError) as e:
                fe.fe_fcg_ir(pa, fe.FE_DIFFUSION, lpc, b, x, 1e-8, 100)
            assert e.value.status == fe.FE_ERR_UNSUPPORTED
            with pytest.raises(fe.FEError):
                fe.fe_fcg_ir(pa, fe.FE_DIFFUSION, lpc, b, x, 1e-8, 100, inner_rtol=1.5)
        finally:
            fe.fe_lpc_destroy(lpc)


def test_fit_linear_matches_adam_and_beats_jacobi():
    """The least-squares fit of the linear patch map (its symmetric part, exactly symmetric in
    FP32) reaches at most the relative loss of 2000 Adam steps on the same training set, and FCG
    with it beats Jacobi-PCG in iterations."""
    torch = torch_cuda()
    n, p = 16, 3
    with gpu_problem(n, n, n, p, ops=1) as (fe, mesh, pa, V, c):
        fe.fe_pa_set_variant(pa, "f32x2")
        nd, _, _ = fe.fe_mesh_sizes(mesh)
        b = torch.empty(nd, dtype=torch.float64, device="cuda")
        fe.fe_load_vector_sine(pa, b)
        x = torch.empty_like(b)
        st, sj = fe.fe_pcg(pa, fe.FE_DIFFUSION, fe.FE_PC_JACOBI, b, x, 1e-8, 20000)
        fit = fe.fe_lpc_create(pa, fe.FE_DIFFUSION, 0, 4)
        adam = fe.fe_lpc_create(pa, fe.FE_DIFFUSION, 0, 4)
        try:
            lf = fe.fe_lpc_fit_linear(fit, 1e-6)
            w0 = fe.fe_lpc_weights(fit).reshape(64, 64)
            assert np.array_equal(w0, w0.T)
            la = fe.fe_lpc_train(adam, 2000, 1024, 1e-3)
            assert 0.0 <= lf <= la * 1.05 + 1e-3, (lf, la)
            st, sf = fe.fe_fcg(pa, fe.FE_DIFFUSION, fit, b, x, 1e-8, 20000)
            assert st == fe.FE_OK and sf["outer_iters"] == 1
            assert sf["iters"] < sj["iters"], (sf, sj)
            with pytest.raises(fe.FEError):
                fe.fe_lpc_fit_linear(fit, -1.0)
        finally:
            fe.fe_lpc_destroy(fit)
            fe.fe_lpc_destroy(adam)
