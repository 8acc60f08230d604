#!/usr/bin/env python3
"""Benchmark of the partial-assembly hot path on GB300; prints ONE JSON line (rank 0).

Workload (one "step"): the 64^3-hex, p = 3 (Q = 5) Poisson problem on the +-0.1h perturbed unit
cube (7,189,057 dofs): Jacobi-preconditioned CG to a relative residual of 1e-8 from a zero guess,
through the C ABI (fe_pcg): diagonal assembly, boundary conditions, one fused PA diffusion apply
per iteration, FP64 vector updates and inner products, and the final true-residual apply.
Inputs (mesh, quadrature data, right-hand side) are resident in HBM before the timed region.

  value        GDOF/s = ndofs * (PCG applies) / time, summed over ranks: the apply throughput
               the solver sustains end to end on the device (every PCG kernel inside the time);
  ms_per_step  time of one PCG solve to 1e-8 (the metric's time-to-solution part);
  e2e          the same, through host buffers: one fe_pcg_host call per step (pinned b ->
               device, the solve, x -> pinned host, inside the library);
  roofline     of the dominant kernel (the fused apply), timed alone with CUDA events;
  cpu_baseline the CPU oracle (sum-factorised FP64 Jacobi-PCG in C/OpenMP) on a bounded sample
               of PCG iterations of the same workload, on every host core;
  pcg_ir       mixed-precision iterative refinement (FP32 inner PCG) to the same residual;
  pcg_chebyshev  Chebyshev-polynomial preconditioned CG (degree 4) to the same residual;
  learned_fcg  the learned element-patch preconditioner (trained on the GPU from the operator's
               own patch solves) inside flexible CG, to the same FP64 residual, against the
               Jacobi-PCG time above, with its fused BF16 tensor-core kernel timed alone;
               learned_fcg_linear the same with the linear patch map (width 0).

--impl reference times the CPU oracle alone (the reference of this build) on the same metric.
Multi-GPU (torchrun): every rank solves its own copy of the problem (independent problems, weak
scaling, no collective on the data path); rank 0 prints.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N_ELEM, ORDER, RTOL = 64, 3, 1e-8
MAXIT = 20000
METRIC = "GDOF/s of FP64 PA diffusion apply (frac of HBM roofline); PCG time-to-1e-8 residual"
UNIT = "GDOF/s"
FP64_DFMA_PER_CLK_PER_SM = 2           # measured on GB300 by fe_probe_throughput
EXTRA_STEPS = 5                        # timed repetitions of the secondary measurements
# DRAM bytes (read + write) of one apply launch from an ncu capture of the same kernel on a
# 32^3 mesh of the same order, with that launch's algorithmic bytes: scaled to the benchmark's
# launch by the algorithmic bytes (traffic grows with the elements).  Only for kernels
# unchanged since the capture; (variant, order) -> (dram bytes, algorithmic bytes, case).
NCU_TRAFFIC = {("f64", 3): (219.807744e6 + 4.559360e6, 219599376, "32^3 hexes, p = 3"),
               ("f32x2", 3): (220.169472e6 + 4.021248e6, 219599376, "32^3 hexes, p = 3"),
               ("mixed", 4, 3): (1401.652e6 + 188.421e6, 1505387536, "48^3 hexes, H1 p = 4 / L2 p = 3")}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def algorithmic(ndofs, ne, p, q, diffusion=True):
    """Minimum bytes and FP64 flops of one apply: x read once, y written once, the dof map and
    the quadrature data read once; flops of the sum-factorised contractions and the pointwise D."""
    D = p + 1
    qd = (6 if diffusion else 1) * q ** 3 * 8
    nbytes = 16 * ndofs + ne * (4 * D ** 3 + qd)
    if diffusion:
        f = 2 * (4 * q * D ** 3 + 6 * q * q * D * D + 6 * q ** 3 * D) + 15 * q ** 3
    else:
        f = 4 * (q * D ** 3 + q * q * D * D + q ** 3 * D) + q ** 3
    return nbytes, ne * f


def mixed_algorithmic(n, ph=4, pl=3):
    """Minimum bytes and FP64 flops of one fused application of the mixed pair (gradient and
    divergence blocks) on n^3 hexes: the 9 quadrature values per point read once, p and u read
    once, G p and G^T u written once, the H1 dof map once; flops of the sum-factorised
    contractions (H1 reference gradient forward and transposed, the L2 basis forward and
    transposed for three components) and the two 3x3 products per point."""
    Dh, Dl, Q = ph + 1, pl + 1, ph + 1
    ne = n ** 3
    nh = (n * ph + 1) ** 3
    nl = 3 * ne * Dl ** 3
    nbytes = ne * (9 * Q ** 3 * 8 + 4 * Dh ** 3) + 16 * nh + 16 * nl
    h1 = 2 * Q * Dh ** 3 + 3 * Q * Q * Dh * Dh + 3 * Q ** 3 * Dh
    l2 = 3 * (Q * Dl ** 3 + Q * Q * Dl * Dl + Q ** 3 * Dl)
    fma = 2 * (h1 + l2 + 9 * Q ** 3)
    return nbytes, 2 * ne * fma, nh, nl


def mixed_traffic(ph, pl, nbytes):
    """DRAM bytes of one fused mixed launch: the ncu capture's bytes scaled by algorithmic bytes
    (None for an order pair without a capture)."""
    if ("mixed", ph, pl) not in NCU_TRAFFIC:
        return None
    meas, algo, _ = NCU_TRAFFIC[("mixed", ph, pl)]
    return meas * nbytes / algo


def measure_mixed(fe, torch, n, stream, reps=10, ph=4, pl=3):
    """The paper's own operator (mixed H1 order 4 / L2 order 3 gradient and divergence pair) on
    n^3 perturbed hexes: the fused launch and each block alone (median of reps, CUDA events),
    GDOF/s of (H1 + L2) values per fused application, against the FP64-pipe and HBM roofs."""
    from paper_2603_09038_gb300.inputs import perturbed_vertices
    mx = fe.fe_mixed_setup(n, n, n, ph, pl, perturbed_vertices(n, n, n))
    try:
        nh, nl = fe.fe_mixed_sizes(mx)
        g = torch.Generator(device="cuda").manual_seed(2)
        p = torch.rand(nh, dtype=torch.float64, device="cuda", generator=g) * 2 - 1
        u = torch.rand(nl, dtype=torch.float64, device="cuda", generator=g) * 2 - 1
        gp = torch.empty(nl, dtype=torch.float64, device="cuda")
        gtu = torch.empty(nh, dtype=torch.float64, device="cuda")

        def timed(a, b, c, d):
            for _ in range(3):
                fe.fe_mixed_apply(mx, a, b, c, d, stream)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(reps)]
            torch.cuda.synchronize()
            for e0, e1 in ev:
                e0.record(stream)
                fe.fe_mixed_apply(mx, a, b, c, d, stream)
                e1.record(stream)
            torch.cuda.synchronize()
            return statistics.median(e0.elapsed_time(e1) for e0, e1 in ev)

        ms = timed(p, u, gp, gtu)
        ms_g = timed(p, None, gp, None)
        ms_d = timed(None, u, None, gtu)
    finally:
        fe.fe_mixed_destroy(mx)
    nbytes, flops, _, _ = mixed_algorithmic(n, ph, pl)
    peaks, src = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    fp64_peak = 152 * FP64_DFMA_PER_CLK_PER_SM * 2 * sm_max * 1e6 / 1e12
    achieved = flops / (ms * 1e-3) / 1e12
    return {"workload": "mixed_h1p%d_l2p%d_%dcubed" % (ph, pl, n), "ndof_h1": nh, "ndof_l2": nl,
            "dofs": nh + nl, "fused_ms": ms, "gradient_only_ms": ms_g, "divergence_only_ms": ms_d,
            "gdofs_fused": (nh + nl) / (ms * 1e-3) / 1e9,
            "fusion_speedup": (ms_g + ms_d) / ms, "dtype": "f64",
            "roofline": {"bound": "alu", "achieved": achieved, "peak": fp64_peak,
                         "unit": "TFLOP/s", "frac": achieved / fp64_peak,
                         "traffic": mixed_traffic(ph, pl, nbytes),
                         "traffic_source": "ncu dram bytes (read + write) of one launch on %s, scaled "
                                           "by algorithmic bytes" % NCU_TRAFFIC[("mixed", 4, 3)][2]
                                           if ("mixed", ph, pl) in NCU_TRAFFIC else None,
                         "kernel": "k_mixed_apply<DH=%d,DL=%d,Q=%d,grad+div>" % (ph + 1, pl + 1, ph + 1),
                         "peak_source": "FP64 pipe: 152 SMs x %d DFMA/clk x 2 flop x %.0f MHz"
                                        % (FP64_DFMA_PER_CLK_PER_SM, sm_max),
                         "flops_per_launch": flops, "bytes_per_launch": nbytes,
                         "hbm": {"achieved": nbytes / (ms * 1e-3) / 1e9,
                                 "peak": float(peaks.get("hbm_gbs", 6800.0)), "unit": "GB/s",
                                 "frac": nbytes / (ms * 1e-3) / 1e9 / float(peaks.get("hbm_gbs", 6800.0)),
                                 "peak_source": src}},
            "paper_context": "GB200 DMMA fused PA 46.60 GDOF/s, GH200 36.15 (FP64, 540 M DOF, "
                             "Table VI; other hardware)"}


def run_refinement(args, local_rank):
    """--refinement on --n^3 hexes of order --p (the mixed-precision configuration is --n 96
    --p 4; manufactured sine load, Jacobi, rtol 1e-8): FP64 Jacobi-PCG, float-float Jacobi-PCG
    and the refinement
    (FP32 inner PCG, FP64 outer residual), each timed with CUDA events; every answer's FP64 true
    residual and its difference from the FP64 solve; one JSON line."""
    import torch
    from paper_2603_09038_gb300 import fe
    from paper_2603_09038_gb300.inputs import perturbed_vertices
    torch.cuda.set_device(local_rank)
    fe.load()
    n, p = args.n, args.p
    mesh = fe.fe_mesh_setup(n, n, n, p, perturbed_vertices(n, n, n))
    pa = fe.fe_pa_setup(mesh, 0, None, fe.FE_DIFFUSION)
    nd, ne, _ = fe.fe_mesh_sizes(mesh)
    stream = torch.cuda.current_stream()
    b = torch.empty(nd, dtype=torch.float64, device="cuda")
    fe.fe_load_vector_sine(pa, b)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {"refinement": True, "workload": "poisson_%dcubed_p%d_jacobi" % (n, p), "ndofs": nd,
           "rtol": args.rtol}
    xs = {}
    for name, variant in (("fp64_pcg", "f64"), ("ff_pcg", "f32x2"), ("ir_f32_inner", "f64")):
        fe.fe_pa_set_variant(pa, variant)
        x = torch.empty_like(b)

        def run():
            if name == "ir_f32_inner":
                return fe.fe_pcg_ir(pa, fe.FE_DIFFUSION, fe.FE_PC_JACOBI, b, x, args.rtol, MAXIT,
                                    args.inner_rtol, stream)
            return fe.fe_pcg(pa, fe.FE_DIFFUSION, fe.FE_PC_JACOBI, b, x, args.rtol, MAXIT, stream)
        run()                                           # warm-up (workspace, copies)
        torch.cuda.synchronize()
        e0.record(stream)
        st, stats = run()
        e1.record(stream)
        torch.cuda.synchronize()
        xs[name] = x
        out[name] = {"status": st, "time_s": e0.elapsed_time(e1) / 1e3, "iters": stats["iters"],
                     "outer_iters": stats["outer_iters"], "true_rel_resid": stats["true_rel_resid"],
                     "variant": variant if name != "ir_f32_inner" else "f32 inner, f64 outer"}
    ref = xs["fp64_pcg"]
    for name in ("ff_pcg", "ir_f32_inner"):
        out[name]["x_vs_fp64_pcg"] = float((xs[name] - ref).abs().max()) / float(ref.abs().max())
        out[name]["speedup_vs_fp64_pcg"] = out["fp64_pcg"]["time_s"] / out[name]["time_s"]
    out["ir_f32_inner"]["speedup_vs_ff_pcg"] = out["ff_pcg"]["time_s"] / out["ir_f32_inner"]["time_s"]
    fe.fe_pa_destroy(pa)
    fe.fe_mesh_destroy(mesh)
    print(json.dumps(out))
    return 0


def c5_learned(fe, torch, vs, b, args, sigma, s_pcg, t_pcg, stream, width=0, n_train=16):
    """C5's learned leg: for each order of the space a patch network -- width 0: the linear map
    fitted by least squares (fe_lpc_fit_linear); else the MLP of that width trained by --lpc-steps
    Adam steps (fe_lpc_train) -- on operator-generated local-solve pairs of an n_train^3
    single-order mesh with the same log-normal coefficient distribution, attached to the space's
    order group (fe_vspace_set_learned), then flexible CG on the first right-hand side to --rtol
    against the single-system Jacobi-PCG above (iterations, time with CUDA events, FP64 true
    residual)."""
    from paper_2603_09038_gb300.inputs import perturbed_vertices, lognormal_coefficient
    t0 = time.perf_counter()
    fits = {}
    for p in (2, 4, 6):
        V = perturbed_vertices(n_train, n_train, n_train, seed=11)
        cm = torch.from_numpy(lognormal_coefficient(n_train ** 3, sigma)).cuda()
        mesh = fe.fe_mesh_setup(n_train, n_train, n_train, p, V)
        pa = fe.fe_pa_setup(mesh, 0, cm, fe.FE_DIFFUSION)
        lpc = fe.fe_lpc_create(pa, fe.FE_DIFFUSION, width, 5)
        try:
            if width == 0:
                fits[p] = fe.fe_lpc_fit_linear(lpc)
            else:
                fits[p] = fe.fe_lpc_train(lpc, args.lpc_steps, 1024, 1e-3)
            fe.fe_vspace_set_learned(vs, fe.FE_DIFFUSION, p, lpc)
        finally:
            fe.fe_lpc_destroy(lpc)
            fe.fe_pa_destroy(pa)
            fe.fe_mesh_destroy(mesh)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    x = torch.empty_like(b)
    fe.fe_vspace_fcg(vs, fe.FE_DIFFUSION, b, x, args.rtol, 20, stream)     # warm-up
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    st, sf = fe.fe_vspace_fcg(vs, fe.FE_DIFFUSION, b, x, args.rtol, MAXIT, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3
    kind = ("linear patch map per order (width 0), fitted by least squares" if width == 0 else
            "MLP per order (3 layers and a linear skip term, width %d, BF16), %d Adam steps"
            % (width, args.lpc_steps))
    return {"preconditioner": kind + " on %d^3 single-order meshes, log-normal sigma %g"
                                     % (n_train, sigma),
            "width": width, ("fit_relative_loss" if width == 0 else "final_batch_loss"): fits,
            "setup_s": t_setup, "status": st,
            "fcg_iters": sf["iters"],
            "time_s": t, "ms_per_iter": 1e3 * t / max(1, sf["iters"]),
            "true_rel_resid": sf["true_rel_resid"], "fallbacks_to_jacobi": sf["outer_iters"] - 1,
            "jacobi_pcg_iters": s_pcg["iters"], "jacobi_pcg_time_s": t_pcg,
            "speedup_vs_jacobi_pcg": t_pcg / t if t > 0 else None}


def run_c5(args, local_rank):
    """--c5: the batched configuration on the variable-order space: --n^3 hexes (64) in 8^3-element
    blocks of orders 2, 4, 6 (seed 7), log-normal coefficient sigma = --sigma (2), 16 right-hand
    sides U[-1, 1] (seeds 100..115), float-float arithmetic.  One single-system Jacobi-PCG solve
    to --rtol gives the iteration count and time; the 16 systems in lockstep
    (fe_vspace_pcg_batched: one persistent launch over all orders and right-hand sides per
    iteration, iteration batches replayed as CUDA graphs) run a bounded number of iterations
    (--c5-iters), timed with CUDA events; the time to the tolerance for all 16 is extrapolated
    from that per-iteration time and the single solve's iteration count.  One JSON line."""
    import numpy as np
    import torch
    from paper_2603_09038_gb300 import fe
    from paper_2603_09038_gb300.inputs import (block_orders, perturbed_vertices,
                                               lognormal_coefficient, uniform_vector)
    torch.cuda.set_device(local_rank)
    fe.load()
    n, nr = args.n, 16
    sigma = args.sigma if args.sigma else 2.0
    orders = block_orders(n, n, n, block=8, orders=(2, 4, 6), seed=7)
    c = lognormal_coefficient(n ** 3, sigma)
    vs = fe.fe_vspace_setup(n, n, n, orders, perturbed_vertices(n, n, n), c, ops=fe.FE_DIFFUSION)
    fe.fe_vspace_set_variant(vs, "f32x2")
    ntrue, _, _ = fe.fe_vspace_sizes(vs)
    stream = torch.cuda.current_stream()
    B = torch.from_numpy(np.stack([uniform_vector(ntrue, seed=100 + j) for j in range(nr)])).cuda()
    X = torch.empty_like(B)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    x1 = torch.empty(ntrue, dtype=torch.float64, device="cuda")
    fe.fe_vspace_pcg(vs, fe.FE_DIFFUSION, B[0].contiguous(), x1, args.rtol, 20)    # warm-up
    torch.cuda.synchronize()
    e0.record(stream)
    st1, s1 = fe.fe_vspace_pcg(vs, fe.FE_DIFFUSION, B[0].contiguous(), x1, args.rtol, MAXIT, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    t1 = e0.elapsed_time(e1) / 1e3
    kb = min(args.c5_iters, s1["iters"])
    fe.fe_vspace_pcg_batched(vs, fe.FE_DIFFUSION, nr, B, ntrue, X, ntrue, args.rtol, 16, stream)
    torch.cuda.synchronize()
    e0.record(stream)
    stb, sb = fe.fe_vspace_pcg_batched(vs, fe.FE_DIFFUSION, nr, B, ntrue, X, ntrue, args.rtol, kb,
                                       stream)
    e1.record(stream)
    torch.cuda.synchronize()
    tb = e0.elapsed_time(e1) / 1e3
    per_iter_b = tb / kb
    per_iter_1 = t1 / max(1, s1["iters"])
    out = {"c5": True, "workload": "diffusion_%dcubed_blocks8_orders246_sigma%g_16rhs" % (n, sigma),
           "ntrue": ntrue, "nrhs": nr, "variant": "f32x2", "rtol": args.rtol,
           "single": {"status": st1, "iters": s1["iters"], "time_s": t1,
                      "true_rel_resid": s1["true_rel_resid"], "ms_per_iter": 1e3 * per_iter_1},
           "batched": {"iters_run": kb, "time_s": tb, "ms_per_iter_16rhs": 1e3 * per_iter_b,
                       "ms_per_iter_per_rhs": 1e3 * per_iter_b / nr,
                       "launches": sb[0]["launches"], "rel_resid_after": [x["rel_resid"] for x in sb],
                       "apply": "one persistent launch over orders 2, 4, 6 and 16 right-hand "
                                "sides per iteration; iteration batches replayed as CUDA graphs"},
           "estimate_16_systems_to_rtol_s": {"batched": per_iter_b * s1["iters"],
                                             "one_by_one": nr * t1},
           "speedup_batched_vs_one_by_one": (nr * t1) / (per_iter_b * s1["iters"]),
           "gdofs_per_rhs_iteration_batched": ntrue * nr / per_iter_b / 1e9,
           "learned": c5_learned(fe, torch, vs, B[0].contiguous(), args, sigma, s1, t1, stream)}
    if args.lpc_width > 0:   # the configured network (C5 names 3 layers of width 256)
        out["learned_mlp"] = c5_learned(fe, torch, vs, B[0].contiguous(), args, sigma, s1, t1,
                                        stream, width=args.lpc_width)
    fe.fe_vspace_destroy(vs)
    print(json.dumps(out))
    return 0


def run_mixed_h1l2(args, local_rank):
    """--mixed-h1l2: only the paper's own operator (mixed H1/L2 pair) on --n^3 hexes."""
    import torch
    from paper_2603_09038_gb300 import fe
    torch.cuda.set_device(local_rank)
    fe.load()
    out = {"mixed_h1l2": True}
    out.update(measure_mixed(fe, torch, args.n, torch.cuda.current_stream()))
    print(json.dumps(out))
    return 0


def max_over_ranks(t, dist=None, device="cpu"):
    """Slowest rank's time: every rank gets max_r t_r (identity on one process)."""
    if dist is None:
        return float(t)
    import torch
    tt = torch.tensor([float(t)], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def job_gdofs(world, ndofs, applies, seconds):
    """Whole-job throughput: every rank solves its own problem (weak scaling), so the units are
    world * ndofs * applies, over the slowest rank's time."""
    return world * ndofs * applies / seconds / 1e9


def parse_clock_samples(text, reasons_names=("hw_slowdown", "hw_thermal_slowdown",
                                              "sw_thermal_slowdown", "sw_power_cap")):
    """Summary of `nvidia-smi --query-gpu=clocks.sm,clocks.max.sm,power.draw,<5 reason columns>
    --format=csv,noheader,nounits` lines: median SM clock under load, the maximum clock, the
    throttle reasons seen Active, and the median board power (W) when it is reported."""
    sm, mx, pw, reasons = [], [], [], set()
    for line in text.splitlines():
        f = [x.strip() for x in line.split(",")]
        if len(f) < 8:
            continue
        try:
            sm.append(float(f[0]))
            mx.append(float(f[1]))
        except ValueError:
            continue
        try:
            pw.append(float(f[2]))
        except ValueError:
            pass
        for name, val in zip(reasons_names, f[4:8]):
            if val.lower() == "active":
                reasons.add(name)
    if not sm:
        return None
    out = {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
           "reasons": sorted(reasons)}
    if pw:
        out["power_w"] = statistics.median(pw)
    return out


class ClockSampler:
    """nvidia-smi clock/throttle/power sampling during the timed region (200 ms period)."""

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.result = None
        if self.proc is None:
            return False
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        self.result = parse_clock_samples(out)
        return False


class CpuOracle:
    """The oracle's sum-factorised FP64 operator and Jacobi-PCG in C with OpenMP over elements
    (oracle/sumfact_omp.c, as it stands) on the benchmark's own workload: the 64^3 p=3 Poisson
    mesh, right-hand side and stopping rule, on every host core.  Set-up (quadrature data, Jacobi
    diagonal, load vector) is untimed; a sample is a bounded number of PCG iterations."""

    def __init__(self, n=N_ELEM, p=ORDER):
        import numpy as np
        from oracle import sumfact_c
        from oracle.mesh import boundary_mask
        from paper_2603_09038_gb300.inputs import perturbed_vertices
        self.n, self.p = n, p
        V = perturbed_vertices(n, n, n)
        self.op = sumfact_c.Operator(n, n, n, p, V, "diffusion")
        self.mask = boundary_mask(n, n, n, p)
        self.diag = self.op.diagonal()
        self.diag[self.mask == 1] = 1.0
        # any b with the workload's structure serves for timing (the iteration count is fixed)
        self.b = self.op.apply(np.ones(self.op.ndofs)) + 1.0
        self.cores = sumfact_c.threads()
        self.t_iter = self.iterate(1)[0]

    def iterate(self, k):
        t0 = time.perf_counter()
        _, it, _ = self.op.pcg(self.b, self.mask, self.diag, 0.0, k)
        return time.perf_counter() - t0, it

    def sample(self, budget_s):
        """PCG iterations for about budget_s seconds: GDOF/s = ndofs x applies / time."""
        k = max(1, int(round(budget_s / max(self.t_iter, 1e-6))))
        sec, it = self.iterate(k)
        gdofs = self.op.ndofs * it / sec / 1e9
        return {"value": gdofs, "unit": UNIT, "cores": self.cores, "kind": "oracle",
                "sample": "oracle sum-factorised FP64 diffusion apply + Jacobi-PCG in C with "
                          "OpenMP over elements (8 colours) on all %d host threads: %d PCG "
                          "iterations (%d applies) of the %d^3 p=%d workload (%d dofs) in %.1f s; "
                          "%.3f s per iteration" % (self.cores, it, it, self.n, self.p,
                                                    self.op.ndofs, sec, sec / max(1, it)),
                "seconds": sec, "applies": it, "s_per_iteration": sec / max(1, it)}


def cpu_oracle_sample(budget_s=12.0):
    return CpuOracle().sample(budget_s)


def run_reference(args, rank, world):
    """--impl reference: the CPU oracle (sum-factorised C/OpenMP Jacobi-PCG) on the same
    workload, metric and unit; every step is a bounded sample of PCG iterations.  Only rank 0
    runs it; the other ranks exit without work."""
    if rank != 0:
        return 0
    oracle = CpuOracle()
    per_step = []
    budget = max(1.0, min(12.0, 60.0 / max(1, args.steps + args.warmup)))
    for i in range(args.warmup + args.steps):
        r = oracle.sample(budget)
        if i >= args.warmup:
            per_step.append(r)
    tot_t = sum(r["seconds"] for r in per_step)
    applies = sum(r["applies"] for r in per_step)
    value = oracle.op.ndofs * applies / tot_t / 1e9
    last = per_step[-1]
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1000.0 * tot_t / len(per_step), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "impl": "reference",
           "config": {"workload": "poisson_%dcubed_p%d_jacobi_pcg" % (oracle.n, oracle.p),
                      "elements": oracle.n ** 3, "order": oracle.p, "q1d": oracle.p + 2,
                      "ndofs": oracle.op.ndofs, "parallelism": "cpu",
                      "step": "a bounded sample of Jacobi-PCG iterations (%.1f s budget)" % budget,
                      "s_per_pcg_iteration": tot_t / max(1, applies)},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": last["cores"],
                            "kind": "oracle", "sample": last["sample"]},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


def dtype_of(variant):
    """Arithmetic type the apply computes in: FP64 for the FMA and DMMA kernels, float-float
    pairs for f32x2."""
    return {"f64": "f64", "dmma": "f64", "f32x2": "f32x2"}[variant]


def apply_roofline(ndofs, ne, p, q, ms, variant, hbm_peak, sm_max, peak_src):
    """Roofline object of one fused diffusion apply of `ms` milliseconds: ALU-bound against the
    FP64 pipe (f64, dmma) or the FP32 issue rate of the anchored float-float step (f32x2), with
    the HBM fraction of the algorithmic bytes beside it."""
    nbytes, flops = algorithmic(ndofs, ne, p, q, True)
    achieved = flops / (ms * 1e-3) / 1e12
    hbm = {"achieved": nbytes / (ms * 1e-3) / 1e9, "peak": hbm_peak, "unit": "GB/s",
           "frac": nbytes / (ms * 1e-3) / 1e9 / hbm_peak, "peak_source": peak_src}
    if variant in ("f64", "dmma"):
        peak = 152 * FP64_DFMA_PER_CLK_PER_SM * 2 * sm_max * 1e6 / 1e12
        src = ("FP64 pipe: 152 SMs x %d DFMA/clk x 2 flop x %.0f MHz (DFMA rate measured on "
               "GB300)" % (FP64_DFMA_PER_CLK_PER_SM, sm_max))
    else:
        peak = 152 * 128 * sm_max * 1e6 / 6 * 2 / 1e12
        src = ("FP32 pipe: 152 SMs x 128 lanes x %.0f MHz / 6 instructions per anchored "
               "float-float multiply-add x 2 flop (FP64-equivalent)" % sm_max)
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": None,
            "kernel": "k_pa_apply<D=%d,Q=%d,diffusion,%s>" % (p + 1, q, variant),
            "peak_source": src, "hbm": hbm, "bytes_per_launch": nbytes,
            "flops_per_launch": flops, "launch_ms": ms}
    key = (variant, p)
    if key in NCU_TRAFFIC:
        meas, algo, case = NCU_TRAFFIC[key]
        roof["traffic"] = meas * nbytes / algo
        roof["traffic_source"] = ("ncu dram bytes (read + write) of one launch of the same kernel "
                                  "on %s, scaled by algorithmic bytes" % case)
    return roof


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch
    from paper_2603_09038_gb300 import fe
    from paper_2603_09038_gb300.inputs import perturbed_vertices

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    fe.load()
    dist = None
    if world > 1:
        import torch.distributed as dist

    def barrier():
        if dist is not None:
            dist.barrier()

    n, p = args.n, args.p
    V = perturbed_vertices(n, n, n)
    mesh = fe.fe_mesh_setup(n, n, n, p, V)
    pa = fe.fe_pa_setup(mesh, 0, None, fe.FE_DIFFUSION)
    fe_mesh_of[pa] = mesh
    ndofs, ne, _ = fe.fe_mesh_sizes(mesh)
    q = p + 2
    stream = torch.cuda.current_stream()
    ff = "f32x2"          # the fastest FP64-accurate arithmetic on this chip (float-float)
    fe.fe_pa_set_variant(pa, ff)           # make the float-pair copy before any timing
    fe.fe_pa_set_variant(pa, args.variant)
    b = torch.empty(ndofs, dtype=torch.float64, device=dev)
    x = torch.empty_like(b)
    fe.fe_load_vector_sine(pa, b)
    torch.cuda.synchronize()
    extra = max(1, min(args.steps, EXTRA_STEPS))

    def solve(pc=fe.FE_PC_JACOBI):
        st, stats = fe.fe_pcg(pa, fe.FE_DIFFUSION, pc, b, x, args.rtol, MAXIT, stream)
        if st != fe.FE_OK:
            raise RuntimeError("fe_pcg failed: %d %s" % (st, fe.fe_last_error()))
        return stats

    def timed_solves(fn, reps, warm):
        for _ in range(warm):
            fn()
        barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        out_ = [fn() for _ in range(reps)]
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        return max_over_ranks(e0.elapsed_time(e1) / 1000.0, dist, dev), out_

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(args.warmup):
        solve()
    torch.cuda.synchronize()

    # ---- timed region: K PCG solves with the headline arithmetic, CUDA events on the stream
    smi_index = int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local_rank)).split(",")[0]) \
        if os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[0].isdigit() else local_rank
    applies, iters, launches = 0, [], 0
    with ClockSampler(smi_index) as clk:
        barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            s_ = solve()
            applies += s_["iters"] + 1
            iters.append(s_["iters"])
            launches += s_["launches"]
            last_stats = s_
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
    t = max_over_ranks(e0.elapsed_time(e1) / 1000.0, dist, dev)
    value = job_gdofs(world, ndofs, applies, t)
    x_head = x.clone()

    # ---- end to end through host buffers, one C-ABI call per step (fe_pcg_host: pinned b ->
    #      device, the solve, x -> pinned host, all inside the library)
    b_host = b.cpu().pin_memory()
    x_host = torch.empty(ndofs, dtype=torch.float64).pin_memory()
    e2e_applies = 0
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(extra):
        st_, s_ = fe.fe_pcg_host(pa, fe.FE_DIFFUSION, fe.FE_PC_JACOBI, b_host, x_host, args.rtol,
                                 MAXIT, stream)
        if st_ != fe.FE_OK:
            raise RuntimeError("fe_pcg_host failed: %d %s" % (st_, fe.fe_last_error()))
        e2e_applies += s_["iters"] + 1
    te = time.perf_counter() - t0
    e2e_dx = float((x_host.to(dev) - x_head).abs().max()) / float(x_head.abs().max())
    barrier()
    te = max_over_ranks(te, dist, dev)
    e2e = {"value": job_gdofs(world, ndofs, e2e_applies, te), "unit": UNIT,
           "h2d_bytes_per_step": 8 * ndofs, "d2h_bytes_per_step": 8 * ndofs,
           "ms_per_step": 1000.0 * te / extra, "steps": extra, "call": "fe_pcg_host",
           "x_vs_device_solve": e2e_dx}

    # ---- the same Jacobi-PCG with the float-float arithmetic (FP64-accurate, FP32 pipe): FP64
    #      vectors, inner products and exit residual; its answer against the FP64 one above
    fe.fe_pa_set_variant(pa, ff)
    t_ff, ff_stats = timed_solves(solve, extra, 1)
    t_ff /= extra
    ff_dx = float((x - x_head).abs().max()) / float(x_head.abs().max())

    # ---- mixed-precision iterative refinement to the same 1e-8 FP64 residual: FP32 inner
    #      Jacobi-PCG, FP64 outer residual
    def solve_ir():
        st, stats = fe.fe_pcg_ir(pa, fe.FE_DIFFUSION, fe.FE_PC_JACOBI, b, x, args.rtol, MAXIT,
                                 args.inner_rtol, stream)
        if st != fe.FE_OK:
            raise RuntimeError("fe_pcg_ir failed: %d %s" % (st, fe.fe_last_error()))
        return stats
    t_ir, ir_stats = timed_solves(solve_ir, extra, 2)
    t_ir /= extra
    pcg_ir = {"time_to_1e-8_s": t_ir, "speedup_vs_fp64_pcg": (t / args.steps) / t_ir,
              "speedup_vs_ff_pcg": t_ff / t_ir,
              "inner_iters": ir_stats[-1]["iters"], "outer_iters": ir_stats[-1]["outer_iters"],
              "inner_rtol": args.inner_rtol or 1e-2,
              "true_rel_resid": ir_stats[-1]["true_rel_resid"],
              "outer_operator": "f64", "inner_operator": "f32",
              "x_vs_fp64_pcg": float((x - x_head).abs().max()) / float(x_head.abs().max())}

    # ---- Chebyshev-polynomial preconditioned CG (degree 4, [1.1 lmax/30, 1.1 lmax], lmax by
    #      20 power steps on the first solve, cached) to the same 1e-8 residual, float-float
    t_ch, cheb_stats = timed_solves(lambda: solve(fe.FE_PC_CHEBYSHEV), extra, 2)
    t_ch /= extra
    pcg_cheb = {"time_to_1e-8_s": t_ch, "speedup_vs_ff_pcg": t_ff / t_ch, "variant": ff,
                "iters": cheb_stats[-1]["iters"], "degree": 4, "applies_per_iter": 4,
                "lmax_estimate": fe.fe_estimate_lmax(pa, fe.FE_DIFFUSION, 20),
                "true_rel_resid": cheb_stats[-1]["true_rel_resid"]}

    # ---- learned patch preconditioner inside flexible CG, to the same FP64 1e-8 residual
    learned = learned_linear = None
    if args.lpc_width > 0:
        learned = learned_fcg(fe, pa, b, x, args, stream, dist, dev, t_ff,
                              ff_stats[-1]["iters"])
        learned_linear = learned_fcg(fe, pa, b, x, args, stream, dist, dev, t_ff,
                                     ff_stats[-1]["iters"], width=0)

    # ---- the dominant kernel alone: fused diffusion apply, CUDA events on its stream
    def time_apply(variant, reps):
        fe.fe_pa_set_variant(pa, variant)
        xa = torch.rand(ndofs, dtype=torch.float64, device=dev) * 2 - 1
        ya = torch.empty_like(xa)
        for _ in range(3):
            fe.fe_apply(pa, fe.FE_DIFFUSION, variant, xa, ya, stream)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(reps)]
        torch.cuda.synchronize()
        for a, z in ev:
            a.record(stream)
            fe.fe_apply(pa, fe.FE_DIFFUSION, variant, xa, ya, stream)
            z.record(stream)
        torch.cuda.synchronize()
        return statistics.median(a.elapsed_time(z) for a, z in ev)

    peaks, peak_src = measured_peaks()
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    kernels = {}
    nbytes, flops = algorithmic(ndofs, ne, p, q, True)
    nbytes32 = 16 * ndofs + ne * (4 * (p + 1) ** 3 + 4 * 6 * q ** 3)   # FP32 quadrature data
    for variant in ("f64", "f32x2", "dmma", "f32"):
        ms = time_apply(variant, 20)
        nb = nbytes32 if variant == "f32" else nbytes
        kernels[variant] = {
            "ms": ms, "gdofs": ndofs / (ms * 1e-3) / 1e9,
            "hbm_gbs": nb / (ms * 1e-3) / 1e9, "hbm_frac": nb / (ms * 1e-3) / 1e9 / hbm_peak,
            "fp64_tflops_equiv": flops / (ms * 1e-3) / 1e12,
        }
    autotune = None
    if world == 1:
        best, ms_at = fe.fe_pa_autotune(pa, fe.FE_DIFFUSION, 1, 10, stream)
        autotune = {"chosen": best, "ms": ms_at, "nrhs": 1}
    fe.fe_pa_set_variant(pa, args.variant)
    roof = apply_roofline(ndofs, ne, p, q, kernels[args.variant]["ms"], args.variant, hbm_peak,
                          sm_max, peak_src)
    roof["fp64_fma_probe_tflops"] = fe.fe_probe_throughput("fp64_fma")
    ff_pcg = {"time_to_1e-8_s": t_ff, "steps": extra, "variant": ff, "dtype": dtype_of(ff),
              "iters": ff_stats[-1]["iters"],
              "gdofs": ndofs * (ff_stats[-1]["iters"] + 1) / t_ff / 1e9,
              "speedup_vs_fp64_pcg": (t / args.steps) / t_ff,
              "true_rel_resid": ff_stats[-1]["true_rel_resid"],
              "x_vs_fp64_pcg": ff_dx,
              "apply_vs_fp64_apply": "parity-tested <= 1e-12 against the FP64 kernel and the "
                                     "oracle (tests); FP64 vectors, dots and exit residual",
              "roofline": apply_roofline(ndofs, ne, p, q, kernels[ff]["ms"], ff, hbm_peak,
                                         sm_max, peak_src)}

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1000.0 * t / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": dtype_of(args.variant), "data": "synthetic",
           "config": {"workload": "poisson_%dcubed_p%d_jacobi_pcg" % (n, p), "elements": ne,
                      "order": p,
                      "q1d": q, "ndofs": ndofs, "rtol": args.rtol, "preconditioner": "jacobi",
                      "variant": args.variant, "pcg_iters": iters[-1] if iters else None,
                      "applies_per_step": applies / max(1, args.steps),
                      "l2_flush": "inputs larger than L2 (1.57 GB quadrature data per apply)",
                      "parallelism": "independent problem per GPU"},
           "e2e": e2e, "gpu_launches": launches, "roofline": roof, "apply_kernel": kernels,
           "pcg_time_to_1e-8_s": t / args.steps, "ff_pcg": ff_pcg, "pcg_ir": pcg_ir,
           "pcg_chebyshev": pcg_cheb, "learned_fcg": learned,
           "learned_fcg_linear": learned_linear, "autotune": autotune,
           "true_rel_resid": last_stats["true_rel_resid"] if args.steps else None}
    if clk.result:
        out["clocks"] = clk.result
        if clk.result.get("power_w"):
            # the paper's energy metric (Table VI): MDOF/s per watt of board power
            out["mdof_per_w"] = 1000.0 * value / (world * clk.result["power_w"])
    fe.fe_pa_destroy(pa)
    fe.fe_mesh_destroy(mesh)
    if world == 1 and args.paper_operator_n > 0:
        # the paper's own operator (Table VI's mixed H1 p=4 / L2 p=3 pair) at its problem size
        torch.cuda.empty_cache()
        out["paper_operator"] = measure_mixed(fe, torch, args.paper_operator_n, stream)
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            cb = cpu_oracle_sample(args.cpu_seconds)
            out["cpu_baseline"] = {k2: cb[k2] for k2 in ("value", "unit", "cores", "kind", "sample")}
            # the same solve on the host cores: the oracle's time per iteration x this solve's
            out["cpu_baseline"]["time_to_1e-8_extrapolated_s"] = \
                cb["s_per_iteration"] * (iters[-1] if iters else 0)
        print(json.dumps(out))
    return 0


def learned_fcg(fe, pa, b, x, args, stream, dist, dev, t_pcg, pcg_iters, width=None, fit=False):
    """The learned element-patch preconditioner inside flexible CG to the same FP64 residual as
    Jacobi-PCG (time t_pcg, pcg_iters iterations): training (data generation from the operator's
    own patch solves + Adam, or with fit=True the least-squares fit of the linear map) timed once
    on the host clock, the solve timed with CUDA events like the PCG, and the fused BF16
    tensor-core preconditioner kernel alone (median of 20)."""
    import torch
    ndofs, ne, p = fe.fe_mesh_sizes(fe_mesh_of[pa])
    t0 = time.perf_counter()
    width = args.lpc_width if width is None else width
    lpc = fe.fe_lpc_create(pa, fe.FE_DIFFUSION, width, 1)
    if args.lpc_fallback == "chebyshev":
        fe.fe_lpc_set_fallback(lpc, fe.FE_PC_CHEBYSHEV)
    if fit:
        loss = fe.fe_lpc_fit_linear(lpc, 1e-6, 0, stream)
    else:
        loss = fe.fe_lpc_train(lpc, args.lpc_steps, 1024, 1e-3, 0, stream)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def solve_fcg(pc):
        st, stats = fe.fe_fcg(pa, fe.FE_DIFFUSION, pc, b, x, args.rtol, MAXIT, stream)
        if st not in (fe.FE_OK, fe.FE_ERR_NOT_CONVERGED):
            raise RuntimeError("fe_fcg failed: %d %s" % (st, fe.fe_last_error()))
        stats["status"] = st
        return stats

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        e0.record(stream)
        out_ = [fn() for _ in range(reps)]
        e1.record(stream)
        torch.cuda.synchronize()
        return max_over_ranks(e0.elapsed_time(e1) / 1000.0, dist, dev) / reps, out_[-1]

    t_fcg, s_fcg = timed(lambda: solve_fcg(lpc), max(1, min(args.steps, EXTRA_STEPS)))
    t_fj, s_fj = timed(lambda: solve_fcg(None), max(1, min(args.steps, EXTRA_STEPS)))
    r_ = torch.rand(ndofs, dtype=torch.float64, device=dev) * 2 - 1
    z_ = torch.empty_like(r_)

    def time_apply():
        for _ in range(3):
            fe.fe_lpc_apply(lpc, r_, z_, stream)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(20)]
        torch.cuda.synchronize()
        for a_, z2 in ev:
            a_.record(stream)
            fe.fe_lpc_apply(lpc, r_, z_, stream)
            z2.record(stream)
        torch.cuda.synchronize()
        return statistics.median(a_.elapsed_time(z2) for a_, z2 in ev)

    # the preconditioner apply alone with every built inference kernel; the solves above used
    # the default one
    kernel_used = fe.fe_lpc_get_kernel(lpc)[0]
    kernel_names = {fe.FE_LPC_KERNEL_TCGEN05: "tcgen05", fe.FE_LPC_KERNEL_MMA_SYNC: "mma_sync",
                    fe.FE_LPC_KERNEL_GEMM: "gemm"}
    ms_by_kernel = {}
    for k_, name_ in kernel_names.items():
        try:
            fe.fe_lpc_set_kernel(lpc, k_)
        except fe.FEError:
            continue
        ms_by_kernel[name_] = time_apply()
    fe.fe_lpc_set_kernel(lpc, fe.FE_LPC_KERNEL_AUTO)
    ms_lpc = ms_by_kernel[kernel_names[kernel_used]]
    tc_faults = fe.fe_lpc_get_kernel(lpc)[1]
    din, w = (p + 1) ** 3, width
    lpc_flops = 2.0 * ne * (2 * din * w + w * w + din * din)
    # algorithmic bytes: the dof map (int32) once, r and z (FP64) and the FP32 scaling once
    # per dof (the kernels read the map a second time in the scatter)
    lpc_bytes = ne * din * 4 + ndofs * (8 + 8 + 4)
    mma_peak = fe.fe_probe_throughput("bf16_mma")
    bf16_peak = float(measured_peaks()[0].get("bf16_tflops", 1900.0))
    # the same preconditioner inside mixed-precision refinement, where an FP32 kernel is built
    def solve_ir():
        st, stats = fe.fe_fcg_ir(pa, fe.FE_DIFFUSION, lpc, b, x, args.rtol, MAXIT,
                                 args.inner_rtol, stream)
        if st != fe.FE_OK:
            raise RuntimeError("fe_fcg_ir failed: %d %s" % (st, fe.fe_last_error()))
        return stats
    try:
        t_ir, s_ir = timed(solve_ir, max(1, min(args.steps, EXTRA_STEPS)))
        ir = {"time_to_1e-8_s": t_ir, "speedup_vs_jacobi_pcg": t_pcg / t_ir if t_pcg else None,
              "inner_iters": s_ir["iters"], "outer_iters": s_ir["outer_iters"],
              "true_rel_resid": s_ir["true_rel_resid"], "inner": "FP32 FCG + this network",
              "inner_rtol": args.inner_rtol or 1e-2,
              "outer_operator": "f64"}
    except (fe.FEError, RuntimeError) as exc:  # no FP32 kernel, or the solve failed
        ir = {"failed": str(exc).splitlines()[-1]}
    fe.fe_lpc_destroy(lpc)
    return {
        "mixed_precision_ir": ir,
        "time_to_1e-8_s": t_fcg, "speedup_vs_jacobi_pcg": t_pcg / t_fcg if t_pcg else None,
        "jacobi_pcg_time_s": t_pcg,
        "variant": {v: k for k, v in fe.VARIANTS.items()}[fe.fe_pa_get_variant(pa)],
        "fcg_iters": s_fcg["iters"], "fcg_status": s_fcg["status"], "jacobi_pcg_iters": pcg_iters,
        "fallbacks_to_jacobi": s_fcg["outer_iters"] - 1,
        "true_rel_resid": s_fcg["true_rel_resid"],
        "jacobi_fcg_time_s": t_fj, "jacobi_fcg_iters": s_fj["iters"],
        "train_s": t_train, "train": "least-squares fit" if fit else "Adam",
        "train_steps": 0 if fit else args.lpc_steps, "train_batch": 1024,
        "final_batch_loss": loss, "width": w, "patch": "element, %d dofs" % din,
        "fallback": args.lpc_fallback,
        "network": ("relu(relu(x W1) W2) W3 + x W0" if w else "x W0 (linear patch map)") +
                   ", BF16 weights/activations, FP32 accumulate",
        "precond_apply_ms": ms_lpc, "precond_tflops": lpc_flops / (ms_lpc * 1e-3) / 1e12,
        "precond_flops_per_launch": lpc_flops,
        "mma_sync_bf16_probe_tflops": mma_peak,
        "frac_of_mma_sync_peak": lpc_flops / (ms_lpc * 1e-3) / 1e12 / mma_peak,
        "frac_of_bf16_peak": lpc_flops / (ms_lpc * 1e-3) / 1e12 / bf16_peak,
        "precond_apply_ms_by_kernel": ms_by_kernel, "tcgen05_faults": tc_faults,
        "precond_bytes_per_launch": lpc_bytes,
        "precond_hbm_frac": lpc_bytes / (ms_lpc * 1e-3) / 1e9 /
                            float(measured_peaks()[0].get("hbm_gbs", 6800.0)),
        "kernel": {"tcgen05": "k_lpc_tc", "mma_sync": "k_lpc_fused", "gemm": "unfused GEMMs"}[
            kernel_names[kernel_used]] + "<DP=%d,W=%d>" % ((din + 15) // 16 * 16, w)}


fe_mesh_of = {}   # fe_pa handle -> its fe_mesh handle (for sizes)


def run_learned(args, local_rank):
    """--learned: only the learned-preconditioner comparison on an --n^3, order --p mesh with a
    log-normal coefficient of --sigma (0: Poisson), as one JSON line."""
    import torch
    from paper_2603_09038_gb300 import fe
    from paper_2603_09038_gb300.inputs import perturbed_vertices, lognormal_coefficient

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    fe.load()
    n, p = args.n, args.p
    mesh = fe.fe_mesh_setup(n, n, n, p, perturbed_vertices(n, n, n))
    c = torch.from_numpy(lognormal_coefficient(n ** 3, args.sigma)).to(dev) if args.sigma else None
    pa = fe.fe_pa_setup(mesh, 0, c, fe.FE_DIFFUSION)
    fe_mesh_of[pa] = mesh
    fe.fe_pa_set_variant(pa, args.variant)
    ndofs, ne, _ = fe.fe_mesh_sizes(mesh)
    stream = torch.cuda.current_stream()
    b = torch.empty(ndofs, dtype=torch.float64, device=dev)
    x = torch.empty_like(b)
    fe.fe_load_vector_sine(pa, b)
    st, s0 = fe.fe_pcg(pa, fe.FE_DIFFUSION, fe.FE_PC_JACOBI, b, x, args.rtol, MAXIT, stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(max(1, args.steps)):
        st, s0 = fe.fe_pcg(pa, fe.FE_DIFFUSION, fe.FE_PC_JACOBI, b, x, args.rtol, MAXIT, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    t_pcg = e0.elapsed_time(e1) / 1000.0 / max(1, args.steps)
    out = {"learned": True, "workload": "diffusion_%dcubed_p%d_sigma%g" % (n, p, args.sigma),
           "ndofs": ndofs, "variant": args.variant, "rtol": args.rtol}
    out.update(learned_fcg(fe, pa, b, x, args, stream, None, dev, t_pcg, s0["iters"]))
    out["linear"] = learned_fcg(fe, pa, b, x, args, stream, None, dev, t_pcg, s0["iters"], width=0)
    if args.lpc_fit:
        out["linear_fit"] = learned_fcg(fe, pa, b, x, args, stream, None, dev, t_pcg, s0["iters"],
                                        width=0, fit=True)
    fe.fe_pa_destroy(pa)
    fe.fe_mesh_destroy(mesh)
    print(json.dumps(out))
    return 0


def run_graphs(args, local_rank):
    """--graphs: Jacobi-PCG time to 1e-8 with the iteration batches replayed as CUDA graphs vs
    launched kernel by kernel, Poisson, p = --p, on meshes from 8^3 to --n^3 (one JSON line each)."""
    import torch
    from paper_2603_09038_gb300 import fe
    from paper_2603_09038_gb300.inputs import perturbed_vertices
    torch.cuda.set_device(local_rank)
    fe.load()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for n in [m for m in (8, 16, 32, 64) if m <= args.n]:
        mesh = fe.fe_mesh_setup(n, n, n, args.p, perturbed_vertices(n, n, n))
        pa = fe.fe_pa_setup(mesh, 0, None, fe.FE_DIFFUSION)
        fe.fe_pa_set_variant(pa, args.variant)
        nd, _, _ = fe.fe_mesh_sizes(mesh)
        b = torch.empty(nd, dtype=torch.float64, device="cuda")
        x = torch.empty_like(b)
        fe.fe_load_vector_sine(pa, b)
        out = {"graphs": True, "workload": "poisson_%dcubed_p%d" % (n, args.p), "ndofs": nd,
               "variant": args.variant}
        for mode in (1, 0):
            fe.fe_pcg_set_graphs(pa, mode)
            for _ in range(2):
                fe.fe_pcg(pa, fe.FE_DIFFUSION, fe.FE_PC_JACOBI, b, x, args.rtol, MAXIT, stream)
            torch.cuda.synchronize()
            reps = max(3, args.steps)
            e0.record(stream)
            for _ in range(reps):
                st, s_ = fe.fe_pcg(pa, fe.FE_DIFFUSION, fe.FE_PC_JACOBI, b, x, args.rtol, MAXIT, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            key = "graph" if mode else "eager"
            out[key + "_ms"] = e0.elapsed_time(e1) / reps
            out[key + "_iters"] = s_["iters"]
        out["speedup"] = out["eager_ms"] / out["graph_ms"]
        print(json.dumps(out), flush=True)
        fe.fe_pa_destroy(pa)
        fe.fe_mesh_destroy(mesh)
    return 0


def run_batched_pcg(args, local_rank):
    """--batched-pcg N: N right-hand sides solved by fe_pcg_batched (one batched apply per
    iteration) against N single fe_pcg solves, on the --n^3, order --p Poisson mesh."""
    import torch
    from paper_2603_09038_gb300 import fe
    from paper_2603_09038_gb300.inputs import perturbed_vertices
    torch.cuda.set_device(local_rank)
    fe.load()
    n, p, nr = args.n, args.p, args.batched_pcg
    mesh = fe.fe_mesh_setup(n, n, n, p, perturbed_vertices(n, n, n))
    pa = fe.fe_pa_setup(mesh, 0, None, fe.FE_DIFFUSION)
    fe.fe_pa_set_variant(pa, args.variant)
    nd, _, _ = fe.fe_mesh_sizes(mesh)
    stream = torch.cuda.current_stream()
    sine = torch.empty(nd, dtype=torch.float64, device="cuda")
    fe.fe_load_vector_sine(pa, sine)
    g = torch.Generator(device="cuda").manual_seed(5)
    B = torch.stack([sine * (1.0 + 0.1 * j) + 0.01 * torch.rand(nd, dtype=torch.float64,
                                                                  device="cuda", generator=g)
                     for j in range(nr)]).reshape(-1).contiguous()
    X = torch.empty_like(B)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fe.fe_pcg_batched(pa, fe.FE_DIFFUSION, fe.FE_PC_JACOBI, nr, B, nd, X, nd, args.rtol, MAXIT, stream)
    torch.cuda.synchronize()
    e0.record(stream)
    st, stats = fe.fe_pcg_batched(pa, fe.FE_DIFFUSION, fe.FE_PC_JACOBI, nr, B, nd, X, nd, args.rtol,
                                  MAXIT, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    t_b = e0.elapsed_time(e1) / 1000.0
    x1 = torch.empty(nd, dtype=torch.float64, device="cuda")
    fe.fe_pcg(pa, fe.FE_DIFFUSION, fe.FE_PC_JACOBI, B[:nd], x1, args.rtol, MAXIT, stream)
    torch.cuda.synchronize()
    e0.record(stream)
    iters1 = []
    for j in range(nr):
        st1, s1 = fe.fe_pcg(pa, fe.FE_DIFFUSION, fe.FE_PC_JACOBI, B[j * nd:(j + 1) * nd], x1,
                            args.rtol, MAXIT, stream)
        iters1.append(s1["iters"])
    e1.record(stream)
    torch.cuda.synchronize()
    t_s = e0.elapsed_time(e1) / 1000.0
    print(json.dumps({"batched_pcg": True, "workload": "poisson_%dcubed_p%d" % (n, p), "nrhs": nr,
                      "ndofs": nd, "variant": args.variant, "status": st,
                      "batched_s": t_b, "single_solves_s": t_s, "speedup": t_s / t_b,
                      "gdofs_per_rhs_iter_batched": nd * sum(x["iters"] for x in stats) / t_b / 1e9,
                      "iters_batched": [x["iters"] for x in stats], "iters_single": iters1,
                      "max_true_rel_resid": max(x["true_rel_resid"] for x in stats)}))
    fe.fe_pa_destroy(pa)
    fe.fe_mesh_destroy(mesh)
    return 0


def sweep_shapes(fe, pa, op, variant, spec):
    """Launch shapes to time: "all" (every built one) or a comma list of indices."""
    if variant == "dmma":
        return [0]
    _, nshapes, _, _ = fe.fe_pa_get_shape(pa, op, variant)
    if spec == "all":
        return list(range(nshapes))
    return [k for k in (int(v) for v in spec.split(",")) if k < nshapes]


def run_sweep(args, local_rank):
    """Order sweep p = 1..8 at ~50 M dofs (log-normal coefficient, sigma = 1; or meshes sized by
    --sweep-qd-gb): device time of one apply (median of --sweep-reps after --sweep-warm warm-ups,
    CUDA events) per operator and variant, one JSON line each.  Not the contract line: the
    per-order roofline table."""
    import torch
    from paper_2603_09038_gb300 import fe
    from paper_2603_09038_gb300.inputs import perturbed_vertices, lognormal_coefficient, ORDER_SWEEP_N
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    fe.load()
    peaks, _ = measured_peaks()
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    fp64_peak = 152 * FP64_DFMA_PER_CLK_PER_SM * 2 * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    stream = torch.cuda.current_stream()
    orders = [int(v) for v in args.orders.split(",")]
    ops = [(fe.FE_DIFFUSION, "diffusion"), (fe.FE_MASS, "mass")]
    ops = [o for o in ops if o[1] in args.sweep_ops.split(",")]
    for p in orders:
        n = ORDER_SWEEP_N[p]
        if args.sweep_qd_gb > 0:
            # a smaller mesh whose diffusion quadrature data take about --sweep-qd-gb GB (still
            # larger than L2), for the per-order ncu captures
            per_elem = 6 * (p + 2) ** 3 * 8
            n = max(4, int(round((args.sweep_qd_gb * 1e9 / per_elem) ** (1.0 / 3.0))))
        V = perturbed_vertices(n, n, n)
        c = torch.from_numpy(lognormal_coefficient(n ** 3, 1.0)).to(dev)
        mesh = fe.fe_mesh_setup(n, n, n, p, V)
        pa = fe.fe_pa_setup(mesh, 0, c, fe.FE_DIFFUSION | fe.FE_MASS)
        ndofs, ne, _ = fe.fe_mesh_sizes(mesh)
        x = torch.rand(ndofs, dtype=torch.float64, device=dev) * 2 - 1
        y = torch.empty_like(x)
        for variant, op, name, shape in (
                (v, o, nm, k) for v in args.variants.split(",") for o, nm in ops
                for k in sweep_shapes(fe, pa, o, v, args.sweep_shapes)):
            fe.fe_pa_set_variant(pa, variant)
            if variant != "dmma":
                fe.fe_pa_set_shape(pa, op, variant, shape)
            _, _, nt, nel = fe.fe_pa_get_shape(pa, op, variant)
            for _ in range(args.sweep_warm):
                fe.fe_apply(pa, op, variant, x, y, stream)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(args.sweep_reps)]
            torch.cuda.synchronize()
            for a, z in ev:
                a.record(stream)
                fe.fe_apply(pa, op, variant, x, y, stream)
                z.record(stream)
            torch.cuda.synchronize()
            ms = statistics.median(a.elapsed_time(z) for a, z in ev)
            nbytes, flops = algorithmic(ndofs, ne, p, p + 2, op == fe.FE_DIFFUSION)
            print(json.dumps({
                "sweep": True, "p": p, "n": n, "ndofs": ndofs, "op": name, "variant": variant,
                "shape": shape, "threads_per_block": nt, "elems_per_block": nel,
                "ms": round(ms, 4), "gdofs": ndofs / ms / 1e6,
                "hbm_gbs": nbytes / ms / 1e6, "hbm_frac": nbytes / ms / 1e6 / hbm_peak,
                "fp64_tflops_equiv": flops / ms / 1e9, "fp64_frac": flops / ms * 1e3 / fp64_peak}))
            sys.stdout.flush()
        fe.fe_pa_destroy(pa)
        fe.fe_mesh_destroy(mesh)
        del x, y, c
        torch.cuda.empty_cache()
    return 0


def run_batched(args, local_rank):
    """Batched apply on the 64^3 p=3 mesh: per-right-hand-side GDOF/s of one launch over nrhs
    right-hand sides against single applies, per variant (one JSON line each)."""
    import torch
    from paper_2603_09038_gb300 import fe
    from paper_2603_09038_gb300.inputs import perturbed_vertices
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    fe.load()
    n, p = args.n, args.p
    mesh = fe.fe_mesh_setup(n, n, n, p, perturbed_vertices(n, n, n))
    pa = fe.fe_pa_setup(mesh, 0, None, fe.FE_DIFFUSION)
    nd, ne, _ = fe.fe_mesh_sizes(mesh)
    stream = torch.cuda.current_stream()
    nr = args.batched
    X = torch.rand(nr, nd, dtype=torch.float64, device=dev) * 2 - 1
    Y = torch.empty_like(X)
    for variant in ("f32x2", "f32", "f64"):
        fe.fe_pa_set_variant(pa, variant)
        res = {}
        for k in (1, nr):
            for _ in range(2):
                fe.fe_apply_batched(pa, fe.FE_DIFFUSION, variant, k, X, nd, Y, nd, stream)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(5)]
            torch.cuda.synchronize()
            for a, z in ev:
                a.record(stream)
                fe.fe_apply_batched(pa, fe.FE_DIFFUSION, variant, k, X, nd, Y, nd, stream)
                z.record(stream)
            torch.cuda.synchronize()
            ms = statistics.median(a.elapsed_time(z) for a, z in ev)
            res[k] = k * nd / ms / 1e6
        print(json.dumps({"batched": True, "workload": "poisson_%dcubed_p%d" % (n, p),
                          "variant": variant, "nrhs": nr, "gdofs_single": res[1],
                          "gdofs_per_rhs_batched": res[nr], "speedup": res[nr] / res[1]}))
    fe.fe_pa_destroy(pa)
    fe.fe_mesh_destroy(mesh)
    return 0


def run_mixed_orders(args, local_rank):
    """Variable-order apply (fe_vspace_apply) on an n^3 mesh cut into 8^3-element blocks whose
    orders are drawn from {2, 4, 6}: the constraint gather E x, one fused apply per order, the
    transpose scatter E^T v.  One JSON line per variant: time, true-dof throughput, and the
    bytes moved (this design's and the minimum: x, y and the quadrature data once)."""
    import torch
    from paper_2603_09038_gb300 import fe
    from paper_2603_09038_gb300.inputs import block_orders, perturbed_vertices
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    fe.load()
    n = args.n
    orders = block_orders(n, n, n, block=8, orders=(2, 4, 6), seed=7)
    t0 = time.perf_counter()
    vs = fe.fe_vspace_setup(n, n, n, orders, perturbed_vertices(n, n, n), ops=fe.FE_DIFFUSION)
    setup_s = time.perf_counter() - t0
    ntrue, nlocal, nnz = fe.fe_vspace_sizes(vs)
    stream = torch.cuda.current_stream()
    x = torch.rand(ntrue, dtype=torch.float64, device=dev) * 2 - 1
    y = torch.empty_like(x)
    e = torch.empty(nlocal, dtype=torch.float64, device=dev)
    nc, cnnz, nct = fe.fe_vspace_constraint_sizes(vs)
    counts = {p: int((orders == p).sum()) for p in (2, 4, 6)}
    qd = sum(c * (p + 2) ** 3 * 6 * 8 for p, c in counts.items())
    dmap = 4 * nlocal
    # this design: x copied into X and y out of Y (16 B each way per dof), C x and C^T (offsets,
    # columns, weights, the constrained values), Y zeroed, X read and Y written once by the
    # kernels (the minimum their gather and scatter-add can move), maps and quadrature data once
    constraint = 2 * 12 * cnnz + 8 * (nc + 1) + 12 * (nct + 1) + 2 * 8 * nc + 16 * nct
    design = 2 * 16 * ntrue + constraint + 8 * (ntrue + nc) + 2 * 8 * (ntrue + nc) + qd + dmap
    minimum = 2 * 8 * ntrue + qd
    peaks, src = measured_peaks()

    def timed(fn, reps=10):
        for _ in range(3):
            fn()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(reps)]
        torch.cuda.synchronize()
        for a, z in ev:
            a.record(stream)
            fn()
            z.record(stream)
        torch.cuda.synchronize()
        return statistics.median(a.elapsed_time(z) for a, z in ev)

    for variant in args.variants.split(","):
        if variant == "dmma":
            continue
        fe.fe_vspace_set_variant(vs, variant)
        fe.fe_vspace_set_persistent(vs, 0)
        ms_per_order = timed(lambda: fe.fe_vspace_apply(vs, fe.FE_DIFFUSION, x, y, stream))
        fe.fe_vspace_set_persistent(vs, 1)
        ms = timed(lambda: fe.fe_vspace_apply(vs, fe.FE_DIFFUSION, x, y, stream))
        ms_gather = timed(lambda: fe.fe_vspace_prolong(vs, x, e, stream))
        print(json.dumps({
            "mixed_orders": True, "workload": "diffusion_%dcubed_blocks8_orders246" % n,
            "variant": variant, "ntrue": ntrue, "nlocal": nlocal, "nnz_E": nnz,
            "constrained_rows": nc, "nnz_C": cnnz,
            "elements_per_order": counts, "setup_s": setup_s, "apply_ms": ms,
            "apply": "one persistent launch over all orders",
            "apply_ms_one_launch_per_order": ms_per_order,
            "gdofs_true": ntrue / ms / 1e6, "gdofs_local": nlocal / ms / 1e6,
            "gather_ms": ms_gather, "design_bytes": design, "min_bytes": minimum,
            "design_gbs": design / ms / 1e6, "frac_of_hbm_design": design / ms / 1e6 / peaks["hbm_gbs"],
            "frac_of_hbm_min_bytes": minimum / ms / 1e6 / peaks["hbm_gbs"], "peak_source": src}))
        # Jacobi-PCG on the variable-order space to the benchmark tolerance (b ~ U[-1, 1])
        from paper_2603_09038_gb300.inputs import uniform_vector
        b = torch.from_numpy(uniform_vector(ntrue, seed=1)).to(dev)
        xs = torch.empty_like(b)
        fe.fe_vspace_pcg(vs, fe.FE_DIFFUSION, b, xs, args.rtol, 50)  # workspace, warm-up
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a0.record(stream)
        st, stats = fe.fe_vspace_pcg(vs, fe.FE_DIFFUSION, b, xs, args.rtol, MAXIT, stream)
        a1.record(stream)
        torch.cuda.synchronize()
        sec = a0.elapsed_time(a1) / 1e3
        print(json.dumps({
            "mixed_orders_pcg": True, "workload": "diffusion_%dcubed_blocks8_orders246" % n,
            "variant": variant, "status": st, "rtol": args.rtol, "iters": stats["iters"],
            "true_rel_resid": stats["true_rel_resid"], "time_to_rtol_s": sec,
            "gdofs_true": ntrue * (stats["iters"] + 1) / sec / 1e9,
            "ms_per_iteration": 1e3 * sec / max(1, stats["iters"])}))
    fe.fe_vspace_destroy(vs)
    return 0


def run_peaks(local_rank):
    """Throughput probes (libfe fe_probe_throughput) behind the FP64 roofline: one JSON line."""
    import torch
    from paper_2603_09038_gb300 import fe
    torch.cuda.set_device(local_rank)
    fe.load()
    out = {"peaks": True}
    for unit in ("fp64_fma", "fp64_dmma", "fp64_dfma_dmma", "fp32_fma", "f32x2_mac", "bf16_mma"):
        out[unit + "_tflops"] = fe.fe_probe_throughput(unit)
    props = torch.cuda.get_device_properties(local_rank)
    out["sms"] = props.multi_processor_count
    print(json.dumps(out))
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--variant", choices=["f64", "f32x2", "dmma"], default="f64",
                    help="arithmetic of the headline apply (f64: FP64 FMA; dmma: FP64 tensor "
                         "instruction; f32x2: float-float on the FP32 pipe, reported as ff_pcg "
                         "beside the FP64 headline by default)")
    ap.add_argument("--n", type=int, default=N_ELEM)
    ap.add_argument("--p", type=int, default=ORDER)
    ap.add_argument("--rtol", type=float, default=RTOL)
    ap.add_argument("--inner-rtol", type=float, default=0.0, help="fe_pcg_ir inner tolerance")
    ap.add_argument("--lpc-width", type=int, default=256,
                    help="width of the learned preconditioner's MLP (3 layers and a linear skip "
                         "term; 0: skip that comparison)")
    ap.add_argument("--lpc-steps", type=int, default=3000, help="Adam steps of its training")
    ap.add_argument("--lpc-fit", action="store_true",
                    help="--learned: also the linear map fitted by least squares (fe_lpc_fit_linear)")
    ap.add_argument("--lpc-fallback", choices=["jacobi", "chebyshev"], default="jacobi",
                    help="what FCG continues with once it gives the network up")
    ap.add_argument("--learned", action="store_true",
                    help="only the learned-preconditioner comparison (with --n, --p, --sigma)")
    ap.add_argument("--batched-pcg", type=int, default=0,
                    help="this many right-hand sides by fe_pcg_batched vs single solves")
    ap.add_argument("--graphs", action="store_true",
                    help="PCG with and without CUDA-graph replay on 8^3 .. --n^3 meshes")
    ap.add_argument("--sigma", type=float, default=0.0,
                    help="--learned: log-normal coefficient sigma (0: Poisson)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sweep", action="store_true", help="order sweep p=1..8 at ~50 M dofs")
    ap.add_argument("--orders", default="1,2,3,4,5,6,7,8")
    ap.add_argument("--sweep-ops", default="diffusion,mass", help="--sweep: operators")
    ap.add_argument("--sweep-warm", type=int, default=3, help="--sweep: untimed applies")
    ap.add_argument("--sweep-reps", type=int, default=10, help="--sweep: timed applies (median)")
    ap.add_argument("--sweep-shapes", default="0",
                    help="--sweep: launch shapes to time per variant (\"all\" or indices)")
    ap.add_argument("--sweep-qd-gb", type=float, default=0.0,
                    help="--sweep: size each order's mesh by this many GB of diffusion quadrature "
                         "data instead of ~50 M dofs (for ncu captures)")
    ap.add_argument("--peaks", action="store_true", help="FP64/DMMA/FP32/BF16-mma.sync throughput probes")
    ap.add_argument("--batched", type=int, default=0, help="batched apply with this many RHS")
    ap.add_argument("--variants", default="f64,f32x2,dmma")
    ap.add_argument("--refinement", action="store_true",
                    help="FP64 / float-float Jacobi-PCG vs mixed-precision refinement on --n^3, "
                         "order --p (the mixed-precision configuration is --n 96 --p 4)")
    ap.add_argument("--c5", action="store_true",
                    help="16 right-hand sides on the 64^3 orders-2/4/6 space, sigma 2 (batched)")
    ap.add_argument("--c5-iters", type=int, default=200,
                    help="--c5: lockstep iterations timed for the 16 systems")
    ap.add_argument("--mixed-h1l2", action="store_true",
                    help="only the paper's mixed H1 p=4 / L2 p=3 pair on --n^3 hexes")
    ap.add_argument("--paper-operator-n", type=int, default=128,
                    help="mesh size of the paper-operator entry of the main line (0: skip)")
    ap.add_argument("--mixed-orders", action="store_true",
                    help="variable-order apply: --n^3 mesh, 8^3 blocks of orders 2, 4, 6")
    args = ap.parse_args()
    if args.warmup < 3:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.sweep:
        return run_sweep(args, local_rank)
    if args.peaks:
        return run_peaks(local_rank)
    if args.batched:
        return run_batched(args, local_rank)
    if args.learned:
        return run_learned(args, local_rank)
    if args.graphs:
        return run_graphs(args, local_rank)
    if args.batched_pcg:
        return run_batched_pcg(args, local_rank)
    if args.mixed_orders:
        return run_mixed_orders(args, local_rank)
    if args.mixed_h1l2:
        return run_mixed_h1l2(args, local_rank)
    if args.refinement:
        return run_refinement(args, local_rank)
    if args.c5:
        return run_c5(args, local_rank)
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    try:
        return run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
