"""Helpers shared by the GPU tests: build/load the library and set up problems through the C ABI."""
import contextlib

import numpy as np

from paper_2603_09038_gb300.inputs import perturbed_vertices, lognormal_coefficient

TOL = 1e-12          # relative max-norm parity bound for every apply (FP64-class)


def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU test needs CUDA"
    return torch


def lib():
    import os
    from paper_2603_09038_gb300 import fe
    if not os.path.exists(fe.LIB_PATH):
        from paper_2603_09038_gb300 import build
        build.build()
    fe.load()
    return fe


@contextlib.contextmanager
def gpu_problem(nx, ny, nz, p, sigma=None, seed=1234, coeff=None, ops=None, amp=0.1):
    """Mesh + partial assembly on cuda:0; yields (fe, mesh, pa, vertices, coeff)."""
    torch = torch_cuda()
    fe = lib()
    V = perturbed_vertices(nx, ny, nz, seed=seed, amp=amp)
    c = coeff
    if c is None and sigma is not None:
        c = lognormal_coefficient(nx * ny * nz, sigma)
    mesh = fe.fe_mesh_setup(nx, ny, nz, p, V)
    pa = None
    try:
        dc = None if c is None else torch.from_numpy(np.ascontiguousarray(c)).cuda()
        pa = fe.fe_pa_setup(mesh, 0, dc, ops or (fe.FE_DIFFUSION | fe.FE_MASS))
        yield fe, mesh, pa, V, c
    finally:
        fe.fe_pa_destroy(pa)
        fe.fe_mesh_destroy(mesh)


def rel_err(y, ref):
    y = np.asarray(y)
    return float(np.abs(y - ref).max() / np.abs(ref).max())
