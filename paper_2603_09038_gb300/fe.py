"""Thin ctypes binding of libfe (C ABI in include/fe.h): argument marshalling only.

Every function here has the name of the C entry point it calls and does no arithmetic of its
own.  Device buffers are passed as torch CUDA tensors (or raw integer device addresses);
streams default to torch's current stream.  A non-OK status raises ``FEError`` carrying the
library's message, except where a status is part of the result (``fe_pcg``).
If ``libfe.so`` has not been built, ``load()`` raises: there is no fallback path.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfe.so")

FE_OK = 0
FE_ERR_ARG = -1
FE_ERR_CUDA = -2
FE_ERR_OOM = -3
FE_ERR_UNSUPPORTED = -4
FE_ERR_NOT_CONVERGED = -5
FE_ERR_BREAKDOWN = -6
FE_ERR_NAN = -7
FE_ERR_TIMEOUT = -8

FE_DIFFUSION = 1
FE_MASS = 2
FE_PC_NONE = 0
FE_PC_JACOBI = 1
FE_PC_CHEBYSHEV = 2
FE_PC_LEARNED = 3
FE_VARIANT_F64 = 0
FE_VARIANT_F32X2 = 1
FE_VARIANT_F64_DMMA = 2
FE_VARIANT_F32 = 3

VARIANTS = {"f64": FE_VARIANT_F64, "f32x2": FE_VARIANT_F32X2, "dmma": FE_VARIANT_F64_DMMA,
            "f32": FE_VARIANT_F32}


class FEError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("libfe status %d: %s" % (status, msg))
        self.status = status


class fe_pcg_stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("rel_resid", ctypes.c_double),
                ("true_rel_resid", ctypes.c_double), ("seconds", ctypes.c_double),
                ("launches", ctypes.c_int), ("outer_iters", ctypes.c_int)]


_lib = None

_VP = ctypes.c_void_p
_SIGS = {
    "fe_mesh_setup": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _VP,
                                     ctypes.POINTER(_VP)]),
    "fe_mesh_sizes": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int64),
                                     ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int)]),
    "fe_mesh_ndofs": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int64)]),
    "fe_basis_1d": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _VP, _VP, _VP, _VP, _VP]),
    "fe_mesh_boundary_mask": (ctypes.c_int, [_VP, _VP, _VP]),
    "fe_mesh_dof_map": (ctypes.c_int, [_VP, _VP, _VP]),
    "fe_pa_setup": (ctypes.c_int, [_VP, ctypes.c_int, _VP, ctypes.c_int, _VP, ctypes.POINTER(_VP)]),
    "fe_pa_set_variant": (ctypes.c_int, [_VP, ctypes.c_int, _VP]),
    "fe_pa_get_variant": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int)]),
    "fe_apply_diffusion": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "fe_apply_mass": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "fe_apply": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, _VP, _VP, _VP]),
    "fe_apply_batched": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, _VP,
                                        ctypes.c_int64, _VP, ctypes.c_int64, _VP]),
    "fe_assemble_diagonal": (ctypes.c_int, [_VP, ctypes.c_int, _VP, _VP]),
    "fe_load_vector_sine": (ctypes.c_int, [_VP, _VP, _VP]),
    "fe_pcg": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, _VP, _VP, ctypes.c_double,
                              ctypes.c_int, ctypes.POINTER(fe_pcg_stats), _VP]),
    "fe_pcg_host": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, _VP, _VP, ctypes.c_double,
                                   ctypes.c_int, ctypes.POINTER(fe_pcg_stats), _VP]),
    "fe_pcg_ir": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, _VP, _VP, ctypes.c_double,
                                 ctypes.c_int, ctypes.c_double, ctypes.POINTER(fe_pcg_stats), _VP]),
    "fe_pcg_noalloc": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, _VP, _VP, ctypes.c_double,
                                      ctypes.c_int, ctypes.POINTER(fe_pcg_stats), _VP]),
    "fe_probe_throughput": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    "fe_pcg_chebyshev": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                        ctypes.c_double, _VP, _VP, ctypes.c_double, ctypes.c_int,
                                        ctypes.POINTER(fe_pcg_stats), _VP]),
    "fe_pcg_set_graphs": (ctypes.c_int, [_VP, ctypes.c_int]),
    "fe_pa_set_shape": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "fe_pa_get_shape": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                       ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "fe_pa_autotune": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      ctypes.POINTER(ctypes.c_int), _VP, _VP]),
    "fe_pcg_batched": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, _VP,
                                      ctypes.c_int64, _VP, ctypes.c_int64, ctypes.c_double,
                                      ctypes.c_int, ctypes.POINTER(fe_pcg_stats), _VP]),
    "fe_estimate_lmax": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_double), _VP]),
    "fe_lpc_create": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                     ctypes.POINTER(_VP)]),
    "fe_lpc_nparams": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int64)]),
    "fe_lpc_train": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                    ctypes.POINTER(ctypes.c_double), _VP]),
    "fe_lpc_weights": (ctypes.c_int, [_VP, _VP, ctypes.c_int]),
    "fe_lpc_fit_linear": (ctypes.c_int, [_VP, ctypes.c_double, ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_double), _VP]),
    "fe_lpc_loss_grad": (ctypes.c_int, [_VP, ctypes.c_int, _VP, _VP, _VP, _VP,
                                        ctypes.POINTER(ctypes.c_double)]),
    "fe_lpc_apply": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "fe_vspace_set_learned": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, _VP, _VP]),
    "fe_vspace_lpc_apply": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "fe_vspace_fcg": (ctypes.c_int, [_VP, ctypes.c_int, _VP, _VP, ctypes.c_double, ctypes.c_int,
                                     ctypes.POINTER(fe_pcg_stats), _VP]),
    "fe_lpc_set_kernel": (ctypes.c_int, [_VP, ctypes.c_int]),
    "fe_lpc_get_kernel": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int),
                                         ctypes.POINTER(ctypes.c_int)]),
    "fe_lpc_adam_step": (ctypes.c_int, [_VP, ctypes.c_int, _VP, _VP, ctypes.c_double,
                                        ctypes.POINTER(ctypes.c_double)]),
    "fe_lpc_sample_pairs": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int64, _VP, _VP, _VP,
                                           ctypes.POINTER(ctypes.c_int64), _VP]),
    "fe_lpc_set_fallback": (ctypes.c_int, [_VP, ctypes.c_int]),
    "fe_pa_set_learned": (ctypes.c_int, [_VP, _VP]),
    "fe_lpc_save": (ctypes.c_int, [_VP, ctypes.c_char_p]),
    "fe_lpc_load": (ctypes.c_int, [_VP, ctypes.c_char_p]),
    "fe_lpc_checkpoint_info": (ctypes.c_int, [ctypes.c_char_p, ctypes.POINTER(ctypes.c_int),
                                              ctypes.POINTER(ctypes.c_int),
                                              ctypes.POINTER(ctypes.c_int64),
                                              ctypes.POINTER(ctypes.c_int)]),
    "fe_fcg": (ctypes.c_int, [_VP, ctypes.c_int, _VP, _VP, _VP, ctypes.c_double, ctypes.c_int,
                              ctypes.POINTER(fe_pcg_stats), _VP]),
    "fe_fcg_ir": (ctypes.c_int, [_VP, ctypes.c_int, _VP, _VP, _VP, ctypes.c_double, ctypes.c_int,
                                 ctypes.c_double, ctypes.POINTER(fe_pcg_stats), _VP]),
    "fe_lpc_destroy": (None, [_VP]),
    "fe_vspace_setup": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _VP, _VP, _VP,
                                       ctypes.c_int, _VP, ctypes.POINTER(_VP)]),
    "fe_vspace_host_E": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _VP,
                                        ctypes.POINTER(ctypes.c_int64),
                                        ctypes.POINTER(ctypes.c_int64),
                                        ctypes.POINTER(ctypes.c_int64), _VP, _VP, _VP, _VP, _VP]),
    "fe_vspace_sizes": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int64),
                                       ctypes.POINTER(ctypes.c_int64),
                                       ctypes.POINTER(ctypes.c_int64)]),
    "fe_vspace_layout": (ctypes.c_int, [_VP, _VP]),
    "fe_vspace_constraint_sizes": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int64),
                                                  ctypes.POINTER(ctypes.c_int64),
                                                  ctypes.POINTER(ctypes.c_int64)]),
    "fe_vspace_boundary_mask": (ctypes.c_int, [_VP, _VP, _VP]),
    "fe_vspace_set_variant": (ctypes.c_int, [_VP, ctypes.c_int, _VP]),
    "fe_vspace_prolong": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "fe_vspace_set_persistent": (ctypes.c_int, [_VP, ctypes.c_int]),
    "fe_vspace_apply_batched": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, _VP,
                                               ctypes.c_int64, _VP, ctypes.c_int64, _VP]),
    "fe_vspace_pcg_batched": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, _VP,
                                             ctypes.c_int64, _VP, ctypes.c_int64,
                                             ctypes.c_double, ctypes.c_int,
                                             ctypes.POINTER(fe_pcg_stats), _VP]),
    "fe_vspace_apply": (ctypes.c_int, [_VP, ctypes.c_int, _VP, _VP, _VP]),
    "fe_vspace_diagonal": (ctypes.c_int, [_VP, ctypes.c_int, _VP, _VP]),
    "fe_vspace_pcg": (ctypes.c_int, [_VP, ctypes.c_int, _VP, _VP, ctypes.c_double, ctypes.c_int,
                                     ctypes.POINTER(fe_pcg_stats), _VP]),
    "fe_vspace_destroy": (None, [_VP]),
    "fe_mixed_setup": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_int, _VP, _VP, ctypes.POINTER(_VP)]),
    "fe_mixed_sizes": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int64),
                                      ctypes.POINTER(ctypes.c_int64)]),
    "fe_mixed_apply": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP]),
    "fe_mixed_destroy": (None, [_VP]),
    "fe_pa_destroy": (None, [_VP]),
    "fe_mesh_destroy": (None, [_VP]),
    "fe_last_error": (ctypes.c_char_p, []),
    "fe_version": (ctypes.c_char_p, []),
}


def load(path=LIB_PATH):
    """Loads libfe.so (once) and declares the C signatures; raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError("libfe.so is not built (%s); run __graft_entry__.build()" % path)
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _check(status):
    if status != FE_OK:
        raise FEError(status, _lib.fe_last_error().decode())
    return status


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return _VP(t)
    return _VP(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        return _VP(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return _VP(stream)
    return _VP(stream.cuda_stream)


# ---------------------------------------------------------------- entry points (same names)

def fe_mesh_setup(nx, ny, nz, order, vertices):
    """vertices: host float64 array [(nx+1)(ny+1)(nz+1), 3]; returns the mesh handle."""
    lib = load()
    v = np.ascontiguousarray(vertices, dtype=np.float64)
    out = _VP()
    _check(lib.fe_mesh_setup(int(nx), int(ny), int(nz), int(order),
                             v.ctypes.data_as(_VP), ctypes.byref(out)))
    return out.value


def fe_mesh_sizes(mesh):
    lib = load()
    nd, ne, p = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int()
    _check(lib.fe_mesh_sizes(_VP(mesh), ctypes.byref(nd), ctypes.byref(ne), ctypes.byref(p)))
    return nd.value, ne.value, p.value


def fe_basis_1d(order, q1d):
    """(nodes[D], pts[Q], wts[Q], B[Q, D], G[Q, D]) of the library's 1D tables (host only)."""
    D, Q = int(order) + 1, int(q1d)
    nodes, pts, wts = np.zeros(max(D, 1)), np.zeros(max(Q, 1)), np.zeros(max(Q, 1))
    B, G = np.zeros((max(Q, 1), max(D, 1))), np.zeros((max(Q, 1), max(D, 1)))
    _check(load().fe_basis_1d(int(order), int(q1d), nodes.ctypes.data_as(_VP),
                              pts.ctypes.data_as(_VP), wts.ctypes.data_as(_VP),
                              B.ctypes.data_as(_VP), G.ctypes.data_as(_VP)))
    return nodes, pts, wts, B, G


def fe_mesh_ndofs(mesh):
    nd = ctypes.c_int64()
    _check(load().fe_mesh_ndofs(_VP(mesh), ctypes.byref(nd)))
    return nd.value


def fe_mesh_boundary_mask(mesh, dev_mask, stream=None):
    _check(load().fe_mesh_boundary_mask(_VP(mesh), _ptr(dev_mask), _stream(stream)))


def fe_mesh_dof_map(mesh, dev_map, stream=None):
    _check(load().fe_mesh_dof_map(_VP(mesh), _ptr(dev_map), _stream(stream)))


def fe_pa_setup(mesh, q1d=0, dev_coeff=None, ops=FE_DIFFUSION | FE_MASS, stream=None):
    lib = load()
    out = _VP()
    _check(lib.fe_pa_setup(_VP(mesh), int(q1d), _ptr(dev_coeff), int(ops), _stream(stream),
                           ctypes.byref(out)))
    return out.value


def fe_pa_set_variant(pa, variant, stream=None):
    v = VARIANTS.get(variant, variant)
    _check(load().fe_pa_set_variant(_VP(pa), int(v), _stream(stream)))


def fe_pa_get_variant(pa):
    v = ctypes.c_int()
    _check(load().fe_pa_get_variant(_VP(pa), ctypes.byref(v)))
    return v.value


def fe_apply_diffusion(pa, dev_x, dev_y, stream=None):
    _check(load().fe_apply_diffusion(_VP(pa), _ptr(dev_x), _ptr(dev_y), _stream(stream)))


def fe_apply_mass(pa, dev_x, dev_y, stream=None):
    _check(load().fe_apply_mass(_VP(pa), _ptr(dev_x), _ptr(dev_y), _stream(stream)))


def fe_apply(pa, op, variant, dev_x, dev_y, stream=None):
    v = VARIANTS.get(variant, variant)
    _check(load().fe_apply(_VP(pa), int(op), int(v), _ptr(dev_x), _ptr(dev_y), _stream(stream)))


def fe_apply_batched(pa, op, variant, nrhs, dev_x, ldx, dev_y, ldy, stream=None):
    """nrhs applies in one launch; x, y hold the right-hand sides at strides ldx, ldy."""
    v = VARIANTS.get(variant, variant)
    _check(load().fe_apply_batched(_VP(pa), int(op), int(v), int(nrhs), _ptr(dev_x), int(ldx),
                                   _ptr(dev_y), int(ldy), _stream(stream)))


def fe_assemble_diagonal(pa, op, dev_diag, stream=None):
    _check(load().fe_assemble_diagonal(_VP(pa), int(op), _ptr(dev_diag), _stream(stream)))


def fe_load_vector_sine(pa, dev_b, stream=None):
    _check(load().fe_load_vector_sine(_VP(pa), _ptr(dev_b), _stream(stream)))


def fe_pcg(pa, op, pc, dev_b, dev_x, rtol, maxit, stream=None):
    """Returns (status, stats dict); the status is not raised (non-convergence is a result)."""
    lib = load()
    st = fe_pcg_stats()
    status = lib.fe_pcg(_VP(pa), int(op), int(pc), _ptr(dev_b), _ptr(dev_x), float(rtol),
                        int(maxit), ctypes.byref(st), _stream(stream))
    if status in (FE_ERR_ARG, FE_ERR_CUDA, FE_ERR_OOM, FE_ERR_UNSUPPORTED):
        _check(status)
    return status, _stats(st)


def _host_f64(a, writable=False):
    """Address of a host FP64 vector: a C-contiguous numpy array or CPU torch tensor (not
    copied, so that pinned memory stays pinned)."""
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags.c_contiguous or (writable and not a.flags.writeable):
            raise ValueError("host vector: need a C-contiguous%s float64 array"
                             % (" writable" if writable else ""))
        return _VP(a.ctypes.data)
    if getattr(a, "is_cuda", True) or not a.is_contiguous() or str(a.dtype) != "torch.float64":
        raise ValueError("host vector: need a contiguous float64 CPU tensor or numpy array")
    return _VP(a.data_ptr())


def fe_pcg_host(pa, op, pc, host_b, host_x, rtol, maxit, stream=None):
    """fe_pcg on host vectors (copies inside the call); same return value as fe_pcg."""
    lib = load()
    st = fe_pcg_stats()
    status = lib.fe_pcg_host(_VP(pa), int(op), int(pc), _host_f64(host_b),
                             _host_f64(host_x, writable=True), float(rtol), int(maxit),
                             ctypes.byref(st), _stream(stream))
    if status in (FE_ERR_ARG, FE_ERR_CUDA, FE_ERR_OOM, FE_ERR_UNSUPPORTED):
        _check(status)
    return status, _stats(st)


def _stats(st):
    return {"iters": st.iters, "rel_resid": st.rel_resid, "true_rel_resid": st.true_rel_resid,
            "seconds": st.seconds, "launches": st.launches, "outer_iters": st.outer_iters}


def fe_pcg_ir(pa, op, pc, dev_b, dev_x, rtol, maxit, inner_rtol=0.0, stream=None):
    """Mixed-precision iterative refinement (FP32 inner PCG, FP64-accurate outer residual);
    same return value as fe_pcg."""
    lib = load()
    st = fe_pcg_stats()
    status = lib.fe_pcg_ir(_VP(pa), int(op), int(pc), _ptr(dev_b), _ptr(dev_x), float(rtol),
                           int(maxit), float(inner_rtol), ctypes.byref(st), _stream(stream))
    if status in (FE_ERR_ARG, FE_ERR_CUDA, FE_ERR_OOM, FE_ERR_UNSUPPORTED):
        _check(status)
    return status, _stats(st)


def fe_pcg_chebyshev(pa, op, dev_b, dev_x, rtol, maxit, degree=0, lmax=0.0, lmin_ratio=0.0,
                     stream=None):
    """Chebyshev-polynomial-preconditioned CG (see include/fe.h); same return value as fe_pcg."""
    lib = load()
    st = fe_pcg_stats()
    status = lib.fe_pcg_chebyshev(_VP(pa), int(op), int(degree), float(lmax), float(lmin_ratio),
                                  _ptr(dev_b), _ptr(dev_x), float(rtol), int(maxit),
                                  ctypes.byref(st), _stream(stream))
    if status in (FE_ERR_ARG, FE_ERR_CUDA, FE_ERR_OOM, FE_ERR_UNSUPPORTED):
        _check(status)
    return status, _stats(st)


def fe_pcg_batched(pa, op, pc, nrhs, dev_b, ldb, dev_x, ldx, rtol, maxit, stream=None):
    """nrhs systems in lockstep with one batched apply per iteration; returns (status, [stats])."""
    lib = load()
    st = (fe_pcg_stats * int(nrhs))()
    status = lib.fe_pcg_batched(_VP(pa), int(op), int(pc), int(nrhs), _ptr(dev_b), int(ldb),
                                _ptr(dev_x), int(ldx), float(rtol), int(maxit), st,
                                _stream(stream))
    if status in (FE_ERR_ARG, FE_ERR_CUDA, FE_ERR_OOM, FE_ERR_UNSUPPORTED):
        _check(status)
    return status, [_stats(x) for x in st]


def fe_pa_set_shape(pa, op, variant, shape):
    _check(load().fe_pa_set_shape(_VP(pa), int(op), VARIANTS.get(variant, variant), int(shape)))


def fe_pa_get_shape(pa, op, variant):
    """(selected shape, built shapes, threads per block, elements per block)."""
    v = [ctypes.c_int() for _ in range(4)]
    _check(load().fe_pa_get_shape(_VP(pa), int(op), VARIANTS.get(variant, variant),
                                  *[ctypes.byref(x) for x in v]))
    return tuple(x.value for x in v)


def fe_pa_autotune(pa, op, nrhs=1, reps=5, stream=None):
    """Selects the fastest FP64-accurate variant; returns (variant name, {name: ms})."""
    import numpy as np
    best = ctypes.c_int()
    ms = np.zeros(4)
    _check(load().fe_pa_autotune(_VP(pa), int(op), int(nrhs), int(reps), ctypes.byref(best),
                                 _VP(ms.ctypes.data), _stream(stream)))
    names = {v: k for k, v in VARIANTS.items()}
    return names[best.value], {names[i]: float(ms[i]) for i in range(4) if ms[i] >= 0}


def fe_pcg_set_graphs(pa, enable):
    _check(load().fe_pcg_set_graphs(_VP(pa), int(bool(enable))))


def fe_estimate_lmax(pa, op, iters=20, stream=None):
    v = ctypes.c_double()
    _check(load().fe_estimate_lmax(_VP(pa), int(op), int(iters), ctypes.byref(v), _stream(stream)))
    return v.value


FE_PCG_NOALLOC_MAX_DOFS = 262144


def fe_pcg_noalloc(pa, op, pc, dev_b, dev_x, rtol, maxit, stream=None):
    """fe_pcg that allocates no device memory (fixed in-library scratch, at most
    FE_PCG_NOALLOC_MAX_DOFS dofs); same return value as fe_pcg."""
    lib = load()
    st = fe_pcg_stats()
    status = lib.fe_pcg_noalloc(_VP(pa), int(op), int(pc), _ptr(dev_b), _ptr(dev_x), float(rtol),
                                int(maxit), ctypes.byref(st), _stream(stream))
    if status in (FE_ERR_ARG, FE_ERR_CUDA, FE_ERR_OOM, FE_ERR_UNSUPPORTED):
        _check(status)
    return status, _stats(st)


PROBE_UNITS = {"fp64_fma": 0, "fp64_dmma": 1, "fp32_fma": 2, "f32x2_mac": 3, "bf16_mma": 4,
               "fp64_dfma_dmma": 5}


def fe_probe_throughput(unit):
    """Sustained TFLOP/s of one arithmetic unit of the current GPU (see include/fe.h)."""
    v = ctypes.c_double()
    _check(load().fe_probe_throughput(int(PROBE_UNITS.get(unit, unit)), ctypes.byref(v)))
    return v.value


# ---------------------------------------------------- learned patch preconditioner and FCG

def fe_lpc_create(pa, op, width=256, seed=0):
    """Learned element-patch preconditioner for operator op of pa (see include/fe.h)."""
    out = _VP()
    _check(load().fe_lpc_create(_VP(pa), int(op), int(width), int(seed), ctypes.byref(out)))
    return out.value


def fe_lpc_nparams(lpc):
    n = ctypes.c_int64()
    _check(load().fe_lpc_nparams(_VP(lpc), ctypes.byref(n)))
    return n.value


def fe_lpc_train(lpc, steps, batch, lr, reps=0, stream=None):
    """Adam steps on the patch training set (made on the first call); returns the last loss."""
    loss = ctypes.c_double()
    _check(load().fe_lpc_train(_VP(lpc), int(steps), int(batch), float(lr), int(reps),
                               ctypes.byref(loss), _stream(stream)))
    return loss.value


def fe_lpc_fit_linear(lpc, ridge=1e-6, reps=0, stream=None):
    """Least-squares fit of the linear term W0 on the training set; returns the fit's loss."""
    loss = ctypes.c_double()
    _check(load().fe_lpc_fit_linear(_VP(lpc), float(ridge), int(reps), ctypes.byref(loss),
                                    _stream(stream)))
    return loss.value


def _f32_host(a, n):
    import numpy as np
    a = np.ascontiguousarray(a, dtype=np.float32).reshape(-1)
    if a.size != n:
        raise ValueError("expected %d floats, got %d" % (n, a.size))
    return a


def fe_lpc_weights(lpc, host_w=None):
    """Returns the packed FP32 master weights (numpy), or sets them from host_w."""
    import numpy as np
    n = fe_lpc_nparams(lpc)
    if host_w is None:
        w = np.empty(n, dtype=np.float32)
        _check(load().fe_lpc_weights(_VP(lpc), _VP(w.ctypes.data), 0))
        return w
    w = _f32_host(host_w, n)
    _check(load().fe_lpc_weights(_VP(lpc), _VP(w.ctypes.data), 1))
    return w


def fe_lpc_loss_grad(lpc, X, T):
    """(loss, Y, grad) of the BF16 tensor-core forward/backward pass on host rows X, T."""
    import numpy as np
    X = np.ascontiguousarray(X, dtype=np.float32)
    T = np.ascontiguousarray(T, dtype=np.float32)
    if X.shape != T.shape or X.ndim != 2:
        raise ValueError("X and T must be [batch, D^3] arrays of the same shape")
    Y = np.empty_like(X)
    g = np.empty(fe_lpc_nparams(lpc), dtype=np.float32)
    loss = ctypes.c_double()
    _check(load().fe_lpc_loss_grad(_VP(lpc), X.shape[0], _VP(X.ctypes.data), _VP(T.ctypes.data),
                                   _VP(Y.ctypes.data), _VP(g.ctypes.data), ctypes.byref(loss)))
    return loss.value, Y, g


def fe_lpc_adam_step(lpc, X, T, lr):
    """One Adam step on host rows X, targets T (float32 [batch, D^3]); returns the loss before it."""
    X = np.ascontiguousarray(X, dtype=np.float32)
    T = np.ascontiguousarray(T, dtype=np.float32)
    loss = ctypes.c_double()
    _check(load().fe_lpc_adam_step(_VP(lpc), int(X.shape[0]), X.ctypes.data_as(_VP),
                                   T.ctypes.data_as(_VP), float(lr), ctypes.byref(loss)))
    return loss.value


def fe_lpc_sample_pairs(lpc, din, reps=0, max_rows=1 << 16, stream=None):
    """The generator's training pairs in FP64: (elements int32 [rows], X, T float64 [rows, din])."""
    cap = int(max_rows)
    el = np.zeros(cap, dtype=np.int32)
    X = np.zeros((cap, din))
    T = np.zeros((cap, din))
    rows = ctypes.c_int64()
    _check(load().fe_lpc_sample_pairs(_VP(lpc), int(reps), cap, el.ctypes.data_as(_VP),
                                      X.ctypes.data_as(_VP), T.ctypes.data_as(_VP),
                                      ctypes.byref(rows), _stream(stream)))
    n = rows.value
    return el[:n], X[:n], T[:n]


def fe_lpc_apply(lpc, dev_r, dev_z, stream=None):
    return _check(load().fe_lpc_apply(_VP(lpc), _ptr(dev_r), _ptr(dev_z), _stream(stream)))


FE_LPC_KERNEL_AUTO, FE_LPC_KERNEL_TCGEN05, FE_LPC_KERNEL_MMA_SYNC, FE_LPC_KERNEL_GEMM = 0, 1, 2, 3


def fe_vspace_set_learned(vs, op, order, trained, stream=None):
    """Attach a copy of a trained single-order network to the order group (None detaches)."""
    return _check(load().fe_vspace_set_learned(_VP(vs), int(op), int(order),
                                               _VP(trained) if trained else None, _stream(stream)))


def fe_vspace_lpc_apply(vs, dev_r, dev_z, stream=None):
    return _check(load().fe_vspace_lpc_apply(_VP(vs), _ptr(dev_r), _ptr(dev_z), _stream(stream)))


def fe_vspace_fcg(vs, op, dev_b, dev_x, rtol, maxit, stream=None):
    """Flexible CG with the attached networks; same return value as fe_pcg."""
    st = fe_pcg_stats()
    status = load().fe_vspace_fcg(_VP(vs), int(op), _ptr(dev_b), _ptr(dev_x), float(rtol),
                                  int(maxit), ctypes.byref(st), _stream(stream))
    if status in (FE_ERR_ARG, FE_ERR_CUDA, FE_ERR_OOM, FE_ERR_UNSUPPORTED):
        _check(status)
    return status, _stats(st)


def fe_lpc_set_kernel(lpc, kernel):
    return _check(load().fe_lpc_set_kernel(_VP(lpc), int(kernel)))


def fe_lpc_get_kernel(lpc):
    """(the inference kernel in use, 1 if a tcgen05 launch has given up a wait else 0)."""
    k, f = ctypes.c_int(), ctypes.c_int()
    _check(load().fe_lpc_get_kernel(_VP(lpc), ctypes.byref(k), ctypes.byref(f)))
    return k.value, f.value


def fe_fcg(pa, op, lpc, dev_b, dev_x, rtol, maxit, stream=None):
    """Flexible CG preconditioned by lpc (None => Jacobi); same return value as fe_pcg."""
    lib = load()
    st = fe_pcg_stats()
    status = lib.fe_fcg(_VP(pa), int(op), _VP(lpc) if lpc else None, _ptr(dev_b), _ptr(dev_x),
                        float(rtol), int(maxit), ctypes.byref(st), _stream(stream))
    if status in (FE_ERR_ARG, FE_ERR_CUDA, FE_ERR_OOM, FE_ERR_UNSUPPORTED):
        _check(status)
    return status, _stats(st)


def fe_fcg_ir(pa, op, lpc, dev_b, dev_x, rtol, maxit, inner_rtol=0.0, stream=None):
    """Mixed-precision refinement around an FP32 flexible CG preconditioned by lpc; same return
    value as fe_pcg."""
    lib = load()
    st = fe_pcg_stats()
    status = lib.fe_fcg_ir(_VP(pa), int(op), _VP(lpc), _ptr(dev_b), _ptr(dev_x), float(rtol),
                           int(maxit), float(inner_rtol), ctypes.byref(st), _stream(stream))
    if status in (FE_ERR_ARG, FE_ERR_CUDA, FE_ERR_OOM, FE_ERR_UNSUPPORTED):
        _check(status)
    return status, _stats(st)


def fe_lpc_save(lpc, path):
    """Checkpoint of the weights and Adam state (format in include/fe.h)."""
    _check(load().fe_lpc_save(_VP(lpc), os.fsencode(path)))


def fe_lpc_load(lpc, path):
    _check(load().fe_lpc_load(_VP(lpc), os.fsencode(path)))


def fe_lpc_checkpoint_info(path):
    """(din, width, nparam, adam_steps) from a checkpoint's header (host only)."""
    din, w, ap = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    n = ctypes.c_int64()
    _check(load().fe_lpc_checkpoint_info(os.fsencode(path), ctypes.byref(din), ctypes.byref(w),
                                         ctypes.byref(n), ctypes.byref(ap)))
    return din.value, w.value, n.value, ap.value


def fe_pa_set_learned(pa, lpc):
    """Attach lpc (or None to detach) as fe_pcg's FE_PC_LEARNED preconditioner."""
    _check(load().fe_pa_set_learned(_VP(pa), _VP(lpc) if lpc else None))


def fe_lpc_set_fallback(lpc, pc):
    """pc: FE_PC_JACOBI or FE_PC_CHEBYSHEV -- what fe_fcg continues with once it gives up lpc."""
    _check(load().fe_lpc_set_fallback(_VP(lpc), int(pc)))


def fe_lpc_destroy(lpc):
    if lpc:
        load().fe_lpc_destroy(_VP(lpc))


def fe_vspace_setup(nx, ny, nz, orders, vertices, coeff=None, ops=FE_DIFFUSION | FE_MASS,
                    stream=None):
    """orders: host int32 [ne]; vertices: host float64 [(nx+1)(ny+1)(nz+1), 3]; coeff: host
    float64 [ne] or None.  Returns the variable-order space handle."""
    lib = load()
    o = np.ascontiguousarray(orders, dtype=np.int32)
    v = np.ascontiguousarray(vertices, dtype=np.float64)
    c = None if coeff is None else np.ascontiguousarray(coeff, dtype=np.float64)
    out = _VP()
    _check(lib.fe_vspace_setup(int(nx), int(ny), int(nz), o.ctypes.data_as(_VP),
                               v.ctypes.data_as(_VP), None if c is None else c.ctypes.data_as(_VP),
                               int(ops), _stream(stream), ctypes.byref(out)))
    return out.value


def fe_vspace_host_E(nx, ny, nz, orders):
    """Host-only E of the variable-order space (no GPU needed): returns (ntrue, rowptr, cols,
    vals, elem_first, mask) with E in CSR, rows in E-vector order."""
    lib = load()
    o = np.ascontiguousarray(orders, dtype=np.int32)
    nt, nl, nz_ = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(lib.fe_vspace_host_E(int(nx), int(ny), int(nz), o.ctypes.data_as(_VP), ctypes.byref(nt),
                                ctypes.byref(nl), ctypes.byref(nz_), None, None, None, None, None))
    rowptr = np.zeros(nl.value + 1, dtype=np.int64)
    cols = np.zeros(nz_.value, dtype=np.int32)
    vals = np.zeros(nz_.value, dtype=np.float64)
    first = np.zeros(o.size, dtype=np.int64)
    mask = np.zeros(nt.value, dtype=np.uint8)
    _check(lib.fe_vspace_host_E(int(nx), int(ny), int(nz), o.ctypes.data_as(_VP), ctypes.byref(nt),
                                ctypes.byref(nl), ctypes.byref(nz_), rowptr.ctypes.data_as(_VP),
                                cols.ctypes.data_as(_VP), vals.ctypes.data_as(_VP),
                                first.ctypes.data_as(_VP), mask.ctypes.data_as(_VP)))
    return nt.value, rowptr, cols, vals, first, mask


def fe_vspace_sizes(vs):
    """(ntrue, nlocal, nnz)."""
    a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(load().fe_vspace_sizes(_VP(vs), ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, c.value


def fe_vspace_constraint_sizes(vs):
    """(constrained rows of E, their nonzeros, true dofs they touch)."""
    a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(load().fe_vspace_constraint_sizes(_VP(vs), ctypes.byref(a), ctypes.byref(b),
                                             ctypes.byref(c)))
    return a.value, b.value, c.value


def fe_vspace_layout(vs, ne):
    first = np.zeros(int(ne), dtype=np.int64)
    _check(load().fe_vspace_layout(_VP(vs), first.ctypes.data_as(_VP)))
    return first


def fe_vspace_boundary_mask(vs, dev_mask, stream=None):
    _check(load().fe_vspace_boundary_mask(_VP(vs), _ptr(dev_mask), _stream(stream)))


def fe_vspace_set_variant(vs, variant, stream=None):
    v = VARIANTS.get(variant, variant)
    _check(load().fe_vspace_set_variant(_VP(vs), int(v), _stream(stream)))


def fe_vspace_set_persistent(vs, enable):
    _check(load().fe_vspace_set_persistent(_VP(vs), int(bool(enable))))


def fe_vspace_apply_batched(vs, op, nrhs, dev_x, ldx, dev_y, ldy, stream=None):
    _check(load().fe_vspace_apply_batched(_VP(vs), int(op), int(nrhs), _ptr(dev_x), int(ldx),
                                          _ptr(dev_y), int(ldy), _stream(stream)))


def fe_vspace_pcg_batched(vs, op, nrhs, dev_b, ldb, dev_x, ldx, rtol, maxit, stream=None):
    """Returns (status, [stats dict per system]); non-convergence is a result, not raised."""
    st = (fe_pcg_stats * int(nrhs))()
    status = load().fe_vspace_pcg_batched(_VP(vs), int(op), int(nrhs), _ptr(dev_b), int(ldb),
                                          _ptr(dev_x), int(ldx), float(rtol), int(maxit), st,
                                          _stream(stream))
    if status in (FE_ERR_ARG, FE_ERR_CUDA, FE_ERR_OOM, FE_ERR_UNSUPPORTED):
        _check(status)
    return status, [_stats(x) for x in st]


def fe_vspace_prolong(vs, dev_x, dev_e, stream=None):
    _check(load().fe_vspace_prolong(_VP(vs), _ptr(dev_x), _ptr(dev_e), _stream(stream)))


def fe_vspace_apply(vs, op, dev_x, dev_y, stream=None):
    _check(load().fe_vspace_apply(_VP(vs), int(op), _ptr(dev_x), _ptr(dev_y), _stream(stream)))


def fe_vspace_diagonal(vs, op, dev_diag, stream=None):
    _check(load().fe_vspace_diagonal(_VP(vs), int(op), _ptr(dev_diag), _stream(stream)))


def fe_vspace_pcg(vs, op, dev_b, dev_x, rtol, maxit, stream=None):
    """Jacobi-PCG on the variable-order space; returns (status, stats dict) like fe_pcg."""
    st = fe_pcg_stats()
    status = load().fe_vspace_pcg(_VP(vs), int(op), _ptr(dev_b), _ptr(dev_x), float(rtol),
                                  int(maxit), ctypes.byref(st), _stream(stream))
    if status in (FE_ERR_ARG, FE_ERR_CUDA, FE_ERR_OOM, FE_ERR_UNSUPPORTED):
        _check(status)
    return status, _stats(st)


def fe_vspace_destroy(vs):
    if vs:
        load().fe_vspace_destroy(_VP(vs))


def fe_mixed_setup(nx, ny, nz, order_h, order_l, vertices, stream=None):
    V = np.ascontiguousarray(vertices, dtype=np.float64)
    out = _VP()
    _check(load().fe_mixed_setup(int(nx), int(ny), int(nz), int(order_h), int(order_l),
                                 V.ctypes.data_as(_VP), _stream(stream), ctypes.byref(out)))
    return out.value


def fe_mixed_sizes(mx):
    h, l = ctypes.c_int64(), ctypes.c_int64()
    _check(load().fe_mixed_sizes(_VP(mx), ctypes.byref(h), ctypes.byref(l)))
    return h.value, l.value


def fe_mixed_apply(mx, dev_p, dev_u, dev_gp, dev_gtu, stream=None):
    """gp = G p and gtu = G^T u in one launch (pass None for both of a pair to skip it)."""
    _check(load().fe_mixed_apply(_VP(mx), _ptr(dev_p), _ptr(dev_u), _ptr(dev_gp),
                                 _ptr(dev_gtu), _stream(stream)))


def fe_mixed_destroy(mx):
    if mx:
        load().fe_mixed_destroy(_VP(mx))


def fe_pa_destroy(pa):
    if pa:
        load().fe_pa_destroy(_VP(pa))


def fe_mesh_destroy(mesh):
    if mesh:
        load().fe_mesh_destroy(_VP(mesh))


def fe_last_error():
    return load().fe_last_error().decode()


def fe_version():
    return load().fe_version().decode()
