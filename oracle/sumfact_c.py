"""ctypes wrapper of ``sumfact_omp.c``: the sum-factorised FP64 operators and Jacobi-PCG in C with
OpenMP over elements (oracle; TEST INFRASTRUCTURE -- the timed CPU baseline).

The shared object is built with gcc on first use (``build()``; ``__graft_entry__.build()`` runs
the same command), so it exists on whichever machine runs the tests or the benchmark.  The 1D
tables and the Gauss rule come from ``quadrature.py``; the C side computes the geometry, the
quadrature data of Section II-B's partial assembly, the apply (Eq. (1) with Eq. (2)'s 1D
contractions), the diagonal and the CG iteration.  Nothing here is shared with the CUDA path.
"""
import ctypes
import os
import subprocess

import numpy as np

from .quadrature import basis_1d

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "sumfact_omp.c")
LIB = os.path.join(HERE, "libsumfact_omp.so")
CFLAGS = ["-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11"]

DIFFUSION, MASS = 1, 2
_lib = None


def build():
    """Compile sumfact_omp.c into libsumfact_omp.so (when missing or older than the source)."""
    if not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        subprocess.run(["gcc"] + CFLAGS + [SRC, "-o", LIB, "-lm"], check=True)
    return LIB


def load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(LIB)
        P = ctypes.c_void_p
        i, d, i64 = ctypes.c_int, ctypes.c_double, ctypes.c_int64
        lib.sf_threads.restype = i
        lib.sf_qdata.argtypes = [i, i, i, i, P, P, P, P, i, P]
        lib.sf_qdata.restype = i64
        lib.sf_apply.argtypes = [i, i, i, i, i, P, P, P, i, P, P]
        lib.sf_apply.restype = None
        lib.sf_diagonal.argtypes = [i, i, i, i, i, P, P, P, i, P]
        lib.sf_diagonal.restype = None
        lib.sf_pcg.argtypes = [i, i, i, i, i, P, P, P, i, P, P, P, P, d, i, P,
                               ctypes.POINTER(ctypes.c_double)]
        lib.sf_pcg.restype = i
        _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def threads():
    """OpenMP threads the C routines use (OMP_NUM_THREADS, else every core)."""
    return load().sf_threads()


class Operator:
    """Partial assembly of one operator (kind DIFFUSION or MASS) on an nx x ny x nz mesh of
    order p with Q = q1d Gauss points per axis; holds the tables and the quadrature data."""

    def __init__(self, nx, ny, nz, p, vertices, kind, coeff=None, q1d=None):
        self.nx, self.ny, self.nz, self.p = nx, ny, nz, p
        self.Q = q1d or p + 2
        self.kind = {"diffusion": DIFFUSION, "mass": MASS}.get(kind, kind)
        B, G, pts, wts, _ = basis_1d(p, self.Q)
        self.B = np.ascontiguousarray(B, dtype=np.float64)
        self.G = np.ascontiguousarray(G, dtype=np.float64)
        self.pts = np.ascontiguousarray(pts, dtype=np.float64)
        self.wts = np.ascontiguousarray(wts, dtype=np.float64)
        self.V = np.ascontiguousarray(vertices, dtype=np.float64).reshape(-1)
        ne = nx * ny * nz
        self.coeff = None if coeff is None else np.ascontiguousarray(coeff, dtype=np.float64)
        per = (6 if self.kind == DIFFUSION else 1) * self.Q ** 3
        self.qd = np.empty(ne * per)
        bad = load().sf_qdata(nx, ny, nz, self.Q, _p(self.pts), _p(self.wts), _p(self.V),
                              None if self.coeff is None else _p(self.coeff), self.kind,
                              _p(self.qd))
        if bad:
            raise ValueError("inverted element: det J <= 0 at %d points" % bad)
        self.ndofs = (nx * p + 1) * (ny * p + 1) * (nz * p + 1)

    def apply(self, x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.empty(self.ndofs)
        load().sf_apply(self.nx, self.ny, self.nz, self.p, self.Q, _p(self.B), _p(self.G),
                        _p(self.qd), self.kind, _p(x), _p(y))
        return y

    def diagonal(self):
        d = np.empty(self.ndofs)
        load().sf_diagonal(self.nx, self.ny, self.nz, self.p, self.Q, _p(self.B), _p(self.G),
                           _p(self.qd), self.kind, _p(d))
        return d

    def pcg(self, b, mask, diag, rtol, maxit):
        """Jacobi-PCG on A_bc from x = 0: (x, iterations, final relative residual)."""
        b = np.ascontiguousarray(b, dtype=np.float64)
        mask = np.ascontiguousarray(mask, dtype=np.uint8)
        diag = np.ascontiguousarray(diag, dtype=np.float64)
        x = np.empty(self.ndofs)
        work = np.empty(4 * self.ndofs)
        rel = ctypes.c_double(0.0)
        it = load().sf_pcg(self.nx, self.ny, self.nz, self.p, self.Q, _p(self.B), _p(self.G),
                           _p(self.qd), self.kind, _p(mask), _p(diag), _p(b), _p(x), float(rtol),
                           int(maxit), _p(work), ctypes.byref(rel))
        return x, it, rel.value
