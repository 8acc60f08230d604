"""The C/OpenMP sum-factorised operators (oracle/sumfact_omp.c, the timed CPU baseline) pinned on
the CPU: brute-force agreement with the element-matrix oracle on tiny meshes of every order
(<= 1e-13), the null space of diffusion, the mesh volume through the mass operator, symmetry,
the diagonal, Jacobi-PCG against the oracle's CG, and results that do not depend on the thread
count (elements are coloured, so the scatter-add order is fixed)."""
import os
import subprocess
import sys

import numpy as np
import pytest

from oracle import operator as oop
from oracle import sumfact_c
from oracle.element import DIFFUSION, MASS
from oracle.mesh import boundary_mask
from oracle.solve import pcg as oracle_pcg, load_vector
from paper_2603_09038_gb300.inputs import perturbed_vertices, uniform_vector, lognormal_coefficient

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CASES = [((1, 1, 1), p) for p in range(1, 9)] + [((2, 2, 2), p) for p in (1, 2, 3, 4, 5)] + \
        [((3, 2, 2), 3), ((2, 3, 4), 2)]


@pytest.mark.parametrize("dims,p", CASES)
def test_apply_matches_element_matrix_oracle(dims, p):
    V = perturbed_vertices(*dims)
    c = lognormal_coefficient(int(np.prod(dims)), 1.0)
    prob = oop.Problem(*dims, p, V, coeff=c)
    x = uniform_vector(prob.ndofs, seed=p)
    for kind in (DIFFUSION, MASS):
        op = sumfact_c.Operator(*dims, p, V, kind, coeff=c)
        ref = oop.apply(prob, x, kind)
        y = op.apply(x)
        assert np.abs(y - ref).max() <= 1e-13 * np.abs(ref).max(), (kind, dims, p)
        d = op.diagonal()
        dref = oop.diagonal(prob, kind)
        assert np.abs(d - dref).max() <= 1e-13 * np.abs(dref).max(), (kind, dims, p)


@pytest.mark.parametrize("p", [1, 3, 6])
def test_invariants_null_space_volume_symmetry(p):
    dims = (3, 2, 4)
    V = perturbed_vertices(*dims)
    K = sumfact_c.Operator(*dims, p, V, "diffusion")
    M = sumfact_c.Operator(*dims, p, V, "mass")
    one = np.ones(K.ndofs)
    Kone = K.apply(one)
    x, y = uniform_vector(K.ndofs, 1), uniform_vector(K.ndofs, 2)
    Kx = K.apply(x)
    assert np.abs(Kone).max() <= 1e-13 * np.abs(Kx).max()            # A 1 = 0
    assert abs(one @ M.apply(one) - 1.0) <= 1e-13                     # 1^T M 1 = |unit cube|
    for op in (K, M):                                                 # x^T A y = y^T A x
        a, b = x @ op.apply(y), y @ op.apply(x)
        assert abs(a - b) <= 1e-13 * abs(a)


def test_pcg_matches_oracle_cg():
    dims, p = (4, 3, 3), 2
    V = perturbed_vertices(*dims)
    c = lognormal_coefficient(int(np.prod(dims)), 1.0)
    prob = oop.Problem(*dims, p, V, coeff=c)
    b = load_vector(prob)
    m = boundary_mask(*dims, p)
    keep = 1.0 - m
    A = oop.assemble(prob, DIFFUSION)
    dref = oop.diagonal(prob, DIFFUSION)
    xr, it, _ = oracle_pcg(lambda v: keep * (A @ (keep * v)) + m * v, b * keep, dref * keep + m,
                           rtol=1e-10)
    op = sumfact_c.Operator(*dims, p, V, "diffusion", coeff=c)
    x, it_c, rel = op.pcg(b, m, op.diagonal(), 1e-10, 1000)
    assert rel <= 1e-10 and abs(it_c - it) <= 1
    assert np.abs(x - xr).max() <= 1e-9 * np.abs(xr).max()
    assert np.all(x[m == 1] == 0.0)


def test_results_do_not_depend_on_the_thread_count():
    code = ("import numpy as np, sys; sys.path.insert(0, %r)\n"
            "from oracle import sumfact_c\n"
            "from paper_2603_09038_gb300.inputs import perturbed_vertices, uniform_vector\n"
            "V = perturbed_vertices(5, 4, 3); op = sumfact_c.Operator(5, 4, 3, 3, V, 'diffusion')\n"
            "y = op.apply(uniform_vector(op.ndofs, 0)); sys.stdout.write(y.tobytes().hex())\n" % ROOT)
    outs = []
    for t in ("1", "3"):
        env = dict(os.environ, OMP_NUM_THREADS=t)
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                           check=True, timeout=300)
        outs.append(r.stdout)
    assert outs[0] == outs[1] and len(outs[0]) > 0
