"""CPU FP64 oracle for the partial-assembly finite element operators (TEST INFRASTRUCTURE).

This package is the plain, slow, obviously-correct reference that the CUDA path is checked
against.  It is test infrastructure only: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it; the library itself never does, and nothing in
it is shared with the CUDA path (no kernels, tables, helpers or constants).

What it computes (paper: Section II-B, Eq. (1) ``A = P^T G^T B^T D B G P`` and Eq. (2), the
tensor-product basis ``B_abc,ijk = B1d_ai B1d_bj B1d_ck``).  The paper only states the generic
decomposition; for the H1 diffusion and mass operators on hexahedra the oracle uses the standard
Galerkin forms (the paper is silent on them):

    K_ab = sum_e sum_q w_q c_e |det J_e(x_q)| (J_e^{-T} grad phi_a) . (J_e^{-T} grad phi_b)
    M_ab = sum_e sum_q w_q c_e |det J_e(x_q)| phi_a phi_b

``element.py`` builds these element matrices by direct quadrature (no sum factorisation) and
``operator.py`` applies them as ``y = sum_e G_e^T K_e G_e x`` -- the plain definition.  The
sum-factorised apply in ``sumfact.py`` is a second, independent route used only to cross-check
the first on tiny meshes (brute-force agreement) and as the timed CPU baseline.
``solve.py`` holds CG / preconditioned CG and the Chebyshev polynomial preconditioner,
``mlp.py`` the learned preconditioner's network (forward, loss, backpropagation), and
``varorder.py`` the variable-order space: the constraint operator P of Eq. (1) under the
minimum rule, its Jacobi diagonal and operator; ``mixed.py`` the paper's own mixed H1/L2
gradient / divergence pair (Eq. (block-mult)'s off-diagonal blocks).

Parity status of every function is pinned by the ``-m "not gpu"`` tests in ``tests/``:
closed-form 1D rules, textbook element matrices, volume, null space, symmetry, exact polynomial
integration, O(h^{p+1}) convergence, dense-solve agreement and brute-force cross-checks; for the
network finite differences and the least-squares special case; for the variable-order space a
hand-derived numbering, the dimension of the continuous space by brute force, polynomial
reproduction, closed-form energies and the single-order case.
"""
