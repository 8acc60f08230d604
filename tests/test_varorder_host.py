"""The library's host construction of the variable-order space (numbering, E, layout, boundary
mask) against the oracle, through the host-only C-ABI entry fe_vspace_host_E (CPU only: no GPU
and no CUDA call is involved)."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle.varorder import VarSpace
from paper_2603_09038_gb300.inputs import block_orders

CASES = [
    ((2, 1, 1), [1, 2]),
    ((2, 2, 2), [1, 2, 3, 2, 2, 1, 3, 2]),
    ((4, 4, 4), block_orders(4, 4, 4, block=2, orders=(2, 4, 6), seed=1)),
    ((5, 4, 3), block_orders(5, 4, 3, block=1, orders=(1, 2, 3, 4, 5), seed=2)),
    ((3, 2, 2), block_orders(3, 2, 2, block=1, orders=(5, 6, 7, 8), seed=4)),
    ((3, 3, 3), [3] * 27),
]


def _library_sparsity(E):
    """The oracle's E with the library's documented drop rule (|weight| <= 1e-13) applied."""
    E = E.tocsr(copy=True)
    E.data[np.abs(E.data) <= 1e-13] = 0.0
    E.eliminate_zeros()
    return E


def _lib():
    from tests.gpu_util import lib
    return lib()


@pytest.mark.parametrize("dims,orders", CASES)
def test_host_E_matches_oracle(dims, orders):
    fe = _lib()
    S = VarSpace(*dims, orders)
    E = S.prolongation()
    ntrue, rowptr, cols, vals, first, mask = fe.fe_vspace_host_E(*dims, orders)
    assert ntrue == S.ntrue and len(rowptr) == S.nlocal + 1
    El = sp.csr_matrix((vals, cols, rowptr), shape=(S.nlocal, S.ntrue))
    perm = np.concatenate([first[e] + np.arange(int(S.local_size[e])) for e in range(S.ne)])
    # by value: the library drops weights of magnitude <= 1e-13 (its documented rule, so that
    # E's sparsity does not depend on rounding); the oracle keeps every computed weight
    assert abs(El[perm] - E).max() <= 1e-13
    assert rowptr[-1] == _library_sparsity(E).nnz
    np.testing.assert_array_equal(mask, S.boundary_mask())
    # layout: groups of ascending order, elements ascending within each
    key = sorted(range(S.ne), key=lambda e: (S.order[e], e))
    expect = np.zeros(S.ne, dtype=np.int64)
    off = 0
    for e in key:
        expect[e] = off
        off += int(S.order[e] + 1) ** 3
    np.testing.assert_array_equal(first, expect)


def test_host_E_rejects_bad_orders():
    fe = _lib()
    for bad in ([0] + [2] * 7, [9] + [2] * 7):
        with pytest.raises(fe.FEError) as ei:
            fe.fe_vspace_host_E(2, 2, 2, bad)
        assert ei.value.status == fe.FE_ERR_ARG
