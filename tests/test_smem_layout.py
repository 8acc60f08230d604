"""The generated shared-memory layouts of the apply kernel (csrc/fe_smem_layout.h): every entry
is large enough for the phases' arrays, keeps the kernel's elements per block and its
shared-memory-limited blocks per SM, and has fewer modelled bank-conflict wavefronts than the
default padded layout (spot check of the model)."""
import os
import re

import pytest

from paper_2603_09038_gb300 import smem_layout as sl

HDR = os.path.join(os.path.dirname(sl.__file__), "csrc", "fe_smem_layout.h")


def entries():
    rows = []
    for line in open(HDR):
        m = re.match(r"\s*\{(\d+), (\d+), (\d+), (\d+), (\d+), (\d+), (\d+), (\d+), (\d+), (\d+)\},", line)
        if m and int(m.group(1)) > 0:
            rows.append(tuple(int(g) for g in m.groups()))
    return rows


def test_entries_valid_and_keep_elements_per_block():
    rows = entries()
    assert rows, "no tuned layouts in the generated header"
    budgets = {(es, rr): smem for _, es, smem, _ in sl.VARIANTS for rr in (0, 1)}
    for D, Q, diff, es, rr, s_dd, s_qd, s_qq, sz_a, sz_b in rows:
        assert Q == D + 1
        amin, bmin = sl.min_sizes(D, Q, bool(diff), s_dd, s_qd, s_qq)
        assert s_dd >= D * D and s_qd >= Q * D and s_qq >= Q * Q
        assert sz_a >= amin and sz_b >= bmin
        smem = budgets[(es, rr)]
        cur = sl.default_layout(D, Q, bool(diff))
        ne = sl.elems_per_block(cur[3] + cur[4], es, smem)
        assert sl.elems_per_block(sz_a + sz_b, es, smem) == ne
        occ = min(sl.blocks_by_smem(cur[3] + cur[4], ne, es), 8)
        assert sl.blocks_by_smem(sz_a + sz_b, ne, es) >= occ


@pytest.mark.parametrize("pick", [0, -1])
def test_tuned_layout_has_fewer_modelled_wavefronts(pick):
    D, Q, diff, es, rr, *lay = entries()[pick]
    budgets = {es_: smem for _, es_, smem, _ in sl.VARIANTS}
    cur = sl.default_layout(D, Q, bool(diff))
    ne = sl.elems_per_block(cur[3] + cur[4], es, budgets[es])
    new = sum(sl.split_cost(D, Q, ne, es, bool(diff), tuple(lay), bool(rr)))
    old = sum(sl.split_cost(D, Q, ne, es, bool(diff), cur, bool(rr)))
    assert new < old


def test_bank_model_known_patterns():
    """Textbook cases of the wavefront model: unit stride is conflict-free (one wavefront for
    4-byte words, one per half-warp for 8-byte words), stride 2 words is a 2-way conflict,
    stride 32 words a 32-way conflict, and a broadcast costs one wavefront."""
    import numpy as np
    t = np.arange(32)[None, :]
    assert sl.wavefronts(t, 4) == 1
    assert sl.wavefronts(2 * t, 4) == 2
    assert sl.wavefronts(32 * t, 4) == 32
    assert sl.wavefronts(0 * t, 4) == 1
    assert sl.wavefronts(t, 8) == 2          # 256 bytes: two half-warps of 128 bytes
    assert sl.wavefronts(2 * t, 8) == 4      # stride 16 bytes: 2-way within each half-warp
    assert sl.wavefronts(17 * t, 8) == 2     # odd stride in 8-byte words: conflict-free halves
