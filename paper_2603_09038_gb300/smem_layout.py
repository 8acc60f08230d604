"""Generator of csrc/fe_smem_layout.h: shared-memory strides of the fused apply kernel chosen to
minimise bank conflicts (a build-time helper; the library itself never runs it).

The apply kernel (csrc/fe_apply_kernel.cuh) keeps two buffers per element, A and B, and every
phase reads or writes them through slabs of fixed stride: S_DD (D^2 slabs), S_QD (QD slabs),
S_QQ (Q^2 slabs), and per-element strides SZ_A, SZ_B.  A warp's shared-memory access costs as
many wavefronts as the largest number of distinct 32-bit words it requests from one of the 32
banks (an 8-byte access as two half-warps of 16 threads, each on its own).  This script
enumerates, for each order, operator, element size (4-byte floats, 8-byte doubles or float pairs)
and z-phase re-read mode, the warp accesses of all seven phases exactly
as the kernel issues them (lines dealt out flat to consecutive threads), counts the wavefronts,
and keeps the strides with the fewest -- among those that leave the kernel's elements per block
(the largest power of two that fits the shared-memory budget) and its blocks per SM as far as
shared memory limits them unchanged.  A stride search per
buffer is exact because the two buffers' phases are disjoint and the buffer B base shifts every
address of a warp alike.

    python paper_2603_09038_gb300/smem_layout.py    # rewrites csrc/fe_smem_layout.h (~minutes)
"""
import multiprocessing as mp
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "csrc", "fe_smem_layout.h")

# (name, element bytes, shared-memory budget, z re-read from order D on) of the three kernels
VARIANTS = [("f64", 8, 96 * 1024, 5), ("f32x2", 8, 96 * 1024, 2), ("f32", 4, 48 * 1024, 2)]
A_PHASES = {"gather.w", "x.r", "y.w", "z.r", "yT.w", "xT.r"}


def odd_pad(n):
    return n + 1 if n % 2 == 0 else n


def default_layout(D, Q, diff):
    s_dd, s_qd, s_qq = odd_pad(D * D), odd_pad(Q * D), odd_pad(Q * Q)
    nf, nq = (2, 3) if diff else (1, 1)
    return (s_dd, s_qd, s_qq, max(D * s_dd, nq * D * s_qq, nf * Q * s_dd),
            max(nf * D * s_qd, nq * Q * s_qd, D ** 3))


def min_sizes(D, Q, diff, s_dd, s_qd, s_qq):
    nf, nq = (2, 3) if diff else (1, 1)
    return (max(D * s_dd, nq * D * s_qq, nf * Q * s_dd), max(nf * D * s_qd, nq * Q * s_qd, D ** 3))


def accesses(D, Q, NE, diff, s_dd, s_qd, s_qq, sz_a, sz_b, reread):
    """(phase, addresses [instructions, threads]) in element units, as the kernel issues them."""
    D2, D3, Q2, QD = D * D, D ** 3, Q * Q, Q * D
    b0 = NE * sz_a
    nf, nq = (2, 3) if diff else (1, 1)
    out = []
    t = np.arange(NE * D3)
    el, a = np.divmod(t, D3)
    out.append(("gather.w", (el * sz_a + (a % D) * s_dd + ((a // D) % D) * D + a // D2)[None, :]))
    t = np.arange(NE * D2)
    el, l = np.divmod(t, D2)
    j, k = np.divmod(l, D)
    out.append(("x.r", np.stack([el * sz_a + l + i * s_dd for i in range(D)])))
    out.append(("x.w", np.stack([b0 + el * sz_b + c * D * s_qd + j * s_qd + k * Q + q
                                 for c in range(nf) for q in range(Q)])))
    t = np.arange(NE * QD)
    el, l = np.divmod(t, QD)
    k, qx = np.divmod(l, Q)
    out.append(("y.r", np.stack([b0 + el * sz_b + l + c * D * s_qd + jj * s_qd
                                 for c in range(nf) for jj in range(D)])))
    out.append(("y.w", np.stack([el * sz_a + c * D * s_qq + k * s_qq + qx + qy * Q
                                 for c in range(nq) for qy in range(Q)])))
    t = np.arange(NE * Q2)
    el, l = np.divmod(t, Q2)
    qy, qx = np.divmod(l, Q)
    reps = Q if reread else 1
    out.append(("z.r", np.stack([el * sz_a + l + c * D * s_qq + kk * s_qq
                                 for _ in range(reps) for c in range(nq) for kk in range(D)])))
    out.append(("z.w", np.stack([b0 + el * sz_b + c * Q * s_qd + qy * s_qd + qx + kk * Q
                                 for c in range(nq) for kk in range(D)])))
    t = np.arange(NE * QD)
    el, l = np.divmod(t, QD)
    k, qx = np.divmod(l, Q)
    out.append(("yT.r", np.stack([b0 + el * sz_b + l + c * Q * s_qd + q * s_qd
                                  for _ in range(2) for c in range(nq) for q in range(Q)])))
    out.append(("yT.w", np.stack([el * sz_a + c * Q * s_dd + qx * s_dd + k + jj * D
                                  for c in range(nf) for jj in range(D)])))
    t = np.arange(NE * D2)
    el, l = np.divmod(t, D2)
    j, k = np.divmod(l, D)
    out.append(("xT.r", np.stack([el * sz_a + l + c * Q * s_dd + q * s_dd
                                  for _ in range(2) for c in range(nf) for q in range(Q)])))
    out.append(("xT.w", np.stack([b0 + el * sz_b + j * D + k * D2 + i for i in range(D)])))
    t = np.arange(NE * D3)
    el, a = np.divmod(t, D3)
    out.append(("scatter.r", (b0 + el * sz_b + a)[None, :]))
    return out


def wavefronts(addr, es):
    """Sum over warp instructions of max over banks of the distinct 32-bit words requested; an
    8-byte access is served as two half-warps of 16 threads, each counted on its own."""
    ni, nt = addr.shape
    lanes = 32 if es == 4 else 16
    nw = (nt + lanes - 1) // lanes
    A = np.pad(addr, ((0, 0), (0, nw * lanes - nt)), constant_values=-1).reshape(ni, nw, lanes)
    wpe = es // 4
    W = (A[..., None] * wpe + np.arange(wpe)).reshape(ni, nw, lanes * wpe)
    W = np.where(np.repeat(A >= 0, wpe, axis=2), W, -1)
    W.sort(axis=2)
    dup = np.zeros_like(W, dtype=bool)
    dup[..., 1:] = W[..., 1:] == W[..., :-1]
    bank = np.where((W >= 0) & ~dup, W % 32, 32)
    cnt = np.zeros((ni, nw, 33), dtype=np.int32)
    np.add.at(cnt, (np.arange(ni)[:, None, None], np.arange(nw)[None, :, None], bank), 1)
    return int(cnt[..., :32].max(axis=2).sum())


def split_cost(D, Q, NE, es, diff, lay, reread):
    ca = cb = 0
    for name, addr in accesses(D, Q, NE, diff, *lay, reread=reread):
        w = wavefronts(addr, es)
        if name in A_PHASES:
            ca += w
        else:
            cb += w
    return ca, cb


def elems_per_block(per_elem, es, smem):
    ne = smem // (per_elem * es)
    p2 = 1
    while p2 * 2 <= ne and p2 < 64:
        p2 *= 2
    return p2


SM_SMEM = 233472      # shared memory per SM on GB300 (228 KB)
BLOCK_RESERVED = 1024  # shared memory the runtime reserves per block


def blocks_by_smem(per_elem, ne, es):
    return SM_SMEM // (ne * per_elem * es + BLOCK_RESERVED)


def search(task):
    D, diff, es, smem, rr = task
    Q = D + 1
    cur = default_layout(D, Q, diff)
    NE = elems_per_block(cur[3] + cur[4], es, smem)
    cap = smem // (NE * es)
    # keep the blocks per SM that shared memory allows (a larger layout could cost occupancy)
    occ = min(blocks_by_smem(cur[3] + cur[4], NE, es), 8)
    while cap > cur[3] + cur[4] and blocks_by_smem(cap, NE, es) < occ:
        cap -= 1
    base = sum(split_cost(D, Q, NE, es, diff, cur, rr))
    slack = 6 if D <= 5 else 4
    best = (base, cur)
    for s_dd in range(D * D, D * D + slack):
        for s_qd in range(Q * D, Q * D + slack):
            for s_qq in range(Q * Q, Q * Q + slack):
                amin, bmin = min_sizes(D, Q, diff, s_dd, s_qd, s_qq)
                ca = [split_cost(D, Q, NE, es, diff, (s_dd, s_qd, s_qq, amin + da, bmin), rr)[0]
                      for da in range(32)]
                cb = [split_cost(D, Q, NE, es, diff, (s_dd, s_qd, s_qq, amin, bmin + db), rr)[1]
                      for db in range(32)]
                for da in range(32):
                    for db in range(32):
                        per = amin + da + bmin + db
                        if per > cap:
                            continue
                        c = ca[da] + cb[db]
                        if c < best[0] or (c == best[0] and per < best[1][3] + best[1][4]):
                            best = (c, (s_dd, s_qd, s_qq, amin + da, bmin + db))
    return task, NE, base, best


def main():
    tasks = set()
    for _, es, smem, rr_from in VARIANTS:
        for D in range(2, 10):
            for diff in (True, False):
                tasks.add((D, diff, es, smem, D >= rr_from))
    tasks = sorted(tasks)
    with mp.get_context("spawn").Pool(min(8, os.cpu_count() or 1)) as pool:
        results = pool.map(search, tasks)
    lines = []
    for (D, diff, es, smem, rr), NE, base, (c, lay) in results:
        if lay == default_layout(D, D + 1, diff):
            continue
        lines.append("    {%d, %d, %d, %d, %d, %d, %d, %d, %d, %d},  // NE %d: %d -> %d wavefronts"
                     % (D, D + 1, int(diff), es, int(rr), *lay, NE, base, c))
    with open(OUT, "w") as f:
        f.write("""// Generated by paper_2603_09038_gb300/smem_layout.py (do not edit): shared-memory strides of the
// fused apply kernel that minimise bank conflicts in a model of its warp accesses, keeping the
// elements per block of the default layout.  Key: D, Q, diffusion, element bytes, z re-read.
#pragma once

namespace fe {

struct SmemLayoutEntry {
  int D, Q, diff, es, rr;
  int s_dd, s_qd, s_qq, sz_a, sz_b;
};

constexpr SmemLayoutEntry kSmemLayouts[] = {
%s
    {0, 0, 0, 0, 0, 0, 0, 0, 0, 0}};

}  // namespace fe
""" % "\n".join(lines))
    print("wrote %s (%d tuned layouts)" % (OUT, len(lines)))


if __name__ == "__main__":
    main()
