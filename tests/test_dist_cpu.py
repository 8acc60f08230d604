"""Multi-process host logic of bench.py on CPU (gloo, world size 2): the slowest rank's time is
what every rank reports, and the whole-job throughput counts every rank's independent problem."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist          # noqa: E402
import torch.multiprocessing as mp        # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=world)
    try:
        t = 1.0 + rank                       # rank 1 is the slow one
        tmax = bench.max_over_ranks(t, dist, "cpu")
        q.put((rank, tmax, bench.job_gdofs(world, 1000, 10, tmax)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_report_the_slowest_time_and_the_job_total():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, tmax, gd in res:
        assert tmax == 2.0
        assert abs(gd - 2 * 1000 * 10 / 2.0 / 1e9) < 1e-18


def test_single_process_identity():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_gdofs(1, 2_000_000_000, 1, 2.0) == 1.0
