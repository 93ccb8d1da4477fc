"""The bench's multi-rank timing on CPU with two gloo ranks: every rank sees the slowest rank's
time, and the whole-job value counts every rank's voxels (replicas, weak scaling)."""
import multiprocessing as mp
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench.max_over_ranks(10.0 + 5.0 * rank, dist, "cpu")
    q.put((rank, t, bench.whole_job_mvox_s(world, 1_000_000, t)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_report_the_slowest_rank():
    pytest.importorskip("torch.distributed")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert [g[1] for g in got] == [15.0, 15.0]
    assert all(abs(g[2] - 2 * 1_000_000 / 15.0 / 1e6) < 1e-12 for g in got)


def test_single_process_is_unchanged():
    import bench
    assert bench.max_over_ranks(3.5, None) == 3.5
    assert bench.whole_job_mvox_s(1, 2_000_000, 0.5) == 4.0
