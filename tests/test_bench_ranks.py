"""The multi-rank bookkeeping of bench.py on CPU: world size 2 over gloo.

With N GPUs the path runs N independent replicas (the method has no exchange
step); the only collective is the max over ranks of the timed region, and the
reported value is the units all replicas processed over that time.  The
reference arm prints from rank 0 only.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys

    sys.path.insert(0, ROOT)
    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 100.0 + 50.0 * rank  # the replicas' own times; rank 1 is the slowest
        m = bench.rank_max(ms, world, "cpu")
        out[rank] = (m, bench.job_value(1000.0, 4, world, m))
        # the reference arm: every rank but 0 returns at once, without output
        if rank != 0:
            out[10 + rank] = bench.run_reference(None, rank, world)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_replicas_over_gloo():
    world = 2
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        m, v = res[r]
        assert m == 150.0  # the slowest replica's time on every rank
        assert v == pytest.approx(2 * 1000.0 * 4 / 0.150)
    assert res[11] is None


def test_single_rank_needs_no_process_group():
    import sys

    sys.path.insert(0, ROOT)
    import bench

    assert bench.rank_max(3.5, 1, "cpu") == 3.5
    assert bench.job_value(10.0, 2, 1, 1000.0) == pytest.approx(20.0)
