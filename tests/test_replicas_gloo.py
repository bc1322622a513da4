"""The N > 1 path of bench.py (independent replicas, max-over-ranks time) on
two CPU ranks with the gloo backend: the job time is the slowest rank's and the
value counts every rank's terms."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r took 1 + r seconds for 2 steps of 100 terms
        value, ms = bench.combine_replicas(1.0 + rank, 100, 2, world, dist, "cpu")
        out[rank] = (value, ms)
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank_time():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        value, ms = res[r]
        assert ms == pytest.approx(1000.0)  # 2 s over 2 steps, the slower rank's
        assert value == pytest.approx(100 * 2 * 2 / 2.0)


def test_single_replica_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    value, ms = bench.combine_replicas(4.0, 9248, 1, 1)
    assert value == pytest.approx(9248 / 4.0)
    assert ms == pytest.approx(4000.0)
