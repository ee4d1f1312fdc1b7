"""Replica aggregation of bench.py with two gloo ranks on the CPU: every rank
times its own independent copy of the step, the slowest rank's time is the
job's time and the value counts all ranks' steps."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        my_ms = 100.0 + 50.0 * rank          # rank 1 is the slow replica
        mx = bench.replica_max(dist, my_ms)
        q.put((rank, mx, bench.replica_value(world, 10, mx)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, mx, value in got:
        assert mx == 150.0
        assert value == pytest.approx(2 * 10 / 0.150)


def test_single_rank_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.replica_max(None, 12.5) == 12.5
    assert bench.replica_value(1, 4, 500.0) == pytest.approx(8.0)
