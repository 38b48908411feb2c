"""The benchmark's multi-rank reduction (replicas: sum of units, max of seconds) on
two gloo ranks on CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    units, secs = bench.aggregate(1000.0 * (rank + 1), 0.5 + rank)
    q.put((rank, units, secs))
    dist.destroy_process_group()


def test_aggregate_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get() for _ in range(2))
    for _, units, secs in res:
        assert units == pytest.approx(3000.0)
        assert secs == pytest.approx(1.5)


def test_single_process_passthrough():
    import bench
    assert bench.aggregate(5.0, 2.0) == (5.0, 2.0)
