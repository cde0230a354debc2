"""The benchmark's multi-rank path on CPU: world size 2 over gloo.  Each rank
is an independent replica; the job's time is the max over ranks and its units
the sum (the only collective of the path)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    out = bench.aggregate(1.5 + rank, 2.0 * (rank + 1), 10 + 5 * rank)
    q.put((rank, out))
    dist.destroy_process_group()


def test_aggregate_world_size_two():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs)
    for r in range(2):
        dev_s, wall, units = res[r]
        assert dev_s == 2.5 and wall == 4.0 and units == 25


def test_aggregate_single_process_is_identity():
    import bench
    assert bench.aggregate(1.0, 2.0, 3) == (1.0, 2.0, 3)
