"""bench.py's whole-job timing over ranks, world size 2 with gloo on CPU."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    sec, work = bench.reduce_over_ranks(1.0 + rank, [10.0 * (rank + 1), 0.5], dist, None)
    out.put((rank, sec, work))
    dist.destroy_process_group()


def test_reduce_over_ranks_gloo():
    mp = pytest.importorskip("torch.multiprocessing")
    import socket
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, sec, work in res:
        assert sec == 2.0                     # slowest rank
        assert work == [30.0, 1.0]            # summed over ranks


def test_reduce_single_rank():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_over_ranks(1.5, [3.0]) == (1.5, [3.0])
