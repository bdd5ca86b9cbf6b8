"""Replica ranks of bench.py on CPU: world size 2 over gloo (127.0.0.1).

The force path shards into independent replicas (or independent volumes)
with no exchange; the only cross-rank operations are the timing barrier and
the max / sum reductions that turn per-rank times and pair counts into the
whole-job figures."""

import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    r = bench.Ranks("gloo")
    r.barrier()
    mx = r.max(10.0 + rank)          # per-rank step times -> the slowest
    sm = r.sum(1000.0 * (rank + 1))  # per-rank pair counts -> whole job
    r.barrier()
    q.put((rank, mx, sm))
    r.close()


def test_two_gloo_ranks_reduce_like_the_bench():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, mx, sm in out:
        assert mx == 11.0
        assert sm == 3000.0
