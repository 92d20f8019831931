"""The benchmark's multi-rank path (replicas only: no data-path collective) on CPU
ranks over gloo: rendezvous, barrier and the max-over-ranks timing reduction."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    os.environ.update({"RANK": str(rank), "LOCAL_RANK": str(rank), "WORLD_SIZE": str(world),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    w, r, local = bench.dist_init()
    bench.barrier(w)
    m = bench.allreduce_max(10.0 * (rank + 1), w)
    q.put((r, w, m, dist.get_backend()))
    dist.destroy_process_group()


def test_two_cpu_ranks_reduce_max():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=5) for _ in range(2))
    assert [o[0] for o in out] == [0, 1]
    assert all(o[1] == 2 and o[2] == 20.0 and o[3] == "gloo" for o in out)
