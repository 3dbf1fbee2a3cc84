"""Multi-rank path of bench.py on the CPU: two gloo ranks, each with its own
per-rank timings; the job's value is the element-wise maximum (replicas run
independent instances; the slowest one ends the job)."""
import os
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    per_rank = [[10.0, 12.5], [11.0, 12.0]]
    res = bench.max_over_ranks(per_rank[rank], torch.device("cpu"))
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, res))


def test_max_over_ranks_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 1000)
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got[0] == got[1] == [11.0, 12.5]
