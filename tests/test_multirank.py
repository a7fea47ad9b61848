"""The benchmark's multi-rank host logic (one process per GPU, replicas
only): disjoint image shards per rank and the job time as the maximum over
ranks, on world size 2 with the gloo backend (CPU only)."""
import os
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        steps = bench.shard_steps(rank, 3, 5)
        t = bench.max_over_ranks(10.0 * (rank + 1), world)
        out.put((rank, steps, t))
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_and_max():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 1000)
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    s0, s1 = set(res[0][1]), set(res[1][1])
    assert len(s0) == len(s1) == 8 and not (s0 & s1)
    assert res[0][2] == res[1][2] == 20.0


def test_single_rank_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert bench.shard_steps(0, 3, 12) == list(range(15))
