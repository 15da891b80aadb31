"""The multi-rank path of bench.py on CPU: world_size 2 over gloo.

Queries are independent, so ranks shard the source list with no data-path
collective; the only exchange is the max-over-ranks of the timed interval.
"""
import os

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _worker(rank, world, port, times, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    sources = np.arange(64, dtype=np.int32) * 7
    mine = bench.shard_sources(sources, rank, world)
    got = bench.max_over_ranks(times[rank], dist, torch.device("cpu"))
    gathered = [None] * world
    dist.all_gather_object(gathered, mine.tolist())
    out.put((rank, got, gathered))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_shard_sources_and_take_the_slowest_time():
    world, port = 2, 29500 + os.getpid() % 1000
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    times = [1.25, 3.5]
    procs = [ctx.Process(target=_worker, args=(r, world, port, times, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, gathered in res:
        assert got == max(times)
        flat = sorted(x for part in gathered for x in part)
        assert flat == sorted((np.arange(64) * 7).tolist())     # every source once
        assert not set(gathered[0]) & set(gathered[1])           # disjoint shards


def test_single_rank_is_identity():
    import bench
    s = np.arange(10)
    assert bench.shard_sources(s, 0, 1) is s
    assert bench.max_over_ranks(2.5, None, None) == 2.5
