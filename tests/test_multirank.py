"""The multi-rank paths on CPU: world_size 2 over gloo.

* Source-parallel benchmark (weak scaling): every rank runs its own 64-source
  list; the only exchange is the max-over-ranks of the timed interval.
* One query split by target range (the owner rule of Section 5.5): rank r
  computes the targets u with floor(u N / n) = r and the slices are
  all-gathered.  The per-rank compute here is the oracle on that rank's
  targets (the CUDA path needs a GPU); the gathered counts, weight sums and
  scores must equal one whole oracle query bit for bit.
"""
import os

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _bench_worker(rank, world, port, times, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    mine = bench.source_list(1 << 16, rank).tolist()
    got = bench.max_over_ranks(times[rank], dist, torch.device("cpu"))
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    out.put((rank, got, gathered))
    dist.barrier()
    dist.destroy_process_group()


def _split_worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import sampler
    from paper_2304_04015_gb300.split import gather_slices, owner_of, owner_range
    from srk_inputs import er_in_csr
    n = 301
    rp, col = er_in_csr(n, 5.0, seed=4)
    b, e = owner_range(n, rank, world)
    assert all(owner_of(u, n, world) == rank for u in range(b, e))
    part = sampler.run(rp, col, n, 7, 0.6, 0.1, 11, targets=np.arange(b, e, dtype=np.int32),
                       z_override=300.0, L_override=12, threads=1)
    got = [gather_slices(torch.from_numpy(a.astype(dt)), n, rank, world).numpy()
           for a, dt in ((part.count, np.int32), (part.wsum, np.int64), (part.scores, np.float64))]
    out.put((rank, got))
    dist.barrier()
    dist.destroy_process_group()


def _spawn(target, world, *args):
    port = 29500 + (os.getpid() * 7 + hash(target.__name__)) % 2000
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=target, args=(r, world, port) + args + (q,))
             for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=180) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return res


def test_two_ranks_run_own_source_lists_and_take_the_slowest_time():
    times = [1.25, 3.5]
    for rank, got, gathered in _spawn(_bench_worker, 2, times):
        assert got == max(times)
        assert len(gathered[0]) == len(gathered[1]) == 64
        assert gathered[0] != gathered[1]     # each rank its own list (weak scaling)


@pytest.fixture(scope="module")
def built():
    import __graft_entry__
    __graft_entry__.build()      # the split helper lives in the package (loads libsrk.so)


def test_target_split_over_two_ranks_equals_one_query(built):
    from oracle import sampler
    from srk_inputs import er_in_csr
    n = 301
    rp, col = er_in_csr(n, 5.0, seed=4)
    whole = sampler.run(rp, col, n, 7, 0.6, 0.1, 11, z_override=300.0, L_override=12,
                        threads=1)
    assert whole.count.sum() > 0
    for rank, (cnt, wsum, scores) in _spawn(_split_worker, 2):
        assert np.array_equal(cnt.astype(np.uint32), whole.count)
        assert np.array_equal(wsum.astype(np.uint64), whole.wsum)
        assert np.array_equal(scores, whole.scores)


def test_owner_ranges_partition_the_targets(built):
    from paper_2304_04015_gb300.split import owner_of, owner_range
    for n in (1, 2, 5, 301, 1 << 20):
        for world in (1, 2, 3, 7, 8):
            ranges = [owner_range(n, r, world) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == n
            for (b0, e0), (b1, _) in zip(ranges, ranges[1:]):
                assert e0 == b1 and b0 <= e0
            for u in {0, n - 1, n // 2, n // 3}:
                r = owner_of(u, n, world)
                assert ranges[r][0] <= u < ranges[r][1]
    with pytest.raises(ValueError):
        owner_range(10, 2, 2)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(2.5, None, None) == 2.5
    a = bench.source_list(1 << 16, 0)
    assert np.array_equal(a, bench.source_list(1 << 16, 0)) and a.size == 64
