"""srk_single_source_noalloc against srk_single_source (GPU).

The no-allocation entry point serves callers that must not allocate device
memory while they query (their own allocator owns the device budget, or the
calling thread must not block on the driver's allocator).  It runs the same
kernels with scratch taken from a static device array.  Its results must equal
those of the allocating entry point bit for bit -- the tolerance every parity
test here uses for counts, weight sums and scores -- on two calls in a row,
the second of which finds the first call's leftovers in the shared scratch.
It must also allocate nothing: across calls made after the first (which takes
the scratch address), neither the library's memory pool (its high-water mark
of memory handed out) nor the device's free memory may change.
This file is collected last so that a stop-at-first-failure run has already
run every other test.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def srk():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2304_04015_gb300 as m
    return m


def _query(fn, g, n, s, eps, seed, dev, **kw):
    import torch
    scores = torch.full((n,), -1.0, dtype=torch.float64, device=dev)
    counts = torch.full((n,), -1, dtype=torch.int32, device=dev)
    wsums = torch.full((n,), -1, dtype=torch.int64, device=dev)
    steps = torch.full((n,), -1, dtype=torch.int32, device=dev)
    fn(g, s, 0.6, eps, seed, scores, counts, wsums, step_counts=steps, **kw)
    torch.cuda.synchronize()
    return [t.cpu().numpy() for t in (scores, counts, wsums, steps)]


def test_no_alloc_matches_allocating_entry_point(srk):
    import torch
    from srk_inputs import er_in_csr, rmat_in_csr
    dev = torch.device("cuda:0")
    cases = []
    rp, col = er_in_csr(1000, 5.0, seed=1)
    cases.append((rp, col, [(0, 0.1, 1, dict(z_override=2000.0, L_override=32)),
                            (17, 0.1, 2, dict(z_override=2000.0, L_override=32)),
                            (5, 0.1, 3, dict(z_override=2000.0, L_override=32,
                                             literal_shuffle=True))]))
    rp16, col16 = rmat_in_csr(16, seed=1)
    hub = int(np.argmax(np.diff(rp16)))
    cases.append((rp16, col16, [(hub, 0.05, 3, {}), (12345, 0.05, 4, {})]))
    for rp, col, calls in cases:
        n = rp.size - 1
        g = srk.srk_graph_load(torch.from_numpy(rp).to(dev), torch.from_numpy(col).to(dev))
        try:
            # two no-alloc calls in a row, each checked against the pool path
            for s, eps, seed, kw in calls:
                got = _query(srk.srk_single_source_noalloc, g, n, s, eps, seed, dev, **kw)
                ref = _query(srk.srk_single_source, g, n, s, eps, seed, dev, **kw)
                for a, b in zip(got, ref):
                    assert np.array_equal(a, b)
                assert got[1].sum() > 0
        finally:
            g.close()


def test_no_alloc_rejects_what_it_cannot_hold(srk):
    import torch
    from srk_inputs import er_in_csr
    dev = torch.device("cuda:0")
    rp, col = er_in_csr(200, 3.0, seed=2)
    g = srk.srk_graph_load(torch.from_numpy(rp).to(dev), torch.from_numpy(col).to(dev))
    try:
        out = torch.empty(200, dtype=torch.float64, device=dev)
        with pytest.raises(srk.SrkError) as e:   # scratch larger than the static array
            srk.srk_single_source_noalloc(g, 0, 0.6, 0.5, 1, out, z_override=2.0e6)
        assert e.value.code == srk.SRK_EINVAL and "scratch" in str(e.value)
        with pytest.raises(srk.SrkError) as e:   # host outputs would need staging
            srk.srk_single_source_noalloc(g, 0, 0.6, 0.5, 1, np.empty(200))
        assert e.value.code == srk.SRK_EINVAL
    finally:
        g.close()


def test_no_alloc_allocates_nothing(srk):
    import torch
    from srk_inputs import rmat_in_csr
    dev = torch.device("cuda:0")
    rp, col = rmat_in_csr(16, seed=1)
    n = rp.size - 1
    hub = int(np.argmax(np.diff(rp)))
    g = srk.srk_graph_load(torch.from_numpy(rp).to(dev), torch.from_numpy(col).to(dev))
    try:
        outs = [torch.empty(n, dtype=torch.float64, device=dev) for _ in range(2)]
        counts = torch.empty(n, dtype=torch.int32, device=dev)
        # the first call in this context looks up the scratch address (and
        # loads the kernels): set-up, outside the measured calls
        srk.srk_single_source_noalloc(g, hub, 0.6, 0.05, 1, outs[0], counts)
        torch.cuda.synchronize()
        _, used0, _ = srk.srk_pool_stats(0, reset_high=True)
        free0, _ = torch.cuda.mem_get_info(dev)
        for k, seed in enumerate((2, 3)):
            srk.srk_single_source_noalloc(g, hub, 0.6, 0.05, seed, outs[k], counts)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info(dev)
        _, used1, high1 = srk.srk_pool_stats(0)
        assert high1 == used0 and used1 == used0     # no pool allocation in the calls
        assert free1 == free0                        # and no other device allocation
        assert not torch.equal(outs[0], outs[1])     # two different queries ran
        assert int(counts.sum()) > 0
    finally:
        g.close()
