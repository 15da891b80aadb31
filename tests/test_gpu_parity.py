"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Counts, weight sums and step counts are integers: they must match bit for
bit.  Scores are W 2^-32 / z evaluated in IEEE FP64 on both sides, so they
must match bit for bit too.  Accuracy against exact SimRank is Theorem 6's
bound |s~ - s| <= eps on the small configuration.
"""
import functools

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

C = 0.6


@pytest.fixture(scope="module")
def srk():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2304_04015_gb300 as m
    return m


@functools.lru_cache(maxsize=None)
def er_graph(n, deg, seed):
    from srk_inputs import er_in_csr
    return er_in_csr(n, deg, seed=seed)


@functools.lru_cache(maxsize=None)
def rmat_graph(scale, seed=1):
    from srk_inputs import rmat_in_csr
    return rmat_in_csr(scale, seed=seed)


@functools.lru_cache(maxsize=None)
def hub_graph():
    """20,000 nodes, 40 of them hubs with ~9,000 in-neighbours each; every
    node also has two hubs among its in-neighbours, so most walk steps land
    on a hub."""
    from srk_inputs import csr_from_edges
    rng = np.random.default_rng(5)
    n = 20000
    hubs = rng.choice(n, size=40, replace=False)
    src, dst = [], []
    for h in hubs:
        src.append(rng.choice(n, size=9000, replace=False))
        dst.append(np.full(9000, h))
    d = rng.poisson(4.0, size=n)
    dst.append(np.repeat(np.arange(n), d))
    src.append(rng.integers(0, n, size=int(d.sum())))
    dst.append(np.repeat(np.arange(n), 2))
    src.append(hubs[rng.integers(0, 40, size=2 * n)])
    return csr_from_edges(n, np.concatenate(src), np.concatenate(dst))


def gpu_query(srk, rp, col, s, eps, seed, device_outputs=True, **kw):
    import torch
    dev = torch.device("cuda:0")
    n = rp.size - 1
    g = srk.srk_graph_load(torch.from_numpy(rp).to(dev), torch.from_numpy(col).to(dev))
    stats = srk.SrkStats()
    try:
        if device_outputs:
            scores = torch.empty(n, dtype=torch.float64, device=dev)
            counts = torch.empty(n, dtype=torch.int32, device=dev)
            wsums = torch.empty(n, dtype=torch.int64, device=dev)
            steps = torch.empty(n, dtype=torch.int32, device=dev)
            srk.srk_single_source(g, s, C, eps, seed, scores, counts, wsums,
                                  step_counts=steps, stats=stats, **kw)
            torch.cuda.synchronize()
            out = (scores.cpu().numpy(), counts.cpu().numpy().view(np.uint32),
                   wsums.cpu().numpy().view(np.uint64), steps.cpu().numpy().view(np.uint32))
        else:
            scores = np.empty(n, dtype=np.float64)
            counts = np.empty(n, dtype=np.uint32)
            wsums = np.empty(n, dtype=np.uint64)
            steps = np.empty(n, dtype=np.uint32)
            srk.srk_single_source(g, s, C, eps, seed, scores, counts, wsums,
                                  step_counts=steps, stats=stats, **kw)
            out = (scores, counts, wsums, steps)
    finally:
        g.close()
    return out + (stats,)


def oracle_query(rp, col, s, eps, seed, targets=None, **kw):
    from oracle import sampler
    return sampler.run(rp, col, rp.size - 1, s, C, eps, seed, targets=targets, **kw)


def assert_parity(gpu, ref, targets=None):
    scores, counts, wsums, steps, stats = gpu
    sel = slice(None) if targets is None else targets
    assert np.array_equal(counts[sel], ref.count)
    assert np.array_equal(wsums[sel], ref.wsum)
    assert np.array_equal(steps[sel].astype(np.uint64), ref.steps)
    assert np.array_equal(scores[sel], ref.scores)
    assert stats.n_walks == ref.table.N_tot and stats.L == ref.table.L
    assert stats.z == ref.table.z
    assert stats.source_steps == ref.source_steps
    if targets is None:
        assert stats.target_steps == int(ref.steps.sum())


TINY = dict(z_override=2000.0, L_override=32)


def test_tiny_configuration_bit_exact(srk):
    # ER n=1000, Poisson(5) in-degrees, source 0, c=0.6, eps=0.1, 2000 pairs, L=32
    rp, col = er_graph(1000, 5.0, 1)
    for seed in (1, 2):
        gpu = gpu_query(srk, rp, col, 0, 0.1, seed, **TINY)
        ref = oracle_query(rp, col, 0, 0.1, seed, **TINY)
        assert_parity(gpu, ref)
        assert ref.count.sum() > 1000     # the case exercises meetings


def test_tiny_configuration_within_eps_of_exact(srk):
    from oracle import exact
    rp, col = er_graph(1000, 5.0, 1)
    S, _ = exact.jeh_widom(rp, col, 1000, C)
    scores = gpu_query(srk, rp, col, 0, 0.1, 1, **TINY)[0]
    assert scores[0] == 1.0
    assert np.abs(scores - S[0]).max() <= 0.1


def test_host_and_device_outputs_agree(srk):
    rp, col = er_graph(1000, 5.0, 1)
    a = gpu_query(srk, rp, col, 3, 0.1, 9, device_outputs=True, **TINY)
    b = gpu_query(srk, rp, col, 3, 0.1, 9, device_outputs=False, **TINY)
    for x, y in zip(a[:4], b[:4]):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("pick", ["hub", "uniform", "zero_in_degree", "leaf"])
def test_rmat16_paper_parameters_bit_exact(srk, pick):
    rp, col = rmat_graph(16)
    deg = np.diff(rp)
    s = {"hub": int(np.argmax(deg)),
         "uniform": 12345,
         "zero_in_degree": int(np.flatnonzero(deg == 0)[7]),
         "leaf": int(np.flatnonzero(deg == 1)[3])}[pick]
    gpu = gpu_query(srk, rp, col, s, 0.05, 17)
    ref = oracle_query(rp, col, s, 0.05, 17)
    assert_parity(gpu, ref)


def test_rmat20_eps002_sampled_targets_bit_exact(srk):
    # the benchmark's workload and launch configuration: R-MAT scale 20,
    # c=0.6, eps=0.02, sources from the uniform list; every output of the full
    # query is computed, the oracle re-computes a sample of targets one by one
    from srk_inputs import uniform_sources
    rp, col = rmat_graph(20)
    n = rp.size - 1
    deg = np.diff(rp)
    sources = uniform_sources(n, 64, seed=2)
    rng = np.random.default_rng(5)
    for s in (int(sources[0]), int(np.argmax(deg))):
        gpu = gpu_query(srk, rp, col, s, 0.02, 2024)
        targets = np.unique(np.concatenate([
            rng.choice(n, 1500, replace=False),
            np.argsort(-deg)[:50],                  # hubs
            [s, 0, n - 1]])).astype(np.int32)
        ref = oracle_query(rp, col, s, 0.02, 2024, targets=targets)
        assert_parity(gpu, ref, targets)
        scores = gpu[0]
        assert np.all(scores[deg == 0][scores[deg == 0] != 1.0] == 0.0)
        assert np.all((scores >= 0.0) & (scores <= 1.0))


def test_edge_cases(srk):
    rp, col = er_graph(200, 3.0, 4)
    deg = np.diff(rp)
    # L = 0: only length-0 walks, no step can meet
    gpu = gpu_query(srk, rp, col, 1, 0.5, 3, z_override=100.0, L_override=0)
    assert gpu[1].sum() == 0 and gpu[0][1] == 1.0 and np.count_nonzero(gpu[0]) == 1
    # source without in-neighbours
    s = int(np.flatnonzero(deg == 0)[0])
    gpu = gpu_query(srk, rp, col, s, 0.5, 3, z_override=300.0)
    ref = oracle_query(rp, col, s, 0.5, 3, z_override=300.0)
    assert_parity(gpu, ref)
    # a graph with no edges at all
    n = 40
    rp0 = np.zeros(n + 1, dtype=np.int32)
    col0 = np.zeros(0, dtype=np.int32)
    gpu = gpu_query(srk, rp0, col0, 5, 0.5, 3)
    assert gpu[1].sum() == 0 and gpu[0][5] == 1.0 and np.count_nonzero(gpu[0]) == 1
    # the largest truncation length, with a ragged pair count
    gpu = gpu_query(srk, rp, col, 2, 0.5, 8, z_override=777.7, L_override=srk.SRK_MAX_LEN)
    ref = oracle_query(rp, col, 2, 0.5, 8, z_override=777.7, L_override=srk.SRK_MAX_LEN)
    assert_parity(gpu, ref)
    # many walks per node (N_tot > 2^17) on a small graph
    gpu = gpu_query(srk, rp, col, 2, 0.5, 8, z_override=150000.5)
    ref = oracle_query(rp, col, 2, 0.5, 8, z_override=150000.5)
    assert_parity(gpu, ref)
    # the knobs of Appendix B.5
    gpu = gpu_query(srk, rp, col, 2, 0.3, 8, p=2.0, q=2.0)
    ref = oracle_query(rp, col, 2, 0.3, 8, p=2.0, q=2.0)
    assert_parity(gpu, ref)


def test_pairs_meeting_at_every_step(srk):
    # I(s) = I(u) = {x}, I(x) = {y}, I(y) = {x}: lockstep walks meet at step 1
    rp = np.array([0, 1, 2, 3, 4], dtype=np.int32)
    col = np.array([2, 2, 3, 2], dtype=np.int32)
    gpu = gpu_query(srk, rp, col, 0, 0.9, 5, z_override=500.0, L_override=9)
    ref = oracle_query(rp, col, 0, 0.9, 5, z_override=500.0, L_override=9)
    assert_parity(gpu, ref)
    assert gpu[1][1] > 0 and gpu[3][1] == gpu[1][1]   # each meeting after one step


def test_deterministic_and_seed_sensitive(srk):
    rp, col = rmat_graph(16)
    a = gpu_query(srk, rp, col, 100, 0.05, 1)
    b = gpu_query(srk, rp, col, 100, 0.05, 1)
    c = gpu_query(srk, rp, col, 100, 0.05, 2)
    for x, y in zip(a[:4], b[:4]):
        assert np.array_equal(x, y)
    assert not np.array_equal(a[2], c[2])


def test_multi_source_equals_single_queries(srk):
    import torch
    rp, col = rmat_graph(16)
    n = rp.size - 1
    sources = [0, 77, 4096, 65535]
    eps = [0.05, 0.1, 0.08, 0.2]
    dev = torch.device("cuda:0")
    g = srk.srk_graph_load(torch.from_numpy(rp).to(dev), torch.from_numpy(col).to(dev))
    try:
        multi = torch.empty((4, n), dtype=torch.float64, device=dev)
        mc = torch.empty((4, n), dtype=torch.int32, device=dev)
        stats = srk.SrkStats()
        srk.srk_multi_source(g, sources, C, eps, 11, multi, mc, stats=stats)
        one = torch.empty(n, dtype=torch.float64, device=dev)
        oc = torch.empty(n, dtype=torch.int32, device=dev)
        total = 0
        for i, s in enumerate(sources):
            st = srk.SrkStats()
            srk.srk_single_source(g, s, C, eps[i], 11, one, oc, stats=st)
            torch.cuda.synchronize()
            assert torch.equal(one, multi[i]) and torch.equal(oc, mc[i])
            total += st.target_steps
        assert stats.target_steps == total
    finally:
        g.close()


def test_invalid_arguments_are_rejected(srk):
    import torch
    rp, col = er_graph(100, 3.0, 2)
    dev = torch.device("cuda:0")
    g = srk.srk_graph_load(torch.from_numpy(rp).to(dev), torch.from_numpy(col).to(dev))
    out = torch.empty(100, dtype=torch.float64, device=dev)
    try:
        for args in [(-1, 0.6, 0.5), (100, 0.6, 0.5), (0, 0.0, 0.5), (0, 1.0, 0.5),
                     (0, 0.6, 0.03), (0, 0.6, 1.0)]:
            with pytest.raises(srk.SrkError) as e:
                srk.srk_single_source(g, args[0], args[1], args[2], 1, out)
            assert e.value.code == srk.SRK_EINVAL
        with pytest.raises(srk.SrkError):
            srk.srk_single_source(g, 0, 0.6, 0.5, 1, out, z_override=1e9)  # N_tot too large
        with pytest.raises(srk.SrkError):
            srk.srk_single_source(g, 0, 0.6, 0.5, 1, out, L_override=srk.SRK_MAX_LEN + 1)
        with pytest.raises(srk.SrkError):
            srk.srk_single_source(g, 0, 0.6, 0.5, 1, out, p=0.5)
        for bad in (float("nan"), -3.0, float("inf")):
            with pytest.raises(srk.SrkError) as e:
                srk.srk_single_source(g, 0, 0.6, 0.5, 1, out, z_override=bad)
            assert e.value.code == srk.SRK_EINVAL
        with pytest.raises(srk.SrkError):
            srk.srk_single_source(g, 0, 0.6, float("nan"), 1, out)
    finally:
        g.close()
    # malformed CSRs are refused at load time (checked by an in-bounds kernel)
    bad_col = col.copy()
    bad_col[5] = 100
    with pytest.raises(srk.SrkError) as e:
        srk.srk_graph_load(torch.from_numpy(rp).to(dev), torch.from_numpy(bad_col).to(dev))
    assert e.value.code == srk.SRK_EINVAL
    bad_rp = rp.copy()
    bad_rp[10], bad_rp[11] = bad_rp[11] + 1, bad_rp[10]
    with pytest.raises(srk.SrkError):
        srk.srk_graph_load(bad_rp, col)


def _multi(srk, rp, col, sources, eps, seed, device_out=True, no_graph=False, **kw):
    import torch
    dev = torch.device("cuda:0")
    n = rp.size - 1
    k = len(sources)
    g = srk.srk_graph_load(torch.from_numpy(rp).to(dev), torch.from_numpy(col).to(dev))
    try:
        stats = srk.SrkStats()
        if device_out:
            sc = torch.empty((k, n), dtype=torch.float64, device=dev)
            mc = torch.empty((k, n), dtype=torch.int32, device=dev)
            srk.srk_multi_source(g, sources, C, eps, seed, sc, mc, stats=stats,
                                 no_graph=no_graph, **kw)
            torch.cuda.synchronize()
            return sc.cpu().numpy(), mc.cpu().numpy().view(np.uint32), stats
        sc = np.empty((k, n), dtype=np.float64)
        mc = np.empty((k, n), dtype=np.uint32)
        srk.srk_multi_source(g, sources, C, eps, seed, sc, mc, stats=stats,
                             no_graph=no_graph, **kw)
        return sc, mc, stats
    finally:
        g.close()


def test_batched_sources_bit_exact_against_oracle(srk):
    # mixed budgets (eps), a zero-in-degree source, a hub and a leaf, in one batch
    rp, col = rmat_graph(16)
    deg = np.diff(rp)
    sources = [int(np.argmax(deg)), int(np.flatnonzero(deg == 0)[3]), 12345,
               int(np.flatnonzero(deg == 1)[5]), 0]
    eps = [0.05, 0.1, 0.08, 0.05, 0.2]
    sc, mc, stats = _multi(srk, rp, col, sources, eps, 23)
    total = 0
    for i, s in enumerate(sources):
        ref = oracle_query(rp, col, s, eps[i], 23)
        assert np.array_equal(mc[i], ref.count)
        assert np.array_equal(sc[i], ref.scores)
        total += int(ref.steps.sum())
    assert stats.target_steps == total


def test_batched_many_batches_graph_and_host_outputs(srk, monkeypatch):
    # a small scratch budget forces one source per batch; the CUDA-graph path,
    # the direct path and host outputs must all agree with single queries
    rp, col = er_graph(1000, 5.0, 1)
    sources = list(range(0, 40, 3))
    eps = [0.1 + 0.01 * (i % 5) for i in range(len(sources))]
    a = _multi(srk, rp, col, sources, eps, 5)
    monkeypatch.setenv("SRK_BATCH_BYTES", "1")
    b = _multi(srk, rp, col, sources, eps, 5, no_graph=True)
    c = _multi(srk, rp, col, sources, eps, 5, device_out=False)
    for x, y in ((a, b), (a, c)):
        assert np.array_equal(x[0], y[0]) and np.array_equal(x[1], y[1])
        assert x[2].target_steps == y[2].target_steps
    for i in (0, 7, len(sources) - 1):
        one = gpu_query(srk, rp, col, sources[i], eps[i], 5)
        assert np.array_equal(one[0], a[0][i]) and np.array_equal(one[1], a[1][i])


def test_target_ranges_compose_the_full_query(srk):
    # the owner rule: slices [b, e) computed separately (device and host
    # outputs) equal the full query and leave everything else untouched
    import torch
    rp, col = rmat_graph(16)
    n = rp.size - 1
    full = gpu_query(srk, rp, col, 4242, 0.05, 31)
    dev = torch.device("cuda:0")
    g = srk.srk_graph_load(torch.from_numpy(rp).to(dev), torch.from_numpy(col).to(dev))
    try:
        cuts = [0, n // 3, n // 3 + 1, 2 * n // 3, n]
        sc = torch.full((n,), -7.0, dtype=torch.float64, device=dev)
        cnt_h = np.full(n, 12345, dtype=np.uint32)
        total = 0
        for b, e in zip(cuts[:-1], cuts[1:]):
            st = srk.SrkStats()
            srk.srk_single_source(g, 4242, C, 0.05, 31, sc, cnt_h, stats=st, target_range=(b, e))
            total += st.target_steps
        torch.cuda.synchronize()
        assert np.array_equal(sc.cpu().numpy(), full[0])
        assert np.array_equal(cnt_h, full[1])
        assert total == full[4].target_steps
        part = np.full(n, 3, dtype=np.uint32)
        sc2 = np.full(n, -1.0)
        srk.srk_single_source(g, 4242, C, 0.05, 31, sc2, part, target_range=(100, 200))
        assert np.all(part[:100] == 3) and np.all(part[200:] == 3)
        assert np.array_equal(part[100:200], full[1][100:200])
        assert np.all(sc2[:100] == -1.0) and np.array_equal(sc2[100:200], full[0][100:200])
        with pytest.raises(srk.SrkError):
            srk.srk_single_source(g, 0, C, 0.05, 1, sc, target_range=(5, n + 1))
    finally:
        g.close()


def test_warmup_rule_bit_exact(srk):
    rp, col = er_graph(200, 3.0, 4)
    gpu = gpu_query(srk, rp, col, 3, 0.3, 12, warmup_rule=True)
    ref = oracle_query(rp, col, 3, 0.3, 12, warmup_rule=True)
    assert_parity(gpu, ref)
    assert gpu[4].L == ref.table.L > 0


@pytest.mark.parametrize("z,L", [(2000.0, 32), (1.0, 0), (37.0, 5)])
def test_literal_shuffle_bit_exact(srk, z, L):
    # every target's walks shuffled by its own keyed permutation (Section 5.2
    # read literally): N_tot = 2018 (an 11-bit network, unequal halves, cycle
    # walking), N_tot = 1 (the identity) and N_tot = 33 (6 bits)
    rp, col = er_graph(1000, 5.0, 1)
    for s, seed in ((0, 1), (17, 9)):
        gpu = gpu_query(srk, rp, col, s, 0.1, seed, z_override=z, L_override=L,
                        literal_shuffle=True)
        ref = oracle_query(rp, col, s, 0.1, seed, z_override=z, L_override=L,
                           literal_shuffle=True)
        assert_parity(gpu, ref)
    plain = gpu_query(srk, rp, col, 0, 0.1, 1, z_override=2000.0, L_override=32)
    lit = gpu_query(srk, rp, col, 0, 0.1, 1, z_override=2000.0, L_override=32,
                    literal_shuffle=True)
    assert not np.array_equal(plain[1], lit[1])


def test_literal_shuffle_rmat_sampled_targets_and_ranges(srk):
    rp, col = rmat_graph(14)
    n = rp.size - 1
    rng = np.random.default_rng(3)
    targets = np.sort(rng.choice(n, 300, replace=False)).astype(np.int64)
    gpu = gpu_query(srk, rp, col, 99, 0.1, 4, literal_shuffle=True, device_outputs=False)
    ref = oracle_query(rp, col, 99, 0.1, 4, targets=targets, literal_shuffle=True)
    assert_parity(gpu, ref, targets)
    import torch
    dev = torch.device("cuda:0")
    g = srk.srk_graph_load(torch.from_numpy(rp).to(dev), torch.from_numpy(col).to(dev))
    try:
        part = np.zeros(n, dtype=np.uint32)
        for b, e in ((0, n // 2), (n // 2, n)):
            srk.srk_single_source(g, 99, C, 0.1, 4, np.empty(n), part,
                                  target_range=(b, e), literal_shuffle=True)
        assert np.array_equal(part, gpu[1])
        with pytest.raises(srk.SrkError):
            srk.srk_multi_source(g, [1, 2], C, [0.1, 0.1], 4,
                                 torch.empty((2, n), dtype=torch.float64, device=dev),
                                 literal_shuffle=True)
    finally:
        g.close()


def test_walk_count_near_the_limit_sampled_targets(srk):
    # N_tot just below SRK_MAX_WALKS = 2^24: the Fisher-Yates resolution, the
    # pair list and the hit table at their largest, checked on sampled targets
    from oracle.params import sample_table
    rp, col = er_graph(1000, 5.0, 1)
    L = 16
    z = float(srk.SRK_MAX_WALKS)
    for _ in range(3):   # N_tot is z times the kept mass plus the round-ups
        z += srk.SRK_MAX_WALKS - 100 - sample_table(1000, C, 0.1, z_override=z, L_override=L).N_tot
    gpu = gpu_query(srk, rp, col, 3, 0.1, 21, z_override=z, L_override=L,
                    device_outputs=False)
    assert srk.SRK_MAX_WALKS - 400 < gpu[4].n_walks <= srk.SRK_MAX_WALKS
    targets = np.array([0, 1, 2, 500, 998, 999], dtype=np.int64)
    ref = oracle_query(rp, col, 3, 0.1, 21, targets=targets, z_override=z, L_override=L)
    assert_parity(gpu, ref, targets)


def test_gather_probe_cache_operators(srk):
    # the measurement utility: every cache operator issues the announced loads
    # and finishes; an unknown operator is refused before any launch
    import torch
    dev = torch.device("cuda:0")
    data = torch.arange(1 << 16, dtype=torch.int32, device=dev)
    sink = torch.zeros(1, dtype=torch.int64, device=dev)
    counts = []
    for op in (srk.SRK_PROBE_DEFAULT, srk.SRK_PROBE_CG, srk.SRK_PROBE_NC, srk.SRK_PROBE_CA):
        counts.append(srk.srk_probe_gather_ex(data, 8, 3, op, sink))
    torch.cuda.synchronize()
    assert len(set(counts)) == 1 and counts[0] > 0 and counts[0] % (256 * 8 * 4) == 0
    with pytest.raises(srk.SrkError) as e:
        srk.srk_probe_gather_ex(data, 8, 3, 7, sink)
    assert e.value.code == srk.SRK_EINVAL


def test_wide_adjacency_layout_bit_exact(srk):
    # the 8-byte-entry layout (forced here on small graphs) gives exactly the
    # results of the 4-byte one: single-source, literal shuffle and batched
    import torch
    dev = torch.device("cuda:0")
    cases = [(er_graph(1000, 5.0, 1), 0, 0.1, TINY), (rmat_graph(16), 4242, 0.05, {})]
    for (rp, col), s, eps, kw in cases:
        n = rp.size - 1
        outs = []
        for layout in ("narrow", "wide", "csr"):
            g = srk.srk_graph_load(torch.from_numpy(rp).to(dev), torch.from_numpy(col).to(dev),
                                   layout=layout)
            assert srk.srk_graph_layout(g) == layout
            try:
                sc = torch.empty(n, dtype=torch.float64, device=dev)
                cn = torch.empty(n, dtype=torch.int32, device=dev)
                stp = torch.empty(n, dtype=torch.int32, device=dev)
                st = srk.SrkStats()
                srk.srk_single_source(g, s, C, eps, 7, sc, cn, step_counts=stp, stats=st, **kw)
                lit = torch.empty(n, dtype=torch.int32, device=dev)
                srk.srk_single_source(g, s, C, eps, 7, torch.empty(n, dtype=torch.float64,
                                                                    device=dev), lit,
                                      literal_shuffle=True, **kw)
                multi = torch.empty((2, n), dtype=torch.float64, device=dev)
                srk.srk_multi_source(g, [s, 3], C, [eps, eps], 7, multi, **kw)
                torch.cuda.synchronize()
                outs.append((sc.cpu().numpy(), cn.cpu().numpy(), stp.cpu().numpy(),
                             lit.cpu().numpy(), multi.cpu().numpy(), st.source_steps,
                             st.target_steps))
            finally:
                g.close()
        for other in outs[1:]:
            for a, b in zip(outs[0], other):
                assert np.array_equal(a, b)
        assert outs[1][1].sum() > 0
    # small graphs default to 4-byte entries
    g = srk.srk_graph_load(*er_graph(1000, 5.0, 1))
    assert srk.srk_graph_layout(g) == "narrow"
    g.close()
    # and the wide layout against the oracle directly
    rp, col = er_graph(1000, 5.0, 1)
    g = srk.srk_graph_load(rp, col, layout="wide")
    try:
        n = rp.size - 1
        counts = np.empty(n, dtype=np.uint32)
        scores = np.empty(n)
        srk.srk_single_source(g, 17, C, 0.1, 2, scores, counts, **TINY)
    finally:
        g.close()
    ref = oracle_query(rp, col, 17, 0.1, 2, **TINY)
    assert np.array_equal(counts, ref.count) and np.array_equal(scores, ref.scores)


def test_hub_headers_bit_exact(srk):
    # With 4-byte entries the degree code holds degrees below 2^(32-b) - 1,
    # 2^b >= n + m + H (here b = 19: 8,191); the 40 hubs keep theirs in the
    # header region.  A hub source, a hub target and landings on hubs all go
    # through it; the other layouts and the batched path must agree.
    import torch
    rp, col = hub_graph()
    n, m = rp.size - 1, col.size
    deg = np.diff(rp)
    hubs = np.flatnonzero(deg >= 8191)
    assert hubs.size == 40 and deg[deg < 8191].max() < 100
    assert 2 ** 18 < n + m + 40 <= 2 ** 19
    plain = int(np.flatnonzero((deg > 0) & (deg < 8191))[7])
    for s, seed in ((int(hubs[3]), 3), (plain, 4)):
        gpu = gpu_query(srk, rp, col, s, 0.1, seed, **TINY)
        assert_parity(gpu, oracle_query(rp, col, s, 0.1, seed, **TINY))
        assert gpu[1][hubs].sum() > 0
    dev = torch.device("cuda:0")
    rows = {}
    for layout in ("narrow", "wide", "csr"):
        g = srk.srk_graph_load(torch.from_numpy(rp).to(dev), torch.from_numpy(col).to(dev),
                               layout=layout)
        try:
            out = torch.empty((2, n), dtype=torch.float64, device=dev)
            cnt = torch.empty((2, n), dtype=torch.int32, device=dev)
            srk.srk_multi_source(g, [int(hubs[3]), plain], C, [0.1, 0.1], 3, out, cnt, **TINY)
            one = torch.empty(n, dtype=torch.float64, device=dev)
            srk.srk_single_source(g, plain, C, 0.1, 3, one, **TINY)
            torch.cuda.synchronize()
            assert torch.equal(one, out[1])
            rows[layout] = (out.cpu().numpy(), cnt.cpu().numpy())
        finally:
            g.close()
    for layout in ("wide", "csr"):
        assert np.array_equal(rows[layout][0], rows["narrow"][0])
        assert np.array_equal(rows[layout][1], rows["narrow"][1])


def test_rejected_step_words_redraw_bit_exact(srk):
    # Two hubs whose in-lists hold all D = 3,144,261 leaves, each leaf with
    # both hubs as in-neighbours: every even step of a walk from a leaf draws
    # an index below D, and 2^32 mod D = 3,051,031, so 7.1e-4 of those words
    # are rejected and replaced by the 64-bit draw of the step's second
    # block (source and target walks, per-source and shared keys).
    import torch
    from oracle import sampler
    from srk_inputs import csr_from_edges
    D = 3144261
    leaves = np.arange(2, D + 2, dtype=np.int32)
    src = np.concatenate([leaves, leaves, np.zeros(D, np.int32), np.ones(D, np.int32)])
    dst = np.concatenate([np.zeros(D, np.int32), np.ones(D, np.int32), leaves, leaves])
    rp, col = csr_from_edges(D + 2, src, dst)
    n = rp.size - 1
    assert np.diff(rp)[0] == D and (1 << 32) % D == 3051031
    s, seed = 77, 31
    kw = dict(z_override=2000.0, L_override=16)
    rng = np.random.default_rng(4)
    targets = np.unique(np.concatenate([[0, 1, s], rng.choice(n, 120, replace=False)]))
    targets = targets.astype(np.int32)
    # words of step 2 (the first hub draw of a pair) that the rule rejects
    key = sampler.walk_key(seed, s)
    t_ = (1 << 32) % D
    rejected = sum(1 for u in targets[2:40] for j in range(2000)
                   if (sampler.philox2x32_10([j, int(u)], key)[1] * D) % (1 << 32) < t_)
    assert rejected >= 20
    dev = torch.device("cuda:0")
    for shared in (False, True):
        gpu = gpu_query(srk, rp, col, s, 0.1, seed, shared_walks=shared, **kw)
        ref = oracle_query(rp, col, s, 0.1, seed, targets=targets, shared_walks=shared, **kw)
        assert_parity(gpu, ref, targets)
        assert ref.count.sum() > 0
    g = srk.srk_graph_load(torch.from_numpy(rp).to(dev), torch.from_numpy(col).to(dev),
                           layout="wide")
    try:
        cnt = torch.empty(n, dtype=torch.int32, device=dev)
        srk.srk_single_source(g, s, C, 0.1, seed, torch.empty(n, dtype=torch.float64,
                                                               device=dev), cnt, **kw)
        torch.cuda.synchronize()
        ref = oracle_query(rp, col, s, 0.1, seed, targets=targets, **kw)
        assert np.array_equal(cnt.cpu().numpy().view(np.uint32)[targets], ref.count)
    finally:
        g.close()


def test_multi_source_long_walks_shared_memory(srk):
    # L = 250: in its 1024-thread launch shape the batched kernel's per-warp
    # rows take ~65 KB of shared memory, above the 48 KB a kernel gets without
    # opting in; the autotuner (first call on a fresh handle) tries every shape
    import torch
    rp, col = er_graph(1000, 5.0, 1)
    n = rp.size - 1
    dev = torch.device("cuda:0")
    g = srk.srk_graph_load(torch.from_numpy(rp).to(dev), torch.from_numpy(col).to(dev))
    try:
        kw = dict(z_override=500.0, L_override=250)
        src = [0, 17, 423]
        multi = torch.empty((3, n), dtype=torch.float64, device=dev)
        st = srk.SrkStats()
        srk.srk_multi_source(g, src, C, [0.1] * 3, 9, multi, stats=st, **kw)
        torch.cuda.synchronize()
        assert st.L == 250 and 0 <= st.batch_shape < 5
        for i, s in enumerate(src):
            one = torch.empty(n, dtype=torch.float64, device=dev)
            srk.srk_single_source(g, s, C, 0.1, 9, one, **kw)
            torch.cuda.synchronize()
            assert torch.equal(one, multi[i])
        assert float(multi.sum()) > 3.0  # some targets besides the sources score
    finally:
        g.close()


def test_degenerate_graphs_and_calls(srk):
    import torch
    dev = torch.device("cuda:0")
    # one node, no edges: s~(0, 0) = 1, single and batched
    g = srk.srk_graph_load(np.array([0, 0], dtype=np.int32), np.zeros(0, dtype=np.int32))
    try:
        sc = torch.full((1,), -1.0, dtype=torch.float64, device=dev)
        srk.srk_single_source(g, 0, C, 0.9, 1, sc, z_override=10.0)
        multi = torch.full((2, 1), -1.0, dtype=torch.float64, device=dev)
        srk.srk_multi_source(g, [0, 0], C, [0.9, 0.9], 1, multi, z_override=10.0)
        torch.cuda.synchronize()
        assert sc.item() == 1.0 and bool(torch.all(multi == 1.0))
        srk.srk_multi_source(g, [], C, [], 1, multi)       # no sources: nothing to do
    finally:
        g.close()
    # self-loops and repeated in-neighbours are valid CSR input: a walk may
    # stay on a node and a repeated neighbour is drawn twice as often
    lists = [[0, 1, 1], [0, 2], [2, 2, 3], [1], [], [0, 4, 4, 5], [5]]
    rp = np.zeros(len(lists) + 1, dtype=np.int32)
    rp[1:] = np.cumsum([len(x) for x in lists])
    col = np.array([y for x in lists for y in x], dtype=np.int32)
    for s in (0, 2, 5):
        gpu = gpu_query(srk, rp, col, s, 0.5, 3, z_override=400.0, L_override=12)
        ref = oracle_query(rp, col, s, 0.5, 3, z_override=400.0, L_override=12)
        assert_parity(gpu, ref)
        assert gpu[1].sum() > 0
    # an empty target range leaves the outputs untouched
    g = srk.srk_graph_load(rp, col)
    try:
        out = np.full(rp.size - 1, -5.0)
        srk.srk_single_source(g, 0, C, 0.5, 3, out, z_override=100.0, target_range=(3, 3))
        assert np.all(out == -5.0)
    finally:
        g.close()


def test_concurrent_queries_on_streams_equal_serial(srk):
    # the graph is read-only after load: queries of different sources on two
    # streams (and a linearised pass on a third) may overlap on the GPU and
    # still give the serial results bit for bit
    import torch
    from srk_inputs import lognormal_weights
    dev = torch.device("cuda:0")
    rp, col = rmat_graph(16)
    n = rp.size - 1
    g = srk.srk_graph_load(torch.from_numpy(rp).to(dev), torch.from_numpy(col).to(dev))
    try:
        sources = [11, 4242, 777, 60000, 5, 31337]
        serial = []
        for s in sources:
            out = torch.empty(n, dtype=torch.float64, device=dev)
            srk.srk_single_source(g, s, C, 0.05, 9, out)
            torch.cuda.synchronize()
            serial.append(out.clone())
        w = torch.from_numpy(lognormal_weights(col.size, seed=3)).to(dev)
        lin_ref = torch.empty(n, dtype=torch.float32, device=dev)
        srk.srk_linear_fwd(g, w, 3, C, 6, lin_ref, keep_context=False)
        torch.cuda.synchronize()
        streams = [torch.cuda.Stream() for _ in range(3)]
        outs = [torch.empty(n, dtype=torch.float64, device=dev) for _ in sources]
        lin = torch.empty(n, dtype=torch.float32, device=dev)
        for k, s in enumerate(sources):
            srk.srk_single_source(g, s, C, 0.05, 9, outs[k], stream=streams[k % 2])
            if k == 2:
                srk.srk_linear_fwd(g, w, 3, C, 6, lin, keep_context=False, stream=streams[2])
        torch.cuda.synchronize()
        for a, b in zip(serial, outs):
            assert torch.equal(a, b)
        assert torch.equal(lin, lin_ref)
    finally:
        g.close()


@pytest.mark.parametrize("opts", [dict(warmup_rule=True), dict(p=1.5, q=2.0),
                                  dict(z_override=900.0, L_override=7)])
def test_multi_source_options_equal_single_queries(srk, opts):
    # the batched path applies the same sample-count options per source
    import torch
    dev = torch.device("cuda:0")
    rp, col = er_graph(1000, 5.0, 1)
    n = rp.size - 1
    sources = [0, 17, 503, 999]
    eps = [0.3, 0.25, 0.35, 0.3]
    g = srk.srk_graph_load(torch.from_numpy(rp).to(dev), torch.from_numpy(col).to(dev))
    try:
        multi = torch.empty((len(sources), n), dtype=torch.float64, device=dev)
        mc = torch.empty((len(sources), n), dtype=torch.int32, device=dev)
        srk.srk_multi_source(g, sources, C, eps, 23, multi, mc, **opts)
        one = torch.empty(n, dtype=torch.float64, device=dev)
        oc = torch.empty(n, dtype=torch.int32, device=dev)
        for i, s in enumerate(sources):
            srk.srk_single_source(g, s, C, eps[i], 23, one, oc, **opts)
            torch.cuda.synchronize()
            assert torch.equal(one, multi[i]) and torch.equal(oc, mc[i])
        assert int(mc.sum()) > 0
    finally:
        g.close()


def test_batched_graph_executable_is_updated_not_rebuilt(srk):
    # the second call of the same shape launches the cached executable after
    # updating its parameters; a call of another shape rebuilds it; results
    # stay equal to single queries throughout
    import torch
    dev = torch.device("cuda:0")
    rp, col = rmat_graph(14)
    n = rp.size - 1
    deg = np.diff(rp)
    order = np.argsort(-deg, kind="stable")
    g = srk.srk_graph_load(torch.from_numpy(rp).to(dev), torch.from_numpy(col).to(dev))
    try:
        single = torch.empty(n, dtype=torch.float64, device=dev)
        for sources, expect_update in (([int(order[0]), int(order[50])], False),
                                       ([int(order[1]), int(order[60])], True),
                                       ([int(order[2])], False),
                                       ([int(order[3])], True)):
            out = torch.empty((len(sources), n), dtype=torch.float64, device=dev)
            st = srk.SrkStats()
            srk.srk_multi_source(g, sources, C, 0.1, 3, out, stats=st)
            torch.cuda.synchronize()
            assert (st.graph_updates >= 1) == expect_update
            for i, s in enumerate(sources):
                srk.srk_single_source(g, s, C, 0.1, 3, single)
                assert torch.equal(single, out[i])
    finally:
        g.close()
