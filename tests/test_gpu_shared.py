"""GPU parity of shared target walks (SRK_OPT_SHARED_WALKS).

With the flag, walk j of target u is keyed by (u, j) alone, as Algorithm 1
draws every node's walks once.  srk_single_source with the flag must equal the
oracle's shared mode bit for bit (counts, weight sums, step counts, scores);
srk_multi_source with the flag walks each target once for all sources of a
batch and must equal the single-source queries bit for bit (scores, counts),
with or without graph capture, over several batches of up to 64 sources, with
host or device outputs; at R-MAT 16 it is also checked against the oracle on
sampled targets.
"""
import numpy as np
import pytest

from test_gpu_parity import (C, TINY, assert_parity, er_graph, gpu_query, oracle_query,
                             rmat_graph)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def srk():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2304_04015_gb300 as m
    return m


@pytest.mark.parametrize("seed", [1, 2])
def test_shared_single_source_bit_exact(srk, seed):
    rp, col = er_graph(1000, 5.0, 1)
    gpu = gpu_query(srk, rp, col, 0, 0.1, seed, shared_walks=True, **TINY)
    ref = oracle_query(rp, col, 0, 0.1, seed, shared_walks=True, **TINY)
    assert_parity(gpu, ref)
    assert ref.count.sum() > 0
    plain = oracle_query(rp, col, 0, 0.1, seed, **TINY)
    assert not np.array_equal(plain.count, ref.count)   # the keying differs


def _single_rows(srk, g, n, sources, eps, seed, dev, **kw):
    import torch
    rows, cnts = [], []
    for s, e in zip(sources, eps):
        out = torch.empty(n, dtype=torch.float64, device=dev)
        cnt = torch.empty(n, dtype=torch.int32, device=dev)
        srk.srk_single_source(g, int(s), C, float(e), seed, out, cnt, shared_walks=True, **kw)
        rows.append(out.cpu().numpy())
        cnts.append(cnt.cpu().numpy())
    return np.stack(rows), np.stack(cnts)


def test_shared_batch_equals_single_queries(srk):
    import torch
    dev = torch.device("cuda:0")
    rp, col = rmat_graph(16)
    n = rp.size - 1
    deg = np.diff(rp)
    order = np.argsort(-deg, kind="stable")
    sources = [int(order[0]), int(order[100]), int(np.flatnonzero(deg == 0)[0]),
               int(np.flatnonzero(deg == 1)[0]), int(order[5000]), int(order[3])]
    eps = [0.05, 0.1, 0.05, 0.08, 0.1, 0.06]
    g = srk.srk_graph_load(torch.from_numpy(rp).to(dev), torch.from_numpy(col).to(dev))
    try:
        ref_s, ref_c = _single_rows(srk, g, n, sources, eps, 9, dev)
        for no_graph in (False, True):
            out = torch.empty((len(sources), n), dtype=torch.float64, device=dev)
            cnt = torch.empty((len(sources), n), dtype=torch.int32, device=dev)
            st = srk.SrkStats()
            srk.srk_multi_source(g, sources, C, eps, 9, out, cnt, shared_walks=True,
                                 no_graph=no_graph, stats=st)
            torch.cuda.synchronize()
            assert np.array_equal(out.cpu().numpy(), ref_s)
            assert np.array_equal(cnt.cpu().numpy(), ref_c)
            assert st.target_steps > 0
        # the zero in-degree source: e_s; the others met somewhere
        assert ref_s[2, sources[2]] == 1.0 and np.count_nonzero(ref_s[2]) == 1
        assert ref_c[0].sum() > 0
        # host outputs
        out_h = np.empty((len(sources), n))
        cnt_h = np.empty((len(sources), n), dtype=np.uint32)
        srk.srk_multi_source(g, sources, C, eps, 9, out_h, cnt_h, shared_walks=True)
        assert np.array_equal(out_h, ref_s)
        assert np.array_equal(cnt_h.view(np.int32), ref_c)
    finally:
        g.close()


def test_shared_batches_of_64_and_the_rest(srk, monkeypatch):
    # 70 sources: a batch of 64 (masks and tables span both 32-bit words) and
    # one of 6; a small scratch budget splits them further; sources repeat
    # and are targets of one another
    import torch
    dev = torch.device("cuda:0")
    rp, col = er_graph(300, 4.0, 3)
    n = rp.size - 1
    rng = np.random.default_rng(2)
    sources = [int(x) for x in rng.integers(0, n, size=70)]
    sources[5] = sources[4]
    sources[50] = sources[4]
    eps = [float(x) for x in rng.choice([0.2, 0.3, 0.5], size=70)]
    g = srk.srk_graph_load(torch.from_numpy(rp).to(dev), torch.from_numpy(col).to(dev))
    try:
        ref_s, ref_c = _single_rows(srk, g, n, sources, eps, 4, dev, z_override=400.0)
        for budget in (None, "2000000"):
            if budget:
                monkeypatch.setenv("SRK_BATCH_BYTES", budget)
            out = torch.empty((70, n), dtype=torch.float64, device=dev)
            cnt = torch.empty((70, n), dtype=torch.int32, device=dev)
            srk.srk_multi_source(g, sources, C, eps, 4, out, cnt, shared_walks=True,
                                 z_override=400.0)
            torch.cuda.synchronize()
            assert np.array_equal(out.cpu().numpy(), ref_s)
            assert np.array_equal(cnt.cpu().numpy(), ref_c)
    finally:
        g.close()


def test_shared_batch_rmat16_against_oracle_sampled(srk):
    import torch
    from srk_inputs import mixed_eps, mixed_sources
    dev = torch.device("cuda:0")
    rp, col = rmat_graph(16)
    n = rp.size - 1
    all_src = mixed_sources(rp, 96, seed=3)
    sources = [int(all_src[i]) for i in (0, 1, 32, 33, 64)]
    eps = [float(x) for x in mixed_eps(5, seed=3)]
    g = srk.srk_graph_load(torch.from_numpy(rp).to(dev), torch.from_numpy(col).to(dev))
    try:
        out = torch.empty((5, n), dtype=torch.float64, device=dev)
        cnt = torch.empty((5, n), dtype=torch.int32, device=dev)
        srk.srk_multi_source(g, sources, C, eps, 21, out, cnt, shared_walks=True)
        torch.cuda.synchronize()
        rng = np.random.default_rng(8)
        hubs = np.argsort(-np.diff(rp))[:16]
        met = 0
        for i, (s, e) in enumerate(zip(sources, eps)):
            tg = np.unique(np.concatenate([rng.choice(n, 48, replace=False), hubs]))
            ref = oracle_query(rp, col, s, e, 21, targets=tg.astype(np.int32),
                               shared_walks=True)
            assert np.array_equal(cnt[i, tg].cpu().numpy().view(np.uint32), ref.count)
            assert np.array_equal(out[i, tg].cpu().numpy(), ref.scores)
            met += int(ref.count.sum())
        assert met > 0
    finally:
        g.close()
