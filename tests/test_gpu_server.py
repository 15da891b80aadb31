"""The query server (srk_server_*): admitted requests give the same scores as
srk_single_source; memory-based admission sheds what does not fit and keeps
the counters consistent."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def srk():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2304_04015_gb300 as m
    return m


@pytest.fixture(scope="module")
def graphs(srk):
    import torch
    from srk_inputs import er_in_csr, rmat_in_csr
    dev = torch.device("cuda:0")
    out = []
    for rp, col in (er_in_csr(1000, 5.0, seed=1), rmat_in_csr(12, seed=2)):
        out.append((srk.srk_graph_load(torch.from_numpy(rp).to(dev),
                                       torch.from_numpy(col).to(dev)), rp.size - 1))
    yield out
    for g, _ in out:
        g.close()


def test_served_scores_equal_single_queries(srk, graphs):
    import torch
    rng = np.random.default_rng(3)
    reqs = []
    with srk.srk_server_create([g for g, _ in graphs], mem_budget=4 << 30, n_workers=3) as srv:
        for k in range(30):
            gi = int(rng.integers(0, 2))
            n = graphs[gi][1]
            s = int(rng.integers(0, n))
            eps = float(rng.choice([0.1, 0.2, 0.3]))
            buf = np.full(n, -1.0)
            assert srk.srk_server_submit(srv, gi, s, 0.6, eps, 99 + k, buf)
            reqs.append((gi, s, eps, 99 + k, buf))
        srk.srk_server_drain(srv)
        st = srk.srk_server_stats(srv)
        assert st.submitted == 30 and st.admitted == 30 and st.shed == 0
        assert st.completed == 30 and st.failed == 0
        assert 0 < st.p50_ms <= st.p99_ms <= st.max_ms
    dev = torch.device("cuda:0")
    for gi, s, eps, seed, buf in reqs:
        g, n = graphs[gi]
        ref = torch.empty(n, dtype=torch.float64, device=dev)
        srk.srk_single_source(g, s, 0.6, eps, seed, ref)
        torch.cuda.synchronize()
        assert np.array_equal(ref.cpu().numpy(), buf)


def test_memory_admission_sheds_and_counts(srk, graphs):
    g, n = graphs[1]
    with srk.srk_server_create([g], mem_budget=2 << 20, n_workers=1) as srv:
        admitted = sum(srk.srk_server_submit(srv, 0, k % n, 0.6, 0.05, k) for k in range(60))
        srk.srk_server_drain(srv)
        st = srk.srk_server_stats(srv)
        assert st.submitted == 60 and st.admitted == admitted and st.shed == 60 - admitted
        assert 0 < admitted < 60
        assert st.completed == admitted and st.reserved_peak <= 2 << 20
        with pytest.raises(srk.SrkError):
            srk.srk_server_submit(srv, 5, 0, 0.6, 0.05, 1)
        with pytest.raises(srk.SrkError):
            srk.srk_server_submit(srv, 0, n, 0.6, 0.05, 1)


def test_latency_target_admission(srk, graphs):
    # a tiny latency target admits only requests estimated to finish in time;
    # sources without in-neighbours have no estimated work and always fit
    g, n = graphs[1]
    import numpy as np
    from srk_inputs import rmat_in_csr
    rp, _ = rmat_in_csr(12, seed=2)
    deg = np.diff(rp)
    zero = [int(v) for v in np.flatnonzero(deg == 0)[:10]]
    busy = [int(v) for v in np.argsort(-deg)[:40]]
    with srk.srk_server_create([g], mem_budget=8 << 30, n_workers=2,
                               latency_target_ms=1e-3) as srv:
        adm_busy = [srk.srk_server_submit(srv, 0, s, 0.6, 0.01, 7) for s in busy]
        adm_zero = [srk.srk_server_submit(srv, 0, s, 0.6, 0.01, 7) for s in zero]
        srk.srk_server_drain(srv)
        st = srk.srk_server_stats(srv)
    assert all(adm_zero)
    assert sum(adm_busy) < len(busy)
    assert st.completed == st.admitted == sum(adm_busy) + len(zero)
