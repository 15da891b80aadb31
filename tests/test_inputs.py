"""The seeded graph generators produce well-formed in-neighbour CSRs with the
stated degree laws (CPU only)."""
import numpy as np

from srk_inputs import er_in_csr, rmat_in_csr, uniform_sources, mixed_sources


def check_csr(rp, col, n):
    assert rp.dtype == np.int32 and col.dtype == np.int32
    assert rp.size == n + 1 and rp[0] == 0 and rp[-1] == col.size
    assert np.all(np.diff(rp) >= 0)
    assert col.size == 0 or (col.min() >= 0 and col.max() < n)
    for v in range(n):
        lst = col[rp[v]:rp[v + 1]]
        assert np.all(np.diff(lst) > 0)          # sorted, no duplicates
        assert not np.any(lst == v)              # no self-loop


def test_er_degree_law():
    rp, col = er_in_csr(2000, 5.0, seed=1)
    check_csr(rp, col, 2000)
    deg = np.diff(rp)
    assert abs(deg.mean() - 5.0) < 0.2
    assert abs(deg.var() - 5.0) < 0.6             # Poisson: variance = mean
    again = er_in_csr(2000, 5.0, seed=1)
    assert np.array_equal(again[0], rp) and np.array_equal(again[1], col)


def test_rmat_structure():
    rp, col = rmat_in_csr(12, seed=3)
    n = 1 << 12
    check_csr(rp, col, n)
    deg = np.diff(rp)
    # node 0 collects the a+c column mass at every level: the largest in-degree
    assert deg[0] == deg.max()
    assert col.size <= 16 * n and col.size > 0.8 * 16 * n
    # in-degree skew: many zero in-degree nodes
    assert (deg == 0).mean() > 0.2


def test_sources():
    s = uniform_sources(1000, 64, seed=2)
    assert s.size == 64 and np.unique(s).size == 64 and s.min() >= 0 and s.max() < 1000
    rp, _ = rmat_in_csr(10, seed=1)
    m = mixed_sources(rp, 12, seed=3)
    deg = np.diff(rp)
    assert m.size == 12 and np.all(deg[m[8:]] == 0)


def test_rmat_torch_generator_structure():
    import torch
    from srk_inputs import rmat_in_csr_torch, mixed_eps
    rp, col = rmat_in_csr_torch(11, seed=2, device="cpu")
    rp, col = rp.numpy(), col.numpy()
    check_csr(rp, col, 1 << 11)
    deg = np.diff(rp)
    assert deg[0] == deg.max() and (deg == 0).mean() > 0.2
    e = mixed_eps(300, seed=3)
    assert set(np.unique(e)) == {0.01, 0.02, 0.05}
