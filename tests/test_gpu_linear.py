"""GPU parity of the linearised form (srk_linear_fwd / srk_linear_bwd).

Forward against the FP64 oracle, backward against the oracle's reverse-mode
gradient on every edge and against FP64 central finite differences on 256
sampled edges (edge-weighted R-MAT scale 18, lognormal(0, 0.5) weights, L=10,
c=0.6, D=(1-c)I, loss = sum_v w_v s(s, v), w ~ N(0, 1)).

Tolerances (FP32 arithmetic, FP64 references): forward
|d| <= 1e-5 |ref| + 1e-7 max|ref|; gradient |d| <= 1e-4 |ref| + 1e-4 rms(ref)
per edge, and normwise ||d|| <= 1e-4 ||ref|| over all checked edges (the
relative error of 1e-4 the differentiable form is held to).  The R-MAT 18
test also prints the realised normwise error and the worst per-edge relative
error over the edges whose gradient is at least 1e-2 rms(ref).
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
def weighted(kind, size, seed):
    from srk_inputs import er_in_csr, rmat_in_csr, lognormal_weights
    rp, col = er_in_csr(size, 4.0, seed=seed) if kind == "er" else rmat_in_csr(size, seed=seed)
    return rp, col, lognormal_weights(col.size, seed=seed + 10)


def run_gpu(srk, rp, col, w, s, L, g):
    import torch
    dev = torch.device("cuda:0")
    n = rp.size - 1
    graph = srk.srk_graph_load(torch.from_numpy(rp).to(dev), torch.from_numpy(col).to(dev))
    try:
        wt = torch.from_numpy(w).to(dev).requires_grad_(True)
        out = srk.linear_simrank(graph, wt, s, C, L)
        loss = (torch.from_numpy(g.astype(np.float32)).to(dev) * out).sum()
        loss.backward()
        torch.cuda.synchronize()
        return out.detach().cpu().numpy().astype(np.float64), wt.grad.cpu().numpy().astype(np.float64)
    finally:
        graph.close()


def check_forward(got, ref):
    tol = 1e-5 * np.abs(ref) + 1e-7 * np.abs(ref).max()
    assert np.all(np.abs(got - ref) <= tol)


def check_grad(got, ref):
    """Per-edge mixed bound and normwise relative bound; returns (normwise
    relative error, worst relative error over edges with |ref| >= 1e-2 rms)."""
    rms = np.sqrt(np.mean(ref ** 2))
    tol = 1e-4 * np.abs(ref) + 1e-4 * rms
    d = got - ref
    assert np.all(np.abs(d) <= tol), float(np.max(np.abs(d) / tol))
    normwise = float(np.linalg.norm(d) / np.linalg.norm(ref))
    assert normwise <= 1e-4, normwise
    big = np.abs(ref) >= 1e-2 * rms
    worst = float(np.max(np.abs(d[big]) / np.abs(ref[big]))) if big.any() else 0.0
    return normwise, worst


def test_small_graph_against_reverse_mode_oracle(srk):
    from oracle import linear
    rp, col, w = weighted("er", 500, 3)
    g = np.random.default_rng(4).normal(size=500)
    # L = 200: the gradient's transpose tile (66 L floats) needs more than
    # 48 KB of shared memory
    for s, L in ((0, 10), (17, 3), (5, 1), (3, 200)):
        out, gr = run_gpu(srk, rp, col, w, s, L, g)
        ref_g, ref_s = linear.grad(rp, col, w.astype(np.float64), 500, s, C, L, g)
        check_forward(out, ref_s)
        check_grad(gr, ref_g)


def test_rmat18_configuration_gradients(srk):
    from oracle import linear
    rp, col, w = weighted("rmat", 18, 1)
    n = rp.size - 1
    deg = np.diff(rp)
    s = int(np.argsort(-deg)[10])
    g = np.random.default_rng(6).normal(size=n)
    out, gr = run_gpu(srk, rp, col, w, s, 10, g)
    w64 = w.astype(np.float64)
    ref_g, ref_s = linear.grad(rp, col, w64, n, s, C, 10, g)
    check_forward(out, ref_s)
    nw, worst = check_grad(gr, ref_g)
    # FP64 central finite differences on 256 sampled edges
    rng = np.random.default_rng(7)
    edges = rng.choice(col.size, 256, replace=False)
    fd = linear.finite_difference_pool(rp, col, w64, n, s, C, 10, g, edges)
    nw_fd, worst_fd = check_grad(gr[edges], fd)
    print("linear gradient, R-MAT 18, L = 10: reverse-mode oracle on all %d edges: normwise "
          "relative error %.3g, worst per-edge relative error (|ref| >= 1e-2 rms) %.3g; "
          "finite differences on 256 edges: normwise %.3g, worst %.3g"
          % (col.size, nw, worst, nw_fd, worst_fd))
    # scaling invariance of each in-list (P is unchanged): exact for the
    # oracle, and for the FP32 gradient within the per-edge tolerance above
    a_of_e = np.repeat(np.arange(n), deg)
    row_dot = np.bincount(a_of_e, weights=w64 * gr, minlength=n)
    rms = np.sqrt(np.mean(ref_g ** 2))
    row_tol = np.bincount(a_of_e, weights=w64 * (1e-4 * np.abs(ref_g) + 1e-4 * rms), minlength=n)
    assert np.all(np.abs(row_dot) <= row_tol + 1e-30)


def test_linear_invalid_weights_and_source(srk):
    import torch
    rp, col, w = weighted("er", 100, 2)
    dev = torch.device("cuda:0")
    graph = srk.srk_graph_load(torch.from_numpy(rp).to(dev), torch.from_numpy(col).to(dev))
    try:
        out = torch.empty(100, dtype=torch.float32, device=dev)
        bad = torch.from_numpy(w).to(dev)
        bad[3] = -1.0
        with pytest.raises(srk.SrkError) as e:
            srk.srk_linear_fwd(graph, bad, 0, C, 10, out)
        assert e.value.code == srk.SRK_EINVAL
        with pytest.raises(srk.SrkError):
            srk.srk_linear_fwd(graph, torch.from_numpy(w).to(dev), 100, C, 10, out)
        with pytest.raises(srk.SrkError):   # no weights given and none loaded
            srk.srk_linear_fwd(graph, None, 0, C, 10, out)
        ctx = srk.srk_linear_fwd(graph, torch.from_numpy(w).to(dev), 0, C, 0, out)
        gw = torch.empty(col.size, dtype=torch.float32, device=dev)
        srk.srk_linear_bwd(ctx, torch.ones(100, device=dev), gw)
        torch.cuda.synchronize()
        assert float(gw.abs().max()) == 0.0 and float(out[0]) == pytest.approx(1 - C)
        ctx.free()
    finally:
        graph.close()


def test_linear_graph_without_edges(srk):
    # P has no entries: s_vec = D e_s = (1 - c) e_s, and there is no weight
    # to differentiate (the edge arrays are empty; no weights are needed)
    import torch
    dev = torch.device("cuda:0")
    n = 70
    rp = torch.zeros(n + 1, dtype=torch.int32, device=dev)
    col = torch.zeros(0, dtype=torch.int32, device=dev)
    graph = srk.srk_graph_load(rp, col)
    try:
        for s, L in ((5, 3), (69, 0)):
            out = torch.full((n,), -1.0, dtype=torch.float32, device=dev)
            ctx = srk.srk_linear_fwd(graph, None, s, C, L, out)
            gw = torch.empty(0, dtype=torch.float32, device=dev)
            srk.srk_linear_bwd(ctx, torch.ones(n, device=dev), gw)
            torch.cuda.synchronize()
            ref = np.zeros(n, dtype=np.float32)
            ref[s] = np.float32(1.0 - C)
            assert np.array_equal(out.cpu().numpy(), ref)
            ctx.free()
    finally:
        graph.close()


def hub_graph(n=12000, seed=5):
    """ER in-lists plus a node whose in-list holds every other node (a list of
    six 2048-entry chunks), a node with 300 in-neighbours (a warp-sized list)
    and a node that is an in-neighbour of 5000 others (a long out-list of the
    transpose); in-lists sorted, no duplicates."""
    from srk_inputs import csr_from_edges, er_in_csr
    rp, col = er_in_csr(n, 4.0, seed=seed)
    dst = np.repeat(np.arange(n), np.diff(rp))
    src = col.astype(np.int64)
    hub_in = np.arange(1, n)
    fan = np.arange(2, 5002)
    mid = np.arange(100, 400)
    dst = np.concatenate([dst, np.zeros(hub_in.size, np.int64), fan, np.full(mid.size, 2)])
    src = np.concatenate([src, hub_in, np.ones(fan.size, np.int64), mid])
    return csr_from_edges(n, src, dst)


def test_hub_lists_every_size_class_and_bitwise_determinism(srk):
    from oracle import linear
    from srk_inputs import lognormal_weights
    rp, col = hub_graph()
    n = rp.size - 1
    deg = np.diff(rp)
    outdeg = np.bincount(col, minlength=n)
    assert deg.max() > 6 * 2048 - 2048 and outdeg.max() >= 5000
    assert np.any((deg > 32) & (deg <= 512)) and np.any(deg <= 32)
    w = lognormal_weights(col.size, seed=9)
    g = np.random.default_rng(8).normal(size=n)
    for s in (0, 1, 7):
        a = run_gpu(srk, rp, col, w, s, 8, g)
        b = run_gpu(srk, rp, col, w, s, 8, g)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
        ref_g, ref_s = linear.grad(rp, col, w.astype(np.float64), n, s, C, 8, g)
        check_forward(a[0], ref_s)
        check_grad(a[1], ref_g)
