"""Pins for the FP64 linearised-SimRank oracle (Appendix A form, D = (1-c)I).

* sparse term-by-term forward == dense matrix powers;
* a one-edge graph in closed form: s(a, a) = (1 - c)(1 + c);
* reverse-mode gradient == central finite differences;
* scaling all in-weights of a node leaves P unchanged, so the gradient is
  orthogonal to the weights of every in-list: sum_{e in I(a)} w_e dL/dw_e = 0;
* uniform weights give the unweighted column-normalised matrix.
"""
import numpy as np
import pytest

from oracle import linear
from srk_inputs import er_in_csr, lognormal_weights

C = 0.6


def small_graph(n=40, seed=3):
    rp, col = er_in_csr(n, 3.0, seed=seed)
    w = lognormal_weights(col.size, seed=seed).astype(np.float64)
    return rp, col, w


def test_sparse_forward_equals_dense_powers():
    rp, col, w = small_graph()
    for s in (0, 7):
        a = linear.forward(rp, col, w, 40, s, C, 6)
        b = linear.forward_dense(rp, col, w, 40, s, C, 6)
        assert np.abs(a - b).max() < 1e-14


def test_horner_form_equals_the_literal_sum():
    rp, col, w = small_graph(60, seed=11)
    for L in (0, 1, 4, 10):
        a = linear.forward(rp, col, w, 60, 3, C, L)
        b = linear.forward_horner(rp, col, w, 60, 3, C, L)
        assert np.abs(a - b).max() < 1e-15


def test_finite_difference_pool_matches_serial():
    rp, col, w = small_graph(30, seed=5)
    g = np.random.default_rng(1).normal(size=30)
    edges = [0, 3, 7]
    a = linear.finite_difference(rp, col, w, 30, 2, C, 5, g, edges)
    b = linear.finite_difference_pool(rp, col, w, 30, 2, C, 5, g, edges, processes=2)
    assert np.abs(a - b).max() < 1e-9


def test_one_edge_closed_form():
    # I(a) = {u}, a = 1, u = 0: s_vec = (1-c) e_a + c (1-c) P^T e_u = (1 - c^2) e_a
    rp = np.array([0, 0, 1], dtype=np.int32)
    col = np.array([0], dtype=np.int32)
    for L in (1, 2, 5):
        out = linear.forward(rp, col, np.array([2.5]), 2, 1, C, L)
        assert out[1] == pytest.approx(1 - C * C, abs=1e-15)
        assert out[0] == 0.0
    out = linear.forward(rp, col, np.array([2.5]), 2, 1, C, 0)
    assert out[1] == pytest.approx(1 - C, abs=1e-15)


def test_reverse_mode_matches_finite_differences():
    rp, col, w = small_graph(30, seed=5)
    g = np.random.default_rng(1).normal(size=30)
    gr, out = linear.grad(rp, col, w, 30, 2, C, 5, g)
    assert np.abs(out - linear.forward(rp, col, w, 30, 2, C, 5)).max() < 1e-14
    edges = list(range(col.size))
    fd = linear.finite_difference(rp, col, w, 30, 2, C, 5, g, edges)
    assert np.abs(fd - gr).max() <= 1e-8 * max(1.0, np.abs(gr).max())


def test_gradient_orthogonal_to_in_list_weights():
    rp, col, w = small_graph(50, seed=7)
    g = np.random.default_rng(2).normal(size=50)
    gr, _ = linear.grad(rp, col, w, 50, 4, C, 8, g)
    for a in range(50):
        lo, hi = rp[a], rp[a + 1]
        if hi > lo:
            assert abs(np.dot(w[lo:hi], gr[lo:hi])) < 1e-12


def test_uniform_weights_are_the_unweighted_matrix():
    rp, col, _ = small_graph(25, seed=9)
    P1 = linear.column_normalised(rp, col, np.ones(col.size), 25).toarray()
    P2 = linear.column_normalised(rp, col, np.full(col.size, 7.0), 25).toarray()
    assert np.abs(P1 - P2).max() < 1e-15
    deg = np.diff(rp)
    for a in range(25):
        if deg[a]:
            assert P1[:, a].sum() == pytest.approx(1.0, abs=1e-14)
            assert set(np.flatnonzero(P1[:, a])) == set(col[rp[a]:rp[a + 1]])
