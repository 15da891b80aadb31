"""Pins for the exact oracle: Eq. 1 (Jeh-Widom) and Lemma 2 (first meeting).

* closed forms that follow from Eq. 1 by hand on 2-6 node graphs;
* invariants: s(u,u) = 1, symmetry, 0 <= s <= c off the diagonal, s = 0 when a
  node has no in-neighbours;
* the fixed point against a direct linear solve of Eq. 1 (Kronecker system);
* the first-meeting recursion against brute-force enumeration of walk pairs;
* Lemma 2: the Jeh-Widom fixed point equals sum_k c^k F_k.
"""
import itertools

import numpy as np
import pytest

from oracle import exact
from srk_inputs import er_in_csr


def csr(lists):
    row_ptr = np.zeros(len(lists) + 1, dtype=np.int32)
    row_ptr[1:] = np.cumsum([len(x) for x in lists])
    col = np.array(list(itertools.chain(*[sorted(x) for x in lists])), dtype=np.int32)
    return row_ptr, col


C = 0.6


def sim(lists, c=C):
    rp, col = csr(lists)
    S, _ = exact.jeh_widom(rp, col, len(lists), c)
    return S


def test_shared_single_in_neighbour_gives_c():
    # I(a) = I(b) = {x}: s(a, b) = c * s(x, x) = c
    S = sim([[], [0], [0]])
    assert S[1, 2] == pytest.approx(C, abs=1e-13)


def test_two_levels_gives_c_squared():
    # I(a)={x}, I(b)={y}, I(x)=I(y)={r}: s(x,y)=c, s(a,b)=c*s(x,y)=c^2
    S = sim([[], [0], [0], [1], [2]])
    assert S[1, 2] == pytest.approx(C, abs=1e-13)
    assert S[3, 4] == pytest.approx(C * C, abs=1e-13)


@pytest.mark.parametrize("k", [1, 2, 3, 5])
def test_k_shared_sources_gives_c_over_k(k):
    # I(a) = I(b) = {x_1..x_k}, the x_i without in-neighbours (s(x_i,x_j)=0):
    # s(a,b) = c/k^2 * sum_i s(x_i, x_i) = c/k
    lists = [[] for _ in range(k)] + [list(range(k)), list(range(k))]
    S = sim(lists)
    assert S[k, k + 1] == pytest.approx(C / k, abs=1e-13)


def test_directed_cycle_is_zero_off_diagonal():
    n = 6
    S = sim([[(v - 1) % n] for v in range(n)])
    off = S - np.diag(np.diag(S))
    assert np.abs(off).max() < 1e-14


def test_no_in_neighbours_gives_zero():
    S = sim([[], [0], [0, 1], []])
    assert S[0, 1] == 0.0 and S[0, 2] == 0.0 and S[3, 1] == 0.0 and S[3, 2] == 0.0


def _random_lists(n, rng, p=0.4):
    return [[u for u in range(n) if u != v and rng.random() < p] for v in range(n)]


def test_invariants_on_tiny_er():
    rp, col = er_in_csr(200, 5.0, seed=1)
    S, _ = exact.jeh_widom(rp, col, 200, C)
    assert np.allclose(np.diag(S), 1.0)
    assert np.abs(S - S.T).max() < 1e-14
    off = S[~np.eye(200, dtype=bool)]
    assert off.min() >= 0.0 and off.max() <= C + 1e-15
    deg = np.diff(rp)
    zero = np.flatnonzero(deg == 0)
    for z in zero:
        row = S[z].copy()
        row[z] = 0.0
        assert np.all(row == 0.0)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_fixed_point_equals_direct_solve(seed):
    # Eq. 1 as one linear system in the n^2 unknowns: for u != v,
    # s(u,v) - c sum T[u,u'] T[v,v'] s(u',v') = 0, and s(u,u) = 1.
    rng = np.random.default_rng(seed)
    n = 6
    lists = _random_lists(n, rng)
    rp, col = csr(lists)
    T = exact.transition(rp, col, n).toarray()
    A = np.eye(n * n) - C * np.kron(T, T)
    b = np.zeros(n * n)
    for u in range(n):
        A[u * n + u, :] = 0.0
        A[u * n + u, u * n + u] = 1.0
        b[u * n + u] = 1.0
    direct = np.linalg.solve(A, b).reshape(n, n)
    S, _ = exact.jeh_widom(rp, col, n, C)
    assert np.abs(S - direct).max() < 1e-12


def _brute_first_meeting(lists, a, b, K):
    """F_k(a, b) by enumerating every pair of uniform in-neighbour paths."""
    F = np.zeros(K + 1)
    if a == b:
        F[0] = 1.0
        return F

    def rec(x, y, k, prob):
        if k == K:
            return
        if not lists[x] or not lists[y]:
            return
        px = 1.0 / len(lists[x])
        py = 1.0 / len(lists[y])
        for x2 in lists[x]:
            for y2 in lists[y]:
                p = prob * px * py
                if x2 == y2:
                    F[k + 1] += p
                else:
                    rec(x2, y2, k + 1, p)

    rec(a, b, 0, 1.0)
    return F


@pytest.mark.parametrize("seed", [3, 4])
def test_first_meeting_against_enumeration(seed):
    rng = np.random.default_rng(seed)
    n, K = 5, 6
    lists = _random_lists(n, rng, p=0.5)
    rp, col = csr(lists)
    F = exact.first_meeting(rp, col, n, K)
    for a in range(n):
        for b in range(n):
            brute = _brute_first_meeting(lists, a, b, K)
            assert np.abs(F[:, a, b] - brute).max() < 1e-14


def test_lemma2_jeh_widom_equals_meeting_probability():
    rp, col = er_in_csr(300, 5.0, seed=7)
    n = 300
    S, _ = exact.jeh_widom(rp, col, n, C)
    rows = [0, 5, 17]
    K = 80   # c^80 < 1e-17
    F = exact.first_meeting(rp, col, n, K, rows=rows)
    S2 = exact.simrank_from_first_meeting(F, C, diag_rows=rows)
    assert np.abs(S[rows] - S2).max() < 1e-12


def test_expectation_closed_form_matches_sum():
    from oracle.params import sample_table
    rp, col = er_in_csr(300, 5.0, seed=7)
    tab = sample_table(300, C, 0.2, z_override=500.0, L_override=12)
    F = exact.first_meeting(rp, col, 300, tab.L, rows=[0])[:, 0, :]
    e_loop = exact.estimator_expectation(F, tab, quantised=False)
    e_closed = exact.estimator_expectation_closed(F, tab)
    assert np.abs(e_loop - e_closed).max() < 1e-14
    e_q = exact.estimator_expectation(F, tab, quantised=True)
    # quantisation moves each weight by at most 2^-33
    assert np.abs(e_q - e_loop).max() < tab.N_tot * 2.0 ** -33 / tab.z + 1e-15
