"""Pins for the oracle's random-number layer (CPU only).

* Philox4x32-10 against the published known-answer vectors (golden file).
* The index draw floor(R d / 2^64) against exact big-integer arithmetic.
* Fisher-Yates: a permutation, and uniform over all N! orders on tiny N.
* Walks: every step follows an in-edge, a walk stops at a node without
  in-neighbours, and the in-neighbour choice is uniform.
"""
import itertools
import math
import os

import numpy as np
import pytest

from oracle import sampler

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat_rows():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            vals = [int(x, 16) for x in line.split()]
            rows.append((vals[:4], vals[4:6], vals[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,expect", _kat_rows())
def test_philox_known_answers(ctr, key, expect):
    assert sampler.philox4x32_10(ctr, key) == expect


def test_philox_counter_sensitivity():
    # changing any counter word or key word changes every output word
    base = sampler.philox4x32_10([1, 2, 3, 4], [5, 6])
    for w in range(4):
        ctr = [1, 2, 3, 4]
        ctr[w] ^= 1
        out = sampler.philox4x32_10(ctr, [5, 6])
        assert all(a != b for a, b in zip(out, base))
    out = sampler.philox4x32_10([1, 2, 3, 4], [5, 7])
    assert all(a != b for a, b in zip(out, base))


def test_index_matches_big_integer():
    rng = np.random.default_rng(0)
    cases = [(0, 1), (0, 7), ((1 << 64) - 1, 1), ((1 << 64) - 1, 5),
             ((1 << 64) - 1, (1 << 32) - 1), (1 << 63, 2), (1 << 63, 3)]
    for _ in range(2000):
        r = int(rng.integers(0, 1 << 63)) * 2 + int(rng.integers(0, 2))
        d = int(rng.integers(1, 1 << 32))
        cases.append((r, d))
    for r, d in cases:
        got = sampler.index(r, d)
        assert got == (r * d) >> 64
        assert 0 <= got < d


def test_fisher_yates_is_permutation():
    for N in (1, 2, 17, 2018):
        sig = sampler.fisher_yates(3, 12345, N)
        assert sorted(sig.tolist()) == list(range(N))


def test_fisher_yates_uniform_on_four_items():
    N, trials = 4, 24 * 400
    counts = {}
    for seed in range(trials):
        key = tuple(sampler.fisher_yates(0, seed, N).tolist())
        counts[key] = counts.get(key, 0) + 1
    assert len(counts) == math.factorial(N)
    exp = trials / math.factorial(N)
    chi2 = sum((c - exp) ** 2 / exp for c in counts.values())
    # 23 degrees of freedom: P[chi2 > 60] < 1e-4
    assert chi2 < 60.0


def test_fisher_yates_depends_on_source_and_seed():
    a = sampler.fisher_yates(1, 7, 100)
    b = sampler.fisher_yates(2, 7, 100)
    c = sampler.fisher_yates(1, 8, 100)
    assert not np.array_equal(a, b) and not np.array_equal(a, c)


def _small_graph():
    # in-neighbour lists: I(0)={1,2,3}, I(1)={0}, I(2)={0,1}, I(3)={}, I(4)={3}
    lists = [[1, 2, 3], [0], [0, 1], [], [3]]
    row_ptr = np.zeros(len(lists) + 1, dtype=np.int32)
    row_ptr[1:] = np.cumsum([len(x) for x in lists])
    col = np.array(list(itertools.chain(*lists)), dtype=np.int32)
    return lists, row_ptr, col


def test_walk_follows_in_edges_and_stops_at_dead_end():
    lists, rp, col = _small_graph()
    for r in range(300):
        for v in range(5):
            w = sampler.walk(rp, col, v, r, 0, 99, 12)
            prev = v
            for x in w:
                assert x in lists[prev]
                prev = x
            if len(w) < 12:
                assert len(lists[prev]) == 0     # stopped only at a dead end
    # node 3 has no in-neighbours: no step at all
    assert sampler.walk(rp, col, 3, 0, 0, 1, 5).size == 0
    # node 4 moves to 3 and stops there
    assert sampler.walk(rp, col, 4, 0, 0, 1, 5).tolist() == [3]


def test_walk_neighbour_choice_is_uniform():
    lists, rp, col = _small_graph()
    counts = np.zeros(5)
    trials = 9000
    for r in range(trials):
        counts[sampler.walk(rp, col, 0, r, 4, 2024, 1)[0]] += 1
    obs = counts[[1, 2, 3]]
    exp = trials / 3
    chi2 = float(((obs - exp) ** 2 / exp).sum())
    assert chi2 < 20.0     # 2 dof: P[chi2 > 20] < 5e-5


def test_walk_is_reproducible_and_keyed():
    _, rp, col = _small_graph()
    a = sampler.walk(rp, col, 0, 5, 1, 77, 20)
    assert np.array_equal(a, sampler.walk(rp, col, 0, 5, 1, 77, 20))
    # a shorter walk with the same key is a prefix of the longer one
    b = sampler.walk(rp, col, 0, 5, 1, 77, 7)
    assert np.array_equal(a[:b.size], b)
    diff = [not np.array_equal(a, sampler.walk(rp, col, 0, 6, 1, 77, 20)),
            not np.array_equal(a, sampler.walk(rp, col, 0, 5, 2, 77, 20)),
            not np.array_equal(a, sampler.walk(rp, col, 0, 5, 1, 78, 20))]
    assert all(diff)
