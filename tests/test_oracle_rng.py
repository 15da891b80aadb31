"""Pins for the oracle's random-number layer (CPU only).

* Philox4x32-10 and Philox2x32-10 against the published known-answer vectors
  (golden files).
* The index draw floor(R d / 2^64) against exact big-integer arithmetic.
* The walk-step draw: Lemire's acceptance rule is exactly uniform (checked
  exhaustively on narrower words), the oracle applies it as stated (big
  integers, words at the threshold), and rejected words fall back to the
  64-bit draw of the step's second block.
* The walk key is injective in its key word.
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
GOLDEN2 = os.path.join(os.path.dirname(__file__), "golden", "philox2x32_10_kat.txt")


def _hex_rows(path):
    rows = []
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append([int(x, 16) for x in line.split()])
    return rows


def _kat_rows():
    return [(v[:4], v[4:6], v[6:10]) for v in _hex_rows(GOLDEN)]


def _kat2_rows():
    return [(v[:2], v[2], v[3:5]) for v in _hex_rows(GOLDEN2)]


@pytest.mark.parametrize("ctr,key,expect", _kat_rows())
def test_philox_known_answers(ctr, key, expect):
    assert sampler.philox4x32_10(ctr, key) == expect


@pytest.mark.parametrize("ctr,key,expect", _kat2_rows())
def test_philox2x32_known_answers(ctr, key, expect):
    assert sampler.philox2x32_10(ctr, key) == expect


def test_philox2x32_counter_and_key_sensitivity():
    base = sampler.philox2x32_10([1, 2], 3)
    for ctr, key in (([0, 2], 3), ([1, 3], 3), ([1, 2], 2)):
        out = sampler.philox2x32_10(ctr, key)
        assert all(a != b for a, b in zip(out, base))


def _lemire_rule(w, d, r, bits=32):
    m = w * d
    if m % (1 << bits) >= (1 << bits) % d:
        return m >> bits, True
    return (r * d) >> 64, False


@pytest.mark.parametrize("bits", [6, 8, 10])
def test_lemire_rule_is_exactly_uniform(bits):
    # every index below d keeps exactly floor(2^bits / d) accepted words
    W = np.arange(1 << bits, dtype=np.int64)
    for d in range(1, (1 << bits) + 1):
        m = W * d
        acc = (m % (1 << bits)) >= ((1 << bits) % d)
        counts = np.bincount(m[acc] >> bits, minlength=d)
        assert counts.size == d
        assert np.all(counts == (1 << bits) // d)
        assert int((~acc).sum()) == (1 << bits) % d


def test_bounded_draw_matches_the_rule():
    rng = np.random.default_rng(3)
    cases = [(0, 1, 5), ((1 << 32) - 1, 1, 5), (0, 3, 7 << 60), (0, 3 << 30, 1 << 63)]
    for _ in range(3000):
        d = int(rng.integers(1, 1 << 32)) if rng.random() < 0.5 else int(rng.integers(1, 1 << 12))
        cases.append((int(rng.integers(0, 1 << 32)), d, int(rng.integers(0, 1 << 63)) * 2 + 1))
    # words at the threshold, both sides: w d = t - 1 and t (mod 2^32), d odd
    for d in (3, 5, 7, 1000003, (1 << 31) + 1, 3 * (1 << 30) + 1, (1 << 32) - 1):
        t = (1 << 32) % d
        inv = pow(d, -1, 1 << 32)
        for target in (t - 1, t):
            if target >= 0:
                cases.append(((target * inv) % (1 << 32), d, 0xDEADBEEF12345678))
    rejected = 0
    for w, d, r in cases:
        want, ok = _lemire_rule(w, d, r)
        assert sampler.bounded(w, d, r) == want
        assert 0 <= want < d
        rejected += not ok
    assert rejected >= 10


def test_step_index_word_and_counter_layout():
    # d = 2^31 never rejects (2^32 mod d = 0): the index is the word >> 1
    key = sampler.walk_key(99, 4)
    for i, r, v in ((1, 0, 0), (2, 0, 0), (3, 7, 11), (4, 7, 11), (255, (1 << 24) - 1, (1 << 31) - 1)):
        blk = sampler.philox2x32_10([((i - 1) >> 1 << 24) | r, v], key)
        assert sampler.step_index(key, i, r, v, 1 << 31) == blk[(i - 1) & 1] >> 1


def test_step_index_redraw_uses_the_second_block():
    # d = 3 * 2^30 rejects a quarter of the words; find rejected steps and
    # check they take floor(R d / 2^64) from the block with the top bit set
    d = 3 << 30
    key = sampler.walk_key(5, 6)
    seen = 0
    for r in range(200):
        for i in (1, 2):
            c0 = ((i - 1) >> 1 << 24) | r
            w = sampler.philox2x32_10([c0, 9], key)[(i - 1) & 1]
            if (w * d) % (1 << 32) >= (1 << 32) % d:
                assert sampler.step_index(key, i, r, 9, d) == (w * d) >> 32
                continue
            alt = [c0 | (1 << 31), 9] if i == 1 else [c0, 9 | (1 << 31)]
            y = sampler.philox2x32_10(alt, key)
            R = (y[0] << 32) | y[1]
            assert sampler.step_index(key, i, r, 9, d) == (R * d) >> 64
            seen += 1
    assert seen > 40


def test_walk_key_is_injective_in_the_key_word():
    for seed in (0, 1, 0xFFFFFFFFFFFFFFFF):
        keys = {sampler.walk_key(seed, q) for q in range(20000)}
        keys.add(sampler.walk_key(seed, 0xFFFFFFFE))
        assert len(keys) == 20001
    assert sampler.walk_key(1, 5) != sampler.walk_key(2, 5)


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
    # replica, key word and seed each change the walks (walks on this graph
    # are short, so two keys can give one walk: compare 16 replicas at once)
    def many(r0, q, seed):
        return [sampler.walk(rp, col, 0, r0 + k, q, seed, 20).tolist() for k in range(16)]
    ref = many(5, 1, 77)
    assert ref != many(21, 1, 77) and ref != many(5, 2, 77) and ref != many(5, 1, 78)
