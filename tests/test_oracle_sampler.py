"""Pins for the oracle's Monte Carlo sampler (steps a2-a5).

* Lemma 3 / Algorithm 2: the literal tuple-sort-PREDECESSOR path gives the same
  counts and weight sums as the direct step-by-step comparison.
* A graph where every pair that takes a step meets at every step: the count is
  the number of pairs with both lengths >= 1, each counted once (Section 5.5).
* Theorem 6 on the small configuration: every |s~ - s| <= eps.
* Unbiasedness: the mean over many seeds equals the exact expectation of the
  estimator (first-meeting recursion) within a CLT band.
* Step totals against a plain re-walk of each pair.
* Shared target walks (keyed by node and replica alone, as Algorithm 1 draws
  every node's walks once): the literal Algorithm 2 path, the mean over seeds
  against the exact expectation, and walks that no longer depend on s.
"""
import numpy as np
import pytest

from oracle import alg2, exact, sampler
from oracle.params import sample_table
from srk_inputs import er_in_csr

C = 0.6


@pytest.mark.parametrize("n,deg,s,seed", [(60, 3.0, 0, 11), (60, 3.0, 7, 12),
                                           (40, 1.5, 3, 13), (80, 2.0, 0, 14)])
def test_literal_algorithm2_equals_direct_compare(n, deg, s, seed):
    rp, col = er_in_csr(n, deg, seed=seed)
    r = sampler.run(rp, col, n, s, C, 0.5, seed, z_override=300.0)
    cnt, ws = alg2.run(rp, col, n, s, C, 0.5, seed, z_override=300.0)
    assert np.array_equal(r.count, cnt)
    assert np.array_equal(r.wsum, ws)
    assert r.count[s] == 0


def test_pairs_meeting_at_every_step_count_once():
    # I(s) = I(u) = {x}, I(x) = {y}, I(y) = {x}: both walks visit x, y, x, ...
    # in lockstep, so every pair with min(l1, l2) >= 1 meets (at every step)
    s, u, x, y = 0, 1, 2, 3
    lists = [[x], [x], [y], [x]]
    rp = np.array([0, 1, 2, 3, 4], dtype=np.int32)
    col = np.array([l[0] for l in lists], dtype=np.int32)
    seed = 5
    r = sampler.run(rp, col, 4, s, C, 0.9, seed, z_override=500.0, L_override=9)
    tab = r.table
    sigma = sampler.fisher_yates(s, seed, tab.N_tot)
    expect_cnt, expect_w, expect_steps = 0, 0, 0
    for j in range(tab.N_tot):
        l2, l1 = tab.stratum(j), tab.stratum(int(sigma[j]))
        if min(l1, l2) >= 1:
            expect_cnt += 1
            expect_w += tab.wq(l1, l2)
            expect_steps += 1        # meets at step 1
    assert r.count[u] == expect_cnt
    assert r.wsum[u] == expect_w
    assert r.steps[u] == expect_steps


def test_source_without_in_neighbours():
    rp, col = er_in_csr(100, 3.0, seed=2)
    deg = np.diff(rp)
    s = int(np.flatnonzero(deg == 0)[0])
    r = sampler.run(rp, col, 100, s, C, 0.5, 1, z_override=200.0)
    assert r.count.sum() == 0 and r.wsum.sum() == 0 and r.steps.sum() == 0
    assert r.scores[s] == 1.0 and np.count_nonzero(r.scores) == 1


def test_theorem6_small_configuration():
    # ER n=1000, Poisson(5) in-degrees, c=0.6, source 0, eps=0.1, z=2000, L=32
    n = 1000
    rp, col = er_in_csr(n, 5.0, seed=1)
    S, _ = exact.jeh_widom(rp, col, n, C)
    for seed in (1, 2, 3):
        r = sampler.run(rp, col, n, 0, C, 0.1, seed, z_override=2000.0, L_override=32)
        err = np.abs(r.scores - S[0])
        assert err.max() <= 0.1
        assert r.scores[0] == 1.0


def test_mean_over_seeds_matches_exact_expectation():
    n, s = 120, 0
    rp, col = er_in_csr(n, 2.0, seed=21)
    tab = sample_table(n, C, 0.5, z_override=300.0, L_override=15)
    F = exact.first_meeting(rp, col, n, tab.L, rows=[s])[:, 0, :]
    expect = exact.estimator_expectation(F, tab, quantised=True)
    seeds = 400
    acc = np.zeros((seeds, n))
    for k in range(seeds):
        r = sampler.run(rp, col, n, s, C, 0.5, 1000 + k, z_override=300.0, L_override=15)
        acc[k] = r.scores
    acc[:, s] = 0.0
    expect[s] = 0.0
    mean = acc.mean(axis=0)
    sd = acc.std(axis=0, ddof=1)
    live = sd > 0
    zscore = np.abs(mean[live] - expect[live]) / (sd[live] / np.sqrt(seeds))
    assert live.sum() > 10
    assert zscore.max() < 5.0
    # where no pair can ever meet, the estimate is exactly zero
    assert np.all(mean[expect == 0.0] == 0.0)


@pytest.mark.parametrize("n,deg,s,seed", [(60, 3.0, 0, 11), (50, 2.0, 9, 4)])
def test_shared_walks_algorithm2_equals_direct(n, deg, s, seed):
    rp, col = er_in_csr(n, deg, seed=seed)
    r = sampler.run(rp, col, n, s, C, 0.5, seed, z_override=300.0, shared_walks=True)
    cnt, ws = alg2.run(rp, col, n, s, C, 0.5, seed, z_override=300.0, shared_walks=True)
    assert np.array_equal(r.count, cnt) and np.array_equal(r.wsum, ws)
    plain = sampler.run(rp, col, n, s, C, 0.5, seed, z_override=300.0)
    assert not np.array_equal(plain.count, r.count)     # the keying changed the walks


def test_shared_walks_do_not_depend_on_the_source():
    rp, col = er_in_csr(60, 3.0, seed=3)
    for v, r in ((5, 0), (17, 33), (42, 7)):
        a = sampler.walk(rp, col, v, r, sampler.SHARED_KEY, 9, 20)
        assert a.size > 0
        for s in (0, 1, 59):   # a source walk from v is keyed by s instead
            assert not np.array_equal(a, sampler.walk(rp, col, v, r, s, 9, 20)) or v == s


def test_shared_walks_mean_matches_exact_expectation():
    # shared target walks leave each (s, u) estimate's law unchanged
    n, s = 120, 0
    rp, col = er_in_csr(n, 2.0, seed=21)
    tab = sample_table(n, C, 0.5, z_override=300.0, L_override=15)
    F = exact.first_meeting(rp, col, n, tab.L, rows=[s])[:, 0, :]
    expect = exact.estimator_expectation(F, tab, quantised=True)
    seeds = 300
    acc = np.zeros((seeds, n))
    for k in range(seeds):
        acc[k] = sampler.run(rp, col, n, s, C, 0.5, 7000 + k, z_override=300.0,
                             L_override=15, shared_walks=True).scores
    acc[:, s] = 0.0
    expect[s] = 0.0
    mean, sd = acc.mean(axis=0), acc.std(axis=0, ddof=1)
    live = sd > 0
    z = np.abs(mean[live] - expect[live]) / (sd[live] / np.sqrt(seeds))
    assert live.sum() > 10 and z.max() < 5.0


def test_step_totals_against_plain_rewalk():
    n, s, seed = 50, 4, 31
    rp, col = er_in_csr(n, 2.5, seed=9)
    r = sampler.run(rp, col, n, s, C, 0.5, seed, z_override=150.0)
    tab = r.table
    sigma = sampler.fisher_yates(s, seed, tab.N_tot)
    spos, seff = sampler.walks(rp, col, s, s, seed, tab)
    assert r.source_steps == int(seff.sum())
    for u in (0, 1, 2, 10):
        if u == s:
            continue
        steps = 0
        for j in range(tab.N_tot):
            w = int(sigma[j])
            cap = min(tab.stratum(j), int(seff[w]))
            tw = sampler.walk(rp, col, u, j, s, seed, tab.stratum(j))
            taken = 0
            for i in range(1, cap + 1):
                if i > tw.size:
                    break
                taken = i
                if tw[i - 1] == spos[w, i - 1]:
                    break
            steps += taken
        assert r.steps[u] == steps


def test_literal_shuffle_permutation_and_marginal():
    for N in (1, 2, 3, 7, 64, 65, 1000, 2018):
        perm = [sampler.feistel(11, 2, 5, N, j) for j in range(N)]
        assert sorted(perm) == list(range(N))
    # pi_u(j) for a fixed j is uniform over targets u (chi-square, 9 dof)
    N, trials = 10, 5000
    counts = np.bincount([sampler.feistel(u, 3, 77, N, 4) for u in range(trials)], minlength=N)
    exp = trials / N
    assert float(((counts - exp) ** 2 / exp).sum()) < 35.0


def test_literal_shuffle_pairing_law_per_target_and_across_targets():
    """Section 5.2 shuffles every node's walks independently, so target u's
    walk t is paired with a uniformly random source walk, independently of
    the other targets.  In the literal mode pair j joins source walk sigma(j)
    (sigma: the source's uniform Fisher-Yates shuffle) and target walk
    pi_u(j), so target walk t meets source walk sigma(pi_u^-1(t)).  Per target
    that composition is a uniform bijection whatever pi_u is: over seeds, its
    law on the 4! pairings of N = 4 walks passes a chi-square test (23 dof,
    critical value 49.7 at p = 1e-3).  pi_u itself, a keyed 4-round Feistel
    network, is only a pseudo-random bijection: on N = 4 its law over seeds
    is far from uniform (chi-square well above the critical value), so the
    independence across targets that Section 5.2 has is approximated, not
    reproduced; Theorem 6 needs only the per-target law."""
    import itertools
    N, K = 4, 4800
    perms = list(itertools.permutations(range(N)))
    composed = dict.fromkeys(perms, 0)
    feistel = dict.fromkeys(perms, 0)
    for seed in range(K):
        sigma = sampler.fisher_yates(7, seed, N)
        pi = [sampler.feistel(11, 7, seed, N, j) for j in range(N)]
        inv = [0] * N
        for j, t in enumerate(pi):
            inv[t] = j
        composed[tuple(int(sigma[inv[t]]) for t in range(N))] += 1
        feistel[tuple(pi)] += 1
    exp = K / len(perms)
    chi_composed = sum((c - exp) ** 2 / exp for c in composed.values())
    chi_feistel = sum((c - exp) ** 2 / exp for c in feistel.values())
    assert chi_composed < 49.7
    assert chi_feistel > 49.7


@pytest.mark.parametrize("n,deg,s,seed", [(60, 3.0, 0, 11), (50, 2.0, 9, 4)])
def test_literal_shuffle_algorithm2_equals_direct(n, deg, s, seed):
    rp, col = er_in_csr(n, deg, seed=seed)
    r = sampler.run(rp, col, n, s, C, 0.5, seed, z_override=200.0, literal_shuffle=True)
    cnt, ws = alg2.run(rp, col, n, s, C, 0.5, seed, z_override=200.0, literal_shuffle=True)
    assert np.array_equal(r.count, cnt) and np.array_equal(r.wsum, ws)
    plain = sampler.run(rp, col, n, s, C, 0.5, seed, z_override=200.0)
    assert not np.array_equal(plain.count, r.count)


def test_literal_shuffle_mean_matches_exact_expectation():
    # shuffling the targets' walks too leaves each target's law unchanged
    n, s = 120, 0
    rp, col = er_in_csr(n, 2.0, seed=21)
    tab = sample_table(n, C, 0.5, z_override=300.0, L_override=15)
    F = exact.first_meeting(rp, col, n, tab.L, rows=[s])[:, 0, :]
    expect = exact.estimator_expectation(F, tab, quantised=True)
    seeds = 300
    acc = np.zeros((seeds, n))
    for k in range(seeds):
        acc[k] = sampler.run(rp, col, n, s, C, 0.5, 5000 + k, z_override=300.0,
                             L_override=15, literal_shuffle=True).scores
    acc[:, s] = 0.0
    expect[s] = 0.0
    mean, sd = acc.mean(axis=0), acc.std(axis=0, ddof=1)
    live = sd > 0
    z = np.abs(mean[live] - expect[live]) / (sd[live] / np.sqrt(seeds))
    assert live.sum() > 10 and z.max() < 5.0
