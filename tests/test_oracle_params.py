"""Pins for the oracle's sample-count table (Algorithm 1 lines 3-5,
Algorithm 2 line 2, Lemma 7, Appendix B.4-B.5)."""
import math

import numpy as np
import pytest

from oracle.params import sample_table


@pytest.mark.parametrize("n,eps", [(1000, 0.1), (1 << 16, 0.05), (1 << 20, 0.02),
                                   (1 << 24, 0.01), (10, 0.5)])
def test_hoeffding_identity_fixes_z(n, eps):
    # Appendix B.4: z = ln(2n) / (2 lambda^2) makes 2 exp(-2 z lambda^2) = 1/n
    tab = sample_table(n, 0.6, eps)
    lam = eps - 3.0 / n
    assert 2.0 * math.exp(-2.0 * tab.z * lam * lam) == pytest.approx(1.0 / n, rel=1e-12)


@pytest.mark.parametrize("n", [5, 1000, 1 << 16, 1 << 20, 1 << 23, 1 << 24])
def test_truncation_keeps_all_but_one_over_n(n):
    # Eq. (small percent): sum_{l<=L} sqrt(c)^l (1 - sqrt(c)) > 1 - 1/n,
    # and L is the largest integer not above log_{1/sqrt c} n
    c = 0.6
    tab = sample_table(n, c, 0.9)
    rc = math.sqrt(c)
    mass = sum(rc ** l * (1 - rc) for l in range(tab.L + 1))
    assert mass > 1.0 - 1.0 / n
    assert rc ** tab.L >= 1.0 / n * (1 - 1e-12)       # L <= log n
    assert rc ** (tab.L + 1) < 1.0 / n                 # L + 1 > log n


def test_counts_round_up_and_weights():
    tab = sample_table(1 << 20, 0.6, 0.02)
    for l in range(tab.L + 1):
        Z = tab.Z[l]
        assert tab.N[l] - 1 < Z <= tab.N[l]           # N_l = ceil(Z_l)
        assert 0.0 < tab.a[l] <= 1.0                   # Lemma 7 weight
        assert tab.a[l] * tab.N[l] == pytest.approx(Z, rel=1e-15)
    assert tab.P[0] == 0 and tab.P[-1] == sum(tab.N)
    assert all(tab.P[l + 1] - tab.P[l] == tab.N[l] for l in range(tab.L + 1))
    # the N_l follow the geometric law: their ratio tends to sqrt(c)
    assert tab.N[5] / tab.N[4] == pytest.approx(math.sqrt(0.6), rel=1e-3)


def test_stratum_lookup():
    tab = sample_table(1000, 0.6, 0.1, z_override=2000.0, L_override=32)
    for l in range(tab.L + 1):
        assert tab.stratum(tab.P[l]) == l
        assert tab.stratum(tab.P[l + 1] - 1) == l


def test_small_configuration_by_hand():
    # z fixed at 2000 walk pairs and L at 32 steps: the counts are
    # ceil(2000 * 0.7745967^l * 0.2254033)
    tab = sample_table(1000, 0.6, 0.1, z_override=2000.0, L_override=32)
    assert tab.L == 32
    assert tab.N[0] == math.ceil(2000 * (1 - math.sqrt(0.6)))
    assert tab.N[0] == 451 and tab.N[1] == 350 and tab.N[32] == 1
    assert tab.N_tot == 2018


def test_quantised_weight():
    tab = sample_table(1 << 20, 0.6, 0.02)
    for l1 in (0, 1, 7, tab.L):
        for l2 in (0, 3, tab.L):
            w = tab.wq(l1, l2)
            assert abs(w - tab.a[l1] * tab.a[l2] * 2.0 ** 32) <= 0.5
            assert 0 < w <= 2 ** 32


def test_threshold_and_failure_knobs():
    # Appendix B.5: z = ln(2 n^q) / (2 (eps - 3/n^p)^2), L = floor(p log n)
    n = 1 << 20
    t1 = sample_table(n, 0.6, 0.02)
    t2 = sample_table(n, 0.6, 0.02, p=2.0, q=2.0)
    lam2 = 0.02 - 3.0 / n ** 2
    assert 2.0 * math.exp(-2.0 * t2.z * lam2 * lam2) == pytest.approx(1.0 / n ** 2, rel=1e-10)
    assert t2.L == math.floor(2.0 * math.log(n) / -math.log(math.sqrt(0.6)))
    assert t2.L >= 2 * t1.L
    assert t2.N_tot > t1.N_tot


@pytest.mark.parametrize("n,eps", [(1000, 0.003), (1000, 0.002), (1000, 1.0), (3, 0.9)])
def test_rejects_eps_at_or_below_threshold(n, eps):
    with pytest.raises(ValueError):
        sample_table(n, 0.6, eps)


def test_rejects_bad_c():
    for c in (0.0, 1.0, -0.1, 1.5):
        with pytest.raises(ValueError):
            sample_table(1000, c, 0.1)


def test_warmup_rule_sample_size_and_truncation():
    # Section 3: N = ln(2 n^2) / (2 eps^2) gives 2 exp(-2 N eps^2) = 1/n^2, and a
    # walk reaches length 3 log_{1/sqrt c}(n/eps) with probability (eps/n)^3
    n, eps, c = 1000, 0.1, 0.6
    tab = sample_table(n, c, eps, warmup_rule=True)
    assert 2.0 * math.exp(-2.0 * tab.z * eps * eps) == pytest.approx(1.0 / n ** 2, rel=1e-12)
    rc = math.sqrt(c)
    assert rc ** tab.L >= (eps / n) ** 3 * (1 - 1e-12)
    assert rc ** (tab.L + 1) < (eps / n) ** 3
    with pytest.raises(ValueError):
        sample_table(n, c, 1.2, warmup_rule=True)
