"""Pins of eq. err and eq. bal / eq. avebal, including Table 1's printed fractions."""
import numpy as np
import pytest

from conftest import golden
from oracle import metrics


def test_error_rate_permutation_invariant():
    truth = np.array([0, 0, 1, 1, 2, 2])
    assert metrics.error_rate(np.array([2, 2, 0, 0, 1, 1]), truth, 3) == 0.0
    # one row misplaced: ||H_hat J - H||_F^2 = 2, divided by n
    assert metrics.error_rate(np.array([2, 2, 0, 1, 1, 1]), truth, 3) == pytest.approx(2 / 6)
    assert metrics.misclustered_fraction(np.array([2, 2, 0, 1, 1, 1]), truth, 3) == pytest.approx(1 / 6)


def test_error_rate_brute_force():
    import itertools

    rng = np.random.default_rng(0)
    k = 4
    truth = rng.integers(0, k, 40)
    comp = rng.integers(0, k, 40)
    Ht = np.eye(k)[truth]
    Hc = np.eye(k)[comp]
    best = min(np.sum((Hc[:, list(p)] - Ht) ** 2) for p in itertools.permutations(range(k))) / 40
    assert metrics.error_rate(comp, truth, k) == pytest.approx(best)


def _counts_from_fractions(n, v1, f11, f12):
    """Integer (|C1|, |V1 cap C1|) reproducing Table 1's 4-digit fractions."""
    sols = []
    for c1 in range(1, n):
        for a in range(0, min(c1, v1) + 1):
            if round(a / c1, 4) == f11 and round((v1 - a) / (n - c1), 4) == f12:
                sols.append((c1, a))
    return sols


@pytest.mark.parametrize("method", ["SC", "FairSC", "sFairSC"])
def test_table1_fractions(method):
    gd = golden("table1_fractions.json")
    n, (v1, v2) = gd["n"], gd["group_sizes"]
    assert round(v1 / n, 4) == gd["whole_graph"][0] and round(v2 / n, 4) == gd["whole_graph"][1]
    t = gd[method]
    sols = _counts_from_fractions(n, v1, t["V1_C1"], t["V1_C2"])
    assert len(sols) >= 1
    c1, a = sols[0]
    groups = np.array([0] * v1 + [1] * v2)
    labels = np.array([0] * a + [1] * (v1 - a) + [0] * (c1 - a) + [1] * (v2 - (c1 - a)))
    M = metrics.group_cluster_counts(labels, groups, 2, 2)
    frac = M / M.sum(axis=1, keepdims=True)
    assert round(frac[0, 0], 4) == t["V1_C1"] and round(frac[1, 0], 4) == t["V1_C2"]
    assert round(frac[0, 1], 4) == t["V2_C1"] and round(frac[1, 1], 4) == t["V2_C2"]


def test_balance_upper_bound_reached_by_fair_clustering():
    """eq. bal-upper: min balance <= min |V_s|/|V_s'|, with equality for a group-fair clustering."""
    groups = np.array([0] * 40 + [1] * 60)
    labels = np.concatenate([np.repeat([0, 1], 20), np.repeat([0, 1], 30)])
    b = metrics.balance(labels, groups, 2, 2)
    np.testing.assert_allclose(b, 40 / 60)
    assert metrics.average_balance(labels, groups, 2, 2) == pytest.approx(40 / 60)
    rng = np.random.default_rng(0)
    for _ in range(20):
        lab = rng.integers(0, 3, 100)
        assert metrics.balance(lab, groups, 3, 2).min() <= 40 / 60 + 1e-12


def test_balance_multiset_by_hand():
    """The sorted rows of the cluster x group count matrix: worked out by hand, unchanged by a
    relabelling of the clusters, changed by moving one vertex, and giving eq. bal's balances."""
    labels = np.array([0, 0, 1, 1, 1, 2])
    groups = np.array([0, 1, 0, 0, 1, 1])
    ms = metrics.balance_multiset(labels, groups, 3, 2)
    assert ms == [(0, 1), (1, 1), (2, 1)]  # cluster 2: (0, 1); cluster 0: (1, 1); cluster 1: (2, 1)
    perm = np.array([2, 0, 1])
    assert metrics.balance_multiset(perm[labels], groups, 3, 2) == ms
    moved = labels.copy()
    moved[2] = 2  # a group-0 vertex from cluster 1 to cluster 2
    assert metrics.balance_multiset(moved, groups, 3, 2) == [(1, 1), (1, 1), (1, 1)]
    bal = sorted(min(r) / max(r) if min(r) > 0 else 0.0 for r in ms)
    np.testing.assert_allclose(sorted(metrics.balance(labels, groups, 3, 2)), bal)
