"""Pins of the oracle's seeded k-means: the published RNG, the sampling law, Lloyd's fixed point."""
import math

import numpy as np
import pytest

from conftest import golden
from oracle import kmeans as km


def test_splitmix64_published_vectors():
    gd = golden("splitmix64.json")
    want = [int(x) for x in gd["outputs"]]
    assert km.splitmix64_sequence(gd["seed"], 5) == want
    assert [km.splitmix64_draw(gd["seed"], q) for q in range(5)] == want


def test_quantised_total_is_exact_sum_within_grid():
    rng = np.random.default_rng(0)
    v = rng.random(10_000).astype(np.float32) ** 3
    tot = km.quantised_total(v)
    exact = math.fsum(float(x) for x in v)
    s = km._scale_shift(float(v.max()), v.size)
    assert 0 <= exact - tot <= v.size * 2.0 ** (-s)
    # order independence
    assert km.quantised_total(v[::-1].copy()) == tot


def test_kmeanspp_first_center_and_law():
    """Center 0 is uniform; center 1 follows D^2 weights (Arthur and Vassilvitskii)."""
    X = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 3.0], [4.0, 4.0]], dtype=np.float32)
    n = 4
    counts = np.zeros((n, n))
    trials = 4000
    for seed in range(trials):
        idx = km.kmeanspp(X, 2, seed)
        assert idx[0] == (km.splitmix64_draw(seed, 0) * n) >> 64
        counts[idx[0], idx[1]] += 1
    for a in range(n):
        d2 = ((X - X[a]) ** 2).sum(axis=1).astype(np.float64)
        p = d2 / d2.sum()
        tot = counts[a].sum()
        assert tot > trials / n * 0.8
        for b in range(n):
            sd = math.sqrt(tot * p[b] * (1 - p[b])) + 1
            assert abs(counts[a, b] - tot * p[b]) < 5 * sd


def test_kmeanspp_never_repeats_a_center():
    rng = np.random.default_rng(1)
    X = rng.standard_normal((50, 3)).astype(np.float32)
    for seed in range(20):
        idx = km.kmeanspp(X, 10, seed)
        assert len(set(idx.tolist())) == 10


def blobs(n_per, k, d, sep, seed):
    rng = np.random.default_rng(seed)
    C = rng.standard_normal((k, d)) * sep
    X = np.concatenate([C[c] + rng.standard_normal((n_per, d)) for c in range(k)])
    return X, np.repeat(np.arange(k), n_per)


def test_lloyd_matches_sklearn_from_same_init():
    sk = pytest.importorskip("sklearn.cluster")
    X, _ = blobs(60, 4, 5, 3.0, 2)
    X32 = X.astype(np.float32)
    seeds = km.kmeanspp(X32, 4, seed=5)
    labels, mu, _ = km.lloyd(X32, X32[seeds].astype(np.float64), 300)
    ref = sk.KMeans(n_clusters=4, init=X32[seeds].astype(np.float64), n_init=1, algorithm="lloyd", tol=0.0,
                    max_iter=300).fit(X32.astype(np.float64))
    assert np.array_equal(labels, ref.labels_)
    np.testing.assert_allclose(mu, ref.cluster_centers_, rtol=1e-6, atol=1e-6)
    # the inertia: the same sum of squared distances as scikit-learn's, and as an FP64 sum over the
    # FP32 points (the oracle's exact fixed-point total of FP32 distances is within FP32 rounding)
    val = km.inertia(X32, labels, mu)
    X64 = X32.astype(np.float64)
    direct = float(((X64 - mu[labels]) ** 2).sum())
    assert val == pytest.approx(direct, rel=1e-5)
    assert val == pytest.approx(ref.inertia_, rel=1e-5)


def test_lloyd_fixed_point():
    """At convergence every centroid is its rows' mean and every row sits at its nearest centroid."""
    X, _ = blobs(80, 5, 4, 2.0, 3)
    labels, mu, H = None, None, X
    labels, mu, inert = km.kmeans(X, 5, seed=2, n_init=2)
    X32 = X.astype(np.float32).astype(np.float64)
    for c in range(5):
        np.testing.assert_allclose(mu[c], X32[labels == c].mean(axis=0), rtol=1e-9, atol=1e-9)
    d = ((X32[:, None, :] - mu[None, :, :]) ** 2).sum(-1)
    best = d.min(axis=1)
    mine = d[np.arange(len(X32)), labels]
    assert np.all(mine <= best * (1 + 1e-5) + 1e-9)


def test_recovers_separated_blobs():
    from oracle.metrics import error_rate

    X, truth = blobs(50, 6, 6, 8.0, 4)
    labels, _, _ = km.kmeans(X, 6, seed=0, n_init=5)
    assert error_rate(labels, truth, 6) == 0.0


def test_empty_cluster_takes_farthest_row():
    X32 = np.array([[0.0], [0.1], [0.2], [10.0]], dtype=np.float32)
    M32 = np.array([[0.1], [10.0], [50.0]], dtype=np.float32)
    labels, dist = km.assign(X32, M32)
    assert labels.tolist() == [0, 0, 0, 1]
    xs = km._scale_shift(10.0, 4)
    mu = km.update(X32, labels, 3, M32, dist, xs)
    # cluster 2 is empty: it takes row 0 or 2 (distance 0.01 to centroid 0.1); the lowest index wins
    assert mu[2, 0] == pytest.approx(0.0)
    assert mu[0, 0] == pytest.approx(0.1, rel=1e-6)


def test_assign_ties_go_to_lowest_index():
    X32 = np.array([[0.0, 0.0]], dtype=np.float32)
    M32 = np.array([[1.0, 0.0], [0.0, 1.0], [-1.0, 0.0]], dtype=np.float32)
    labels, _ = km.assign(X32, M32)
    assert labels[0] == 0
