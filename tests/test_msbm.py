"""The m-SBM generator (Appendix B.2): layout, structure, determinism, edge rates."""
import numpy as np
import pytest
import scipy.sparse as sp

from conftest import golden
from msbm import cell_sizes_equal, cell_sizes_from_proportions, category_probabilities, sample_msbm, configs


def _probs(a, b, c, d):
    return {(True, True): a, (False, True): b, (True, False): c, (False, False): d}


def test_example_b2_layout():
    gd = golden("example_b2.json")
    p = gd["probabilities"]
    g = sample_msbm(np.array(gd["cells"]), _probs(p["a_same_cluster_same_group"], p["b_diff_cluster_same_group"],
                                                   p["c_same_cluster_diff_group"], p["d_diff_cluster_diff_group"]),
                    seed=0, allow_isolated=True)
    assert (g.groups == 0).astype(int).tolist() == gd["g1"]
    assert (g.groups == 1).astype(int).tolist() == gd["g2"]
    for c, col in enumerate(gd["H_columns"]):
        assert (g.clusters == c).astype(int).tolist() == col


def test_example_b1_layout_h1():
    gd = golden("example_b1.json")
    g = sample_msbm(np.array(gd["cells"]), _probs(0.6, 0.2, 0.6, 0.2), seed=3, allow_isolated=True)
    assert np.all(g.groups == 0)
    for c, col in enumerate(gd["H_columns"]):
        assert (g.clusters == c).astype(int).tolist() == col


def test_fair_blocks_when_divisible():
    cells = cell_sizes_from_proportions(1200, [1, 2, 3], [1, 1, 2])
    # eq. fair-block: u_i^(j) / |C_i| = |V_j| / n for every cluster i
    n = cells.sum()
    np.testing.assert_allclose(cells / cells.sum(1, keepdims=True), np.tile(cells.sum(0) / n, (3, 1)))


@pytest.mark.parametrize("seed", [0, 7])
def test_structure_and_determinism(seed):
    cells = cell_sizes_equal(300, 3, 2)
    pr = _probs(0.3, 0.1, 0.2, 0.05)
    g = sample_msbm(cells, pr, seed=seed)
    W = g.to_scipy()
    assert abs(W - W.T).sum() == 0
    assert W.diagonal().sum() == 0
    for r in range(g.n):
        seg = g.col_idx[g.row_ptr[r]:g.row_ptr[r + 1]]
        assert np.all(np.diff(seg) > 0)
    g2 = sample_msbm(cells, pr, seed=seed)
    assert np.array_equal(g.col_idx, g2.col_idx) and np.array_equal(g.row_ptr, g2.row_ptr)
    g3 = sample_msbm(cells, pr, seed=seed + 1)
    assert not np.array_equal(g.col_idx, g3.col_idx[: g.col_idx.size]) or g.nnz != g3.nnz


def test_category_edge_rates():
    """Edge frequency per (same cluster?, same group?) category matches p (eq. p-msbm)."""
    cells = cell_sizes_equal(2000, 5, 2)
    pr = _probs(0.40, 0.20, 0.30, 0.10)
    g = sample_msbm(cells, pr, seed=0)
    rows = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    cols = g.col_idx
    up = rows < cols
    same_cl = g.clusters[rows[up]] == g.clusters[cols[up]]
    same_gr = g.groups[rows[up]] == g.groups[cols[up]]
    from msbm.generator import _pair_counts
    pc = _pair_counts(cells)
    for key, p in pr.items():
        cnt = np.sum((same_cl == key[0]) & (same_gr == key[1]))
        npairs = pc[key]
        sd = np.sqrt(npairs * p * (1 - p))
        assert abs(cnt - npairs * p) < 5 * sd, (key, cnt, npairs * p)


def test_degree_split_probabilities():
    cells = cell_sizes_equal(50_000, 20, 5)
    pr = category_probabilities(cells, 100.0, configs.SPLIT)
    # the printed per-category probabilities of this workload
    assert pr[(True, True)] == pytest.approx(0.1002, rel=2e-3)
    assert pr[(True, False)] == pytest.approx(0.0125, rel=2e-3)
    assert pr[(False, True)] == pytest.approx(1.58e-3, rel=5e-3)
    assert pr[(False, False)] == pytest.approx(2.63e-4, rel=5e-3)


def test_small_workload_shapes():
    c = configs.msbm_n2000_k5_h2()
    g = c["graph"]
    assert g.n == 2000 and abs(g.nnz / g.n - 379.6) < 5
    assert np.all(np.bincount(g.groups) == 1000)
    assert np.all(np.bincount(g.clusters) == 400)


@pytest.mark.parametrize("s", [2, 3, 5, 17, 64, 301])
def test_tri_unrank_is_the_row_order_enumeration(s):
    """Every rank maps to its pair (r, c), r < c, in row order: exactly np.triu_indices(s, 1)."""
    from msbm.generator import _tri_unrank

    idx = np.arange(s * (s - 1) // 2)
    r, c = _tri_unrank(idx, np.full(idx.size, s))
    rr, cc = np.triu_indices(s, 1)
    assert np.array_equal(r, rr) and np.array_equal(c, cc)


def test_tri_unrank_row_boundaries_at_large_sizes():
    """Around every tested row start of a large cell (where a float square root alone would land in
    the neighbouring row), the rank maps to the closed-form pair."""
    from msbm.generator import _tri_unrank

    rng = np.random.default_rng(0)
    for s in (10**5, 999_983, 2_000_000):
        rows = np.concatenate([[0, 1, s - 3, s - 2], rng.integers(0, s - 1, 200)])
        start = rows * (2 * s - rows - 1) // 2
        for off in (-1, 0, 1):
            idx = start + off
            ok = (idx >= 0) & (idx < s * (s - 1) // 2)
            idx, base = idx[ok], rows[ok]
            r, c = _tri_unrank(idx, np.full(idx.size, s))
            want_r = np.where(off < 0, base - 1, base)
            want_start = want_r * (2 * s - want_r - 1) // 2
            assert np.array_equal(r, want_r)
            assert np.array_equal(c, idx - want_start + want_r + 1)
            assert np.all((r < c) & (c < s))


def test_pair_counts_brute_force():
    from msbm.generator import _pair_counts

    cells = np.array([[3, 1, 0], [2, 2, 4], [1, 0, 5]])
    clu = np.repeat(np.repeat(np.arange(3), 3), cells.reshape(-1))
    grp = np.repeat(np.tile(np.arange(3), 3), cells.reshape(-1))
    n = clu.size
    want = {(a, b): 0 for a in (True, False) for b in (True, False)}
    for i in range(n):
        for j in range(i + 1, n):
            want[(bool(clu[i] == clu[j]), bool(grp[i] == grp[j]))] += 1
    assert _pair_counts(cells) == want


def test_gaussian_edge_weights_recomputed():
    """w_ij = exp(-||x_i - x_j||^2 / (2 s^2)) on every stored entry, from the returned features, and
    symmetric (w_ij = w_ji)."""
    from msbm.generator import gaussian_edge_weights

    cells = cell_sizes_equal(300, 3, 2)
    g = sample_msbm(cells, category_probabilities(cells, 12, (0.5, 0.25, 0.15, 0.10)), seed=5)
    w, r2, x = gaussian_edge_weights(g, dim=4, mean_scale=2.0, bandwidth=1.5, seed=6)
    rows = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    np.testing.assert_allclose(r2, ((x[rows] - x[g.col_idx]) ** 2).sum(axis=1), rtol=1e-12)
    np.testing.assert_allclose(w, np.exp(-r2 / (2 * 1.5**2)), rtol=1e-12)
    W = sp.csr_matrix((w, g.col_idx, g.row_ptr), shape=(g.n, g.n))
    assert abs(W - W.T).max() == 0.0
    assert np.all((w > 0) & (w <= 1))
