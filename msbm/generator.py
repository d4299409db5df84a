"""m-SBM graph sampler (Appendix B.2, eq. p-msbm / w-msbm / fair-block).

Vertex order is cluster-major and group-minor: cluster 1's group-1 vertices
come first, then cluster 1's group-2 vertices, and so on.  This is the layout
of Example B.2, whose g^(1), g^(2) and H the tests pin.

Sampling: for every unordered pair of (cluster, group) cells the number of
edges is Binomial(#pairs, p) and the edges are a uniform subset of that size
without replacement, which is exactly an independent Bernoulli(p) draw per
vertex pair.  Every graph is returned as a symmetric CSR matrix with int32
indices, sorted column indices per row and no diagonal entries.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Graph",
    "cell_sizes_equal",
    "cell_sizes_from_proportions",
    "category_probabilities",
    "sample_msbm",
    "gaussian_edge_weights",
    "graph_from_dense",
]


@dataclass
class Graph:
    """A symmetric graph in CSR form plus its planted partition.

    row_ptr: int32[n+1]; col_idx: int32[nnz]; values: float64[nnz]
    groups: int32[n] in [0, h)  (the protected groups V_1..V_h)
    clusters: int32[n] in [0, k) (the planted ground-truth clusters C_1..C_k)
    """

    row_ptr: np.ndarray
    col_idx: np.ndarray
    values: np.ndarray
    groups: np.ndarray
    clusters: np.ndarray
    h: int
    k: int
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.row_ptr.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.col_idx.shape[0])

    def degrees(self) -> np.ndarray:
        return np.add.reduceat(self.values, self.row_ptr[:-1]) if self.nnz else np.zeros(self.n)

    def to_scipy(self):
        import scipy.sparse as sp

        return sp.csr_matrix((self.values, self.col_idx, self.row_ptr), shape=(self.n, self.n))


def _largest_remainder(total: int, proportions: np.ndarray) -> np.ndarray:
    """Integer split of `total` proportional to `proportions` (Hamilton's method).

    Ties in the fractional parts go to the lower index, so the split is
    deterministic.
    """
    p = np.asarray(proportions, dtype=np.float64)
    p = p / p.sum()
    raw = total * p
    base = np.floor(raw).astype(np.int64)
    rest = int(total - base.sum())
    if rest > 0:
        frac = raw - base
        order = np.lexsort((np.arange(p.size), -frac))
        base[order[:rest]] += 1
    return base


def cell_sizes_equal(n: int, k: int, h: int) -> np.ndarray:
    """k x h cell sizes |V_j cap C_i| for equal clusters and equal groups."""
    return cell_sizes_from_proportions(n, np.ones(k), np.ones(h))


def cell_sizes_from_proportions(n: int, cluster_props, group_props) -> np.ndarray:
    """k x h cell sizes: clusters split n, then each cluster splits over groups.

    Each cluster is divided over the groups in the global group proportions,
    which is the fair-block condition (eq. fair-block) up to integer rounding.
    """
    csize = _largest_remainder(n, np.asarray(cluster_props))
    gp = np.asarray(group_props, dtype=np.float64)
    return np.stack([_largest_remainder(int(c), gp) for c in csize]).astype(np.int64)


def _pair_counts(cells: np.ndarray):
    """Unordered vertex-pair counts per category (same cluster?, same group?)."""
    cells = np.asarray(cells, dtype=np.int64)
    n = int(cells.sum())
    ss = int((cells * (cells - 1) // 2).sum())
    csum = cells.sum(axis=1)
    gsum = cells.sum(axis=0)
    same_cluster = int((csum * (csum - 1) // 2).sum())
    same_group = int((gsum * (gsum - 1) // 2).sum())
    total = n * (n - 1) // 2
    return {
        (True, True): ss,
        (True, False): same_cluster - ss,
        (False, True): same_group - ss,
        (False, False): total - same_cluster - same_group + ss,
    }


def category_probabilities(cells, mean_degree: float, split) -> dict:
    """Edge probability per category from an expected mean degree and a split.

    split = (same cluster & same group, same cluster & diff group,
             diff cluster & same group, diff cluster & diff group) shares of
    the expected edge count n * mean_degree / 2.
    """
    cells = np.asarray(cells, dtype=np.int64)
    n = int(cells.sum())
    edges = n * mean_degree / 2.0
    pc = _pair_counts(cells)
    keys = [(True, True), (True, False), (False, True), (False, False)]
    out = {}
    for key, share in zip(keys, split):
        npairs = pc[key]
        out[key] = 0.0 if npairs == 0 else min(1.0, share * edges / npairs)
    return out


def _tri_unrank(idx: np.ndarray, s: np.ndarray):
    """Map a rank in [0, s(s-1)/2) to the pair (r, c), r < c, in row order."""
    idx = idx.astype(np.int64)
    s = s.astype(np.int64)
    two_s1 = 2 * s - 1
    r = np.floor((two_s1 - np.sqrt(np.maximum(two_s1.astype(np.float64) ** 2 - 8.0 * idx, 0.0))) / 2.0).astype(np.int64)
    r = np.clip(r, 0, np.maximum(s - 2, 0))

    def start(rr):
        return rr * (2 * s - rr - 1) // 2

    for _ in range(4):  # exact integer correction of the float estimate
        hi = start(r) > idx
        r = np.where(hi, r - 1, r)
        lo = start(r + 1) <= idx
        r = np.where(lo & (r + 1 <= s - 2), r + 1, r)
    c = idx - start(r) + r + 1
    return r, c


def _sample_pairs(rng, cells: np.ndarray, probs: dict):
    """Edge list (i < j) of one m-SBM draw."""
    k, h = cells.shape
    sizes = cells.reshape(-1).astype(np.int64)
    offs = np.concatenate([[0], np.cumsum(sizes)[:-1]])
    ncell = sizes.size
    A, B = np.triu_indices(ncell)
    sa, sb = sizes[A], sizes[B]
    npairs = np.where(A == B, sa * (sa - 1) // 2, sa * sb)
    same_cl = (A // h) == (B // h)
    same_gr = (A % h) == (B % h)
    p = np.empty(A.size)
    for key, val in probs.items():
        p[(same_cl == key[0]) & (same_gr == key[1])] = val
    keep = (npairs > 0) & (p > 0)
    A, B, sa, sb, npairs, p = A[keep], B[keep], sa[keep], sb[keep], npairs[keep], p[keep]
    counts = rng.binomial(npairs, p)

    rows_i, rows_j = [], []
    dense = counts > 0.05 * npairs
    # Dense blocks: exact subset without replacement.
    for t in np.nonzero(dense)[0]:
        sel = rng.choice(int(npairs[t]), size=int(counts[t]), replace=False)
        rows_i.append(np.full(sel.size, t, dtype=np.int64))
        rows_j.append(sel.astype(np.int64))
    # Sparse blocks: draw with replacement, drop repeats, top up the deficit.
    # Keys are global pair ranks base[block] + local rank; only the (few)
    # repeats need a block lookup.
    sp_blocks = np.nonzero(~dense & (counts > 0))[0]
    if sp_blocks.size:
        need = counts[sp_blocks].astype(np.int64)
        npb = npairs[sp_blocks].astype(np.int64)
        base = np.concatenate([[0], np.cumsum(npb)[:-1]]).astype(np.int64)
        keys = np.empty(0, dtype=np.int64)
        todo = need.copy()
        for _ in range(64):
            tot = int(todo.sum())
            if tot == 0:
                break
            blk = np.repeat(np.arange(sp_blocks.size), todo)
            loc = np.minimum((rng.random(tot) * npb[blk]).astype(np.int64), npb[blk] - 1)
            keys = np.sort(np.concatenate([keys, base[blk] + loc]))
            dup = np.nonzero(keys[1:] == keys[:-1])[0] + 1
            if dup.size == 0:
                break
            lost = np.bincount(np.searchsorted(base, keys[dup], side="right") - 1, minlength=sp_blocks.size)
            keys = np.delete(keys, dup)
            todo = lost
        blk_of = np.searchsorted(base, keys, side="right") - 1
        rows_i.append(sp_blocks[blk_of].astype(np.int64))
        rows_j.append(keys - base[blk_of])
    if not rows_i:
        return np.empty(0, np.int64), np.empty(0, np.int64)
    t = np.concatenate(rows_i)
    loc = np.concatenate(rows_j)
    a, b = A[t], B[t]
    same = a == b
    i = np.empty(t.size, dtype=np.int64)
    j = np.empty(t.size, dtype=np.int64)
    # Off-diagonal cell pairs: rank = r * |b| + c.
    nd = ~same
    i[nd] = offs[a[nd]] + loc[nd] // sizes[b[nd]]
    j[nd] = offs[b[nd]] + loc[nd] % sizes[b[nd]]
    # Same-cell pairs: triangular rank.
    if same.any():
        r, c = _tri_unrank(loc[same], sizes[a[same]])
        i[same] = offs[a[same]] + r
        j[same] = offs[a[same]] + c
    return i, j


def _to_csr(n: int, i: np.ndarray, j: np.ndarray, w: np.ndarray | None = None):
    rows = np.concatenate([i, j]).astype(np.int64)
    cols = np.concatenate([j, i]).astype(np.int64)
    if w is None:
        key = rows * n + cols
        key.sort()
        rows, cols, vals = key // n, key % n, None
    else:
        order = np.argsort(rows * n + cols, kind="stable")
        rows, cols, vals = rows[order], cols[order], np.concatenate([w, w])[order]
    counts = np.bincount(rows, minlength=n)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    if row_ptr[-1] > np.iinfo(np.int32).max:
        raise ValueError("nnz exceeds int32 CSR range")
    return row_ptr.astype(np.int32), cols.astype(np.int32), vals


def sample_msbm(cells, probs: dict, seed: int, max_attempts: int = 8, allow_isolated: bool = False) -> Graph:
    """Draw an m-SBM graph with the given k x h cell sizes and category probabilities.

    probs maps (same_cluster, same_group) -> edge probability (eq. p-msbm).
    Unit edge weights (alpha = beta = 1).  A draw with an isolated vertex is
    redrawn with seed * 2**32 + attempt, since the method assumes D > 0.
    """
    cells = np.asarray(cells, dtype=np.int64)
    k, h = cells.shape
    n = int(cells.sum())
    sizes = cells.reshape(-1)
    groups = np.repeat(np.tile(np.arange(h), k), sizes).astype(np.int32)
    clusters = np.repeat(np.repeat(np.arange(k), h), sizes).astype(np.int32)
    for attempt in range(max_attempts):
        s = seed if attempt == 0 else seed * 2**32 + attempt
        rng = np.random.default_rng(s)
        i, j = _sample_pairs(rng, cells, probs)
        deg = np.bincount(i, minlength=n) + np.bincount(j, minlength=n)
        if allow_isolated or (deg > 0).all():
            row_ptr, col, _ = _to_csr(n, i, j)
            vals = np.ones(col.size, dtype=np.float64)
            return Graph(row_ptr, col, vals, groups, clusters, h, k,
                         meta={"seed": int(s), "attempt": attempt, "probs": {str(kk): v for kk, v in probs.items()}})
    raise RuntimeError(f"m-SBM draw kept an isolated vertex after {max_attempts} attempts")


def random_weighted_graph(n: int, density: float, seed: int, max_attempts: int = 8) -> Graph:
    """A random symmetric sparse weight matrix (the random-Laplacian workload, Sec. 4 datasets):
    every unordered pair of distinct vertices is an edge with probability `density`, with a
    weight drawn uniformly from (0, 1]; no self loops; redrawn (seed * 2**32 + attempt) while a
    vertex is isolated.  There is no cluster structure: groups and clusters are all zero."""
    cells = np.array([[n]], dtype=np.int64)
    for attempt in range(max_attempts):
        s = seed if attempt == 0 else seed * 2**32 + attempt
        rng = np.random.default_rng(s)
        i, j = _sample_pairs(rng, cells, {(True, True): density})
        deg = np.bincount(i, minlength=n) + np.bincount(j, minlength=n)
        if (deg > 0).all():
            w = 1.0 - rng.random(i.size)  # (0, 1]
            row_ptr, col, vals = _to_csr(n, i, j, w)
            z = np.zeros(n, dtype=np.int32)
            return Graph(row_ptr, col, vals, z, z.copy(), 1, 1, meta={"seed": int(s), "density": density})
    raise RuntimeError(f"random graph kept an isolated vertex after {max_attempts} attempts")


def random_constraints(n: int, p: int, seed: int) -> np.ndarray:
    """A dense n x p constraint matrix with entries uniform in [0, 1) (the random-Laplacian
    experiment's F, a placeholder without group meaning); full column rank with probability 1."""
    return np.random.default_rng(seed).random((n, p))


def gaussian_edge_weights(g: Graph, dim: int, mean_scale: float, bandwidth: float, seed: int):
    """Gaussian-kernel weights on the graph's pattern.

    x_i ~ N(mu_{cluster(i)}, I_dim) with mu_c ~ N(0, mean_scale^2 I_dim);
    w_ij = exp(-||x_i - x_j||^2 / (2 s^2)).  Returns (weights, squared
    distances r2, features) with weights and r2 aligned to g.col_idx.
    """
    rng = np.random.default_rng(seed)
    mu = rng.normal(0.0, mean_scale, size=(g.k, dim))
    x = mu[g.clusters] + rng.normal(0.0, 1.0, size=(g.n, dim))
    x = x.astype(np.float32).astype(np.float64)
    rows = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    r2 = np.zeros(g.nnz)
    for c in range(dim):
        d = x[rows, c] - x[g.col_idx, c]
        r2 += d * d
    w = np.exp(-r2 / (2.0 * bandwidth * bandwidth))
    return w, r2, x


def graph_from_dense(W: np.ndarray, groups, clusters=None, k: int | None = None) -> Graph:
    """CSR Graph from a dense symmetric weight matrix (zero diagonal)."""
    W = np.asarray(W, dtype=np.float64)
    n = W.shape[0]
    if not np.allclose(W, W.T) or np.any(np.diag(W) != 0):
        raise ValueError("W must be symmetric with zero diagonal")
    rows, cols = np.nonzero(W)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=row_ptr[1:])
    groups = np.asarray(groups, dtype=np.int32)
    clusters = np.zeros(n, np.int32) if clusters is None else np.asarray(clusters, dtype=np.int32)
    return Graph(row_ptr.astype(np.int32), cols.astype(np.int32), W[rows, cols].copy(), groups, clusters,
                 int(groups.max()) + 1, int(k if k is not None else clusters.max() + 1))
