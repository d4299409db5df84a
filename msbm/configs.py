"""The synthetic m-SBM workloads, by name, with their sizes and seeds.

Each builder returns a dict with the graph(s) and the solve parameters.  The
`scale` argument shrinks n (keeping degree, k, h and the split) so tests can
run the same shape at sizes the CPU oracle finishes in seconds.

Workloads (sizes as named):
  msbm_n2000_k5_h2        n = 2,000, 5 equal clusters, 2 equal groups,
                          p = .40 / .30 / .20 / .10, FP64 values, seed 0
  msbm_n50k_k20_h5        n = 50,000, 20 equal clusters, 5 equal groups,
                          mean degree 100, split 50/25/15/10, FP32, seed 1
  msbm_n1m_k50_h10        n = 1,000,000, 50 clusters ~ Dirichlet(5),
                          10 groups with Zipf(1) shares, mean degree 32,
                          split 50/25/15/10, BF16 0/1 values, seed 2
  msbm_batch256           256 graphs, n ~ logU[1e3, 6.4e4], k in {3..10},
                          h in {2..6}, mean degree ~ U[16, 64], seed 3
  msbm_n200k_k10_h4_gauss n = 200,000, 10 clusters, 4 groups, mean degree 48,
                          Gaussian-kernel weights exp(-r^2 / (2 s^2)), s = 2,
                          16-d features, seed 4
  random_laplacian(n, h)  the random-Laplacian workload (Exp. 4): random sparse
                          symmetric W (density 100 / n, weights U(0, 1]) and a
                          dense random constraint matrix F (n x (h-1), U[0, 1))
  paper_msbm(n, h)        the experiments' m-SBM (Exp. 1, App. C): k = 5 equal
                          clusters, h equal groups, probabilities
                          (a, b, c, d) = (10, 7, 4, 1) (log n / n)^(2/3) with
                          a same cluster & same group, b other cluster & same
                          group, c same cluster & other group, d neither
"""
from __future__ import annotations

import numpy as np

from .generator import (
    random_constraints,
    random_weighted_graph,
    cell_sizes_equal,
    cell_sizes_from_proportions,
    category_probabilities,
    gaussian_edge_weights,
    sample_msbm,
)

SPLIT = (0.50, 0.25, 0.15, 0.10)


def _scaled(n: int, scale: float, minimum: int) -> int:
    return max(minimum, int(round(n * scale)))


def msbm_n2000_k5_h2(scale: float = 1.0):
    n = _scaled(2000, scale, 40)
    k, h = 5, 2
    cells = cell_sizes_equal(n, k, h)
    probs = {(True, True): 0.40, (True, False): 0.30, (False, True): 0.20, (False, False): 0.10}
    g = sample_msbm(cells, probs, seed=0)
    return {"name": "msbm_n2000_k5_h2", "graph": g, "k": k, "h": h, "value_dtype": "f64", "prec": "fp64"}


def msbm_n50k_k20_h5(scale: float = 1.0):
    n = _scaled(50_000, scale, 400)
    k, h = 20, 5
    cells = cell_sizes_equal(n, k, h)
    probs = category_probabilities(cells, min(100.0, 0.5 * n), SPLIT)
    g = sample_msbm(cells, probs, seed=1)
    return {"name": "msbm_n50k_k20_h5", "graph": g, "k": k, "h": h, "value_dtype": "f32", "prec": "mixed"}


def zipf_shares(h: int, s: float = 1.0) -> np.ndarray:
    w = 1.0 / np.arange(1, h + 1) ** s
    return w / w.sum()


def msbm_n1m_k50_h10(scale: float = 1.0):
    n = _scaled(1_000_000, scale, 2000)
    k, h = 50, 10
    rng = np.random.default_rng(2)
    cluster_props = rng.dirichlet(np.full(k, 5.0))
    cells = cell_sizes_from_proportions(n, cluster_props, zipf_shares(h))
    probs = category_probabilities(cells, 32.0, SPLIT)
    g = sample_msbm(cells, probs, seed=2)
    return {"name": "msbm_n1m_k50_h10", "graph": g, "k": k, "h": h, "value_dtype": "bf16", "prec": "mixed"}


def msbm_batch256(count: int = 256, scale: float = 1.0, seed: int = 3):
    """Independent graphs of uneven size, with their per-graph k and h."""
    rng = np.random.default_rng(seed)
    out = []
    for t in range(count):
        n = int(round(np.exp(rng.uniform(np.log(1000), np.log(64000))) * scale))
        k = int(rng.integers(3, 11))
        h = int(rng.integers(2, 7))
        deg = float(rng.uniform(16, 64))
        n = max(n, 4 * k * h)
        cells = cell_sizes_equal(n, k, h)
        probs = category_probabilities(cells, min(deg, 0.5 * n), SPLIT)
        g = sample_msbm(cells, probs, seed=seed * 100_000 + t)
        out.append({"graph": g, "k": k, "h": h})
    return {"name": "msbm_batch256", "graphs": out, "value_dtype": "f32", "prec": "mixed", "block": 4}


def msbm_n200k_k10_h4_gauss(scale: float = 1.0, bandwidth: float = 2.0):
    n = _scaled(200_000, scale, 400)
    k, h = 10, 4
    cells = cell_sizes_equal(n, k, h)
    probs = category_probabilities(cells, min(48.0, 0.5 * n), SPLIT)
    g = sample_msbm(cells, probs, seed=4)
    w, r2, x = gaussian_edge_weights(g, dim=16, mean_scale=2.0, bandwidth=bandwidth, seed=4)
    g.values = w.astype(np.float32).astype(np.float64)
    return {"name": "msbm_n200k_k10_h4_gauss", "graph": g, "k": k, "h": h, "value_dtype": "f32",
            "prec": "mixed", "r2": r2, "features": x, "bandwidth": bandwidth}


def paper_msbm(n: int, h: int, k: int = 5, seed: int = 0):
    """The m-SBM of the paper's experiments (App. B.2 model, Exp. 1 and App. C sizes): fair
    ground truth (equal cells), a > b > c > d so that edges follow groups more than clusters and
    unconstrained SC tends to split by group."""
    cells = cell_sizes_equal(n, k, h)
    base = (np.log(n) / n) ** (2.0 / 3.0)
    probs = {(True, True): min(1.0, 10 * base), (False, True): min(1.0, 7 * base),
             (True, False): min(1.0, 4 * base), (False, False): min(1.0, base)}
    g = sample_msbm(cells, probs, seed=seed * 1000 + 7 * h + n % 997)
    return {"name": f"paper_msbm_n{n}_h{h}", "graph": g, "k": k, "h": h, "value_dtype": "f64", "prec": "fp64"}


def random_laplacian(n: int, h: int = 5, k: int = 5, mean_degree: float = 100.0, seed: int = 0):
    """The random-Laplacian workload of Exp. 4: a random sparse symmetric W and a random dense F
    (the paper does not state the sparsity of this experiment; mean degree 100 is the reading
    taken here)."""
    g = random_weighted_graph(n, min(1.0, mean_degree / (n - 1)), seed=seed * 1000 + 11)
    F = random_constraints(n, h - 1, seed=seed * 1000 + 12)
    return {"name": f"random_laplacian_n{n}_h{h}", "graph": g, "F": F, "k": k, "h": h, "value_dtype": "f64",
            "prec": "fp64"}


BUILDERS = {
    "msbm_n2000_k5_h2": msbm_n2000_k5_h2,
    "msbm_n50k_k20_h5": msbm_n50k_k20_h5,
    "msbm_n1m_k50_h10": msbm_n1m_k50_h10,
    "msbm_batch256": msbm_batch256,
    "msbm_n200k_k10_h4_gauss": msbm_n200k_k10_h4_gauss,
}
