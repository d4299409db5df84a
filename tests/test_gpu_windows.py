"""The operator's shared-memory windows (SpMV input staged per row segment).

A window changes where a gather reads ytil from (shared memory or L2), never
the arithmetic: the windowed and the plain SpMV must agree bit for bit, and
both must match the oracle's literal matvec P(L_n(P w)) - sigma P w + sigma w
(Sec. 3.4 (i)).  Checked on cluster-ordered m-SBM graphs (vertices numbered
cluster by cluster as in App. B.2, so windows serve most gathers), with a
ragged last window (n not a multiple of 4, the final window cut by n), and on
the same graph with its vertices shuffled (no locality: windows mostly off).
"""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

from conftest import graph_tensors
from msbm import category_probabilities, cell_sizes_from_proportions, graph_from_dense, sample_msbm
from oracle.sfairsc import SFairSCOperator

pytestmark = pytest.mark.gpu


def clustered(n, k, h, deg, seed):
    cells = cell_sizes_from_proportions(n, np.linspace(1, 2, k), 1.0 / np.arange(1, h + 1))
    return sample_msbm(cells, category_probabilities(cells, deg, (0.6, 0.25, 0.1, 0.05)), seed=seed)


def shuffled(g, seed):
    """The same graph with its vertices renumbered at random."""
    from msbm import Graph

    perm = np.random.default_rng(seed).permutation(g.n)
    inv = np.empty_like(perm)
    inv[perm] = np.arange(g.n)
    W = sp.csr_matrix((g.values, g.col_idx, g.row_ptr), shape=(g.n, g.n))
    P = W[perm][:, perm].tocsr()
    P.sort_indices()
    return Graph(P.indptr.astype(np.int32), P.indices.astype(np.int32), P.data.astype(np.float64),
                 g.groups[perm].astype(np.int32), g.clusters[perm].astype(np.int32), g.h, g.k)


def run(g, prec, vdt, nvec, window, seed=0):
    from paper_2210_16435_gb300.solver import FairSC

    rp, ci, v, gr = graph_tensors(g, vdt)
    s = FairSC(rp, ci, v, gr, k=4, h=g.h, prec=prec, block=4, spmv_window=window)
    rng = np.random.default_rng(seed)
    w = rng.standard_normal((g.n, nvec))
    if prec == "mixed":
        w = w.astype(np.float32).astype(np.float64)
    out = s.apply_operator(torch.as_tensor(w, device="cuda")).double().cpu().numpy()
    _, _, _, info = s.solve(want_labels=False)
    sigma = s.sigma
    s.close()
    return w, out, info, sigma


@pytest.mark.parametrize("prec,vdt", [("mixed", torch.bfloat16), ("mixed", torch.float32), ("fp64", torch.float64)])
def test_windowed_equals_plain_and_oracle(built_lib, prec, vdt):
    g = clustered(150_003, 8, 4, 24, seed=31)
    vals = g.values if vdt != torch.bfloat16 else g.values  # 0/1 weights are exact in every type
    op = SFairSCOperator(sp.csr_matrix((vals, g.col_idx, g.row_ptr), shape=(g.n, g.n)), g.groups, g.h)
    for nvec in (1, 2, 4):
        w, out_w, info, sigma = run(g, prec, vdt, nvec, 1, seed=nvec)
        _, out_p, info_p, _ = run(g, prec, vdt, nvec, 0, seed=nvec)
        # the two schedules sum each row's entries in the same order: the same bits
        assert np.array_equal(out_w, out_p), (prec, nvec)
        ref = op.apply(w)
        err = np.abs(out_w - ref).max() / (op.sigma * np.abs(w).max())
        assert err < (1e-13 if prec == "fp64" else 3e-6), (prec, nvec, err)
        assert info["spmv_windowed"] > 0 and info["spmv_in_window"] > 0.25, info
        assert info_p["spmv_windowed"] == 0
        assert info["max_resid"] <= 1e-6


def test_shuffled_vertices_still_correct(built_lib):
    g = shuffled(clustered(120_000, 6, 3, 20, seed=32), seed=5)
    op = SFairSCOperator(sp.csr_matrix((g.values, g.col_idx, g.row_ptr), shape=(g.n, g.n)), g.groups, g.h)
    w, out, info, _ = run(g, "mixed", torch.float32, 4, 1)
    err = np.abs(out - op.apply(w)).max() / (op.sigma * np.abs(w).max())
    assert err < 3e-6, err
    assert info["spmv_in_window"] < 0.5, info
