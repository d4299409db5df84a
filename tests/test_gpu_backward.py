"""Eigenvalue-sum gradient kernel (SDDMM) against the oracle's closed form and finite differences."""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

from conftest import graph_tensors
from msbm import category_probabilities, cell_sizes_equal, gaussian_edge_weights, sample_msbm
from oracle import fairsc, gradient

pytestmark = pytest.mark.gpu


def small_graph(seed, n=240, k=3, h=2, gauss=False):
    cells = cell_sizes_equal(n, k, h)
    probs = category_probabilities(cells, 30, (0.5, 0.25, 0.15, 0.10))
    g = sample_msbm(cells, probs, seed=seed)
    if gauss:
        w, r2, _ = gaussian_edge_weights(g, 4, 2.0, 2.0, seed)
        g.values = w
        g.r2 = r2
    return g


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_backward_matches_closed_form(built_lib, prec):
    from paper_2210_16435_gb300.solver import FairSC

    g = small_graph(1)
    k = 3
    rp, ci, v, gr = graph_tensors(g)
    # eigenvector error is about residual / gap, so the FP64 path is solved tightly
    s = FairSC(rp, ci, v, gr, k=k, h=2, prec=prec, tol=1e-12 if prec == "fp64" else 1e-6)
    lam, H, _, _ = s.solve(want_labels=False)
    grad, _ = s.backward(torch.ones(k, dtype=torch.float64))
    W = g.to_scipy()
    lref, Href, *_ = fairsc.sfairsc_dense(W, g.groups, 2, k + 1)
    assert lref[k] - lref[k - 1] > 1e-3
    gref = gradient.edge_gradient(g.row_ptr, g.col_idx, lref[:k], Href[:, :k])
    tol = 1e-8 if prec == "fp64" else 1e-4
    scale = np.abs(gref).max()
    assert np.abs(grad.cpu().numpy() - gref).max() <= tol * scale
    s.close()


def test_backward_vs_finite_differences_and_bandwidth(built_lib):
    from paper_2210_16435_gb300.solver import FairEigenvalueSum

    g = small_graph(2, n=180, gauss=True)
    k = 3
    s_bw = 2.0
    rp, ci, v, gr = graph_tensors(g)
    vals = v.clone().requires_grad_(True)
    bw = torch.tensor(s_bw, dtype=torch.float64, requires_grad=True)
    lam = FairEigenvalueSum.apply(vals, rp, ci, gr, k, 2, bw, {"prec": "fp64", "tol": 1e-12})
    lam.sum().backward()
    gv = vals.grad.cpu().numpy()
    rows = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    rng = np.random.default_rng(0)
    f0 = float(lam.sum())
    for e in rng.choice(g.nnz, 6, replace=False):
        a, b = rows[e], g.col_idx[e]
        e2 = np.nonzero((rows == b) & (g.col_idx == a))[0][0]
        for step in (1e-6, 1e-4):
            fd = gradient.edge_gradient_fd(g.row_ptr, g.col_idx, g.values, g.groups, 2, k, a, b, step=step)
            # rounding noise of a central difference of dense FP64 eigenvalue sums
            noise = 10 * np.finfo(float).eps * g.n * abs(f0) / step
            assert abs(gv[e] + gv[e2] - fd) <= 1e-5 * abs(fd) + noise, (e, step, gv[e] + gv[e2], fd)

    def f(sb):
        w = np.exp(-g.r2 / (2 * sb * sb))
        return gradient.eigsum_dense(g.row_ptr, g.col_idx, w, g.groups, 2, k)

    fd_s = (f(s_bw + 1e-6) - f(s_bw - 1e-6)) / 2e-6
    noise = 10 * np.finfo(float).eps * g.n * abs(f0) / 1e-6
    assert abs(bw.grad.item() - fd_s) <= 1e-5 * abs(fd_s) + noise
