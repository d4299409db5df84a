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


def _warm_eigsum(op_base, X0, row_ptr, col_idx, values, groups, h, k, tol=1e-13):
    """Sum of the k smallest eigenvalues of the problem with new weights, by the oracle's own
    Lanczos (tol 1e-13 sigma), started from a fixed combination of the base eigenvectors."""
    from oracle.lanczos import thick_restart_lanczos
    from oracle.problem import adjacency
    from oracle.sfairsc import SFairSCOperator

    op = SFairSCOperator(adjacency(row_ptr, col_idx, values), groups, h, sigma=op_base.sigma)
    v0 = X0 @ np.random.default_rng(7).standard_normal(X0.shape[1])
    lam, _, info = thick_restart_lanczos(op.apply, op.n, k + 1, tol=tol, anorm=op.sigma, v0=v0)
    return float(lam[:k].sum())


def test_differentiation_workload_full_size(built_lib):
    """m-SBM n = 200,000, k = 10, h = 4, Gaussian weights (s = 2): the gradient of the sum of the 10
    smallest eigenvalues w.r.t. the weights and the bandwidth, at full size.

    GPU gradient vs the oracle's closed form (oracle solve at 1e-13 sigma) on 100 random edges and a
    200,000-entry sample, FP64 (tol 1e-12) and MIXED (tol 1e-6); scale invariance sum_e w_e g_e = 0;
    FP64 central differences of oracle solves: along a random +-1 combination of the 100 edges at
    steps 1e-6 (the stated step; bound from the eigenvalue-sum rounding) and 1e-4, per edge at step
    1e-4 on the four largest-gradient edges, and in the bandwidth s at step 1e-6."""
    from msbm import configs
    from oracle.lanczos import thick_restart_lanczos
    from oracle.sfairsc import operator_from_graph
    from paper_2210_16435_gb300.solver import FairEigenvalueSum

    c = configs.msbm_n200k_k10_h4_gauss()
    g, k, h, s_bw, r2 = c["graph"], c["k"], c["h"], c["bandwidth"], c["r2"]
    rp, ci, v, gr = graph_tensors(g, torch.float32)
    grads = {}
    for prec, tol in (("fp64", 1e-12), ("mixed", 1e-6)):
        vals = v.clone().requires_grad_(True)
        bw = torch.tensor(s_bw, dtype=torch.float64, requires_grad=True)
        lam = FairEigenvalueSum.apply(vals, rp, ci, gr, k, h, bw, {"prec": prec, "tol": tol})
        lam.sum().backward()
        grads[prec] = (vals.grad.double().cpu().numpy(), bw.grad.item(), lam.detach().cpu().numpy())
    gv, gs, lam64 = grads["fp64"]
    # scale invariance of the normalized problem: f(cW) = f(W)  =>  sum_e w_e g_e = 0
    assert abs(np.dot(g.values, gv)) <= 1e-8 * np.abs(g.values * gv).sum()

    op = operator_from_graph(g)
    lref, Xref, _ = thick_restart_lanczos(op.apply, g.n, k + 1, tol=1e-13, anorm=op.sigma, seed=0)
    assert np.abs(lam64 - lref[:k]).max() <= 1e-10 * op.sigma
    Href = Xref[:, :k] / np.sqrt(op.d)[:, None]
    rows = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.row_ptr))
    rng = np.random.default_rng(4)
    sample = rng.choice(g.nnz, 200_000, replace=False)
    ha, hb = Href[rows[sample]], Href[g.col_idx[sample]]
    gref = 0.5 * ((ha - hb) ** 2 - lref[None, :k] * (ha ** 2 + hb ** 2)).sum(axis=1)
    scale = np.abs(gref).max()
    # FP64 path at tol 1e-12: a vertex of small degree d amplifies its eigenvector error by d^{-1/2}
    # in H; relative to the largest gradient entry the difference stays near 1e-7
    assert np.abs(gv[sample] - gref).max() <= 1e-6 * scale
    assert np.abs(grads["mixed"][0][sample] - gref).max() <= 1e-4 * scale

    # 100 random undirected edges: both CSR entries of each
    edges = rng.choice(g.nnz, 100, replace=False)
    a_, b_ = rows[edges], g.col_idx[edges].astype(np.int64)
    key = rows * g.n + g.col_idx
    order = np.argsort(key)
    twin = order[np.searchsorted(key[order], b_ * g.n + a_)]
    g_und = gv[edges] + gv[twin]
    ha, hb = Href[a_], Href[b_]
    g_und_ref = ((ha - hb) ** 2 - lref[None, :k] * (ha ** 2 + hb ** 2)).sum(axis=1)
    assert np.abs(g_und - g_und_ref).max() <= 1e-6 * np.abs(g_und_ref).max()

    def f_with(values):
        return _warm_eigsum(op, Xref, g.row_ptr, g.col_idx, values, g.groups, h, k)

    sgn = rng.choice([-1.0, 1.0], 100)
    dirv = np.zeros(g.nnz)
    dirv[edges] = sgn
    dirv[twin] = sgn
    directional = float(np.dot(sgn, g_und))
    for step, rel, noise in ((1e-6, 1e-3, 2e-14 / 1e-6), (1e-4, 1e-3, 2e-14 / 1e-4)):
        fd = (f_with(g.values + step * dirv) - f_with(g.values - step * dirv)) / (2 * step)
        assert abs(fd - directional) <= rel * abs(directional) + noise, (step, fd, directional)
    for i in np.argsort(-np.abs(g_und))[:4]:
        e = np.zeros(g.nnz)
        e[edges[i]] = e[twin[i]] = 1.0
        fd = (f_with(g.values + 1e-4 * e) - f_with(g.values - 1e-4 * e)) / 2e-4
        assert abs(fd - g_und[i]) <= 1e-3 * abs(g_und[i]) + 2e-10, (i, fd, g_und[i])
    # bandwidth: w = exp(-r^2 / (2 s^2)) recomputed at s +- 1e-6
    fs = [f_with(np.exp(-r2 / (2 * sb * sb))) for sb in (s_bw + 1e-6, s_bw - 1e-6)]
    fd_s = (fs[0] - fs[1]) / 2e-6
    assert abs(gs - fd_s) <= 1e-4 * abs(fd_s) + 2e-8, (gs, fd_s)
    assert abs(grads["mixed"][1] - gs) <= 1e-3 * abs(gs)
