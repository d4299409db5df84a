"""The dense-constraint form (sfairsc_create_dense): a random dense F in place of group labels,
the random-Laplacian workload of Exp. 4, against the oracle.

The fused operator with P = I - C (C^T C)^{-1} C^T for C = D^{-1/2} F (eq. mv-Pw) is compared
element by element with the oracle's literal operator; the eigenpairs with dense Algorithm 2
(FairSC) given the same F; F^T H = 0 and H^T D H = I; a group F times an invertible R must give
the labelled problem's eigenvalues (only range(F) matters); p = 0 is plain SC; the eigenvalue
gradient (whose formula does not involve F) against the oracle's closed form.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

from conftest import graph_tensors
from msbm import configs
from oracle import fairsc, gradient, problem
from oracle.sfairsc import SFairSCOperator

pytestmark = pytest.mark.gpu


def dense_ctx(g, F, k, prec, **kw):
    from paper_2210_16435_gb300.solver import FairSC

    rp, ci, v, _ = graph_tensors(g)
    return FairSC(rp, ci, v, None, k=k, prec=prec, F=torch.as_tensor(F, device="cuda"), **kw)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("n,h", [(3001, 5), (2000, 2), (1500, 9)])
def test_dense_operator_matches_oracle(built_lib, prec, n, h):
    c = configs.random_laplacian(n, h, seed=n % 7)
    g, F = c["graph"], c["F"]
    op = SFairSCOperator(g.to_scipy(), None, h, F=F)
    s = dense_ctx(g, F, 2, prec)
    assert s.sigma == pytest.approx(op.sigma, rel=1e-12)
    rng = np.random.default_rng(n)
    for nvec in (1, 2, 3, 4):
        w = rng.standard_normal((g.n, nvec))
        if prec == "mixed":
            w = w.astype(np.float32).astype(np.float64)
        got = s.apply_operator(torch.as_tensor(w, device="cuda")).double().cpu().numpy()
        err = np.abs(got - op.apply(w)).max() / (op.sigma * np.abs(w).max())
        assert err < (1e-13 if prec == "fp64" else 3e-6), (prec, nvec, err)
    s.close()


@pytest.mark.parametrize("prec,block", [("fp64", 1), ("mixed", 4), ("mixed", 1)])
def test_dense_solve_matches_fairsc(built_lib, prec, block):
    c = configs.random_laplacian(3000, 5, seed=3)
    g, F, h = c["graph"], c["F"], c["h"]
    W = g.to_scipy()
    for k in (5, 8, 10):
        lref, Href = fairsc.fairsc_dense(W, None, h, k + 1, F=F)
        s = dense_ctx(g, F, k, prec, block=block)
        lam, H, lab, info = s.solve()
        s.close()
        lam, H = lam.cpu().numpy(), H.cpu().numpy()
        tol = 1e-6 if prec == "fp64" else 1e-4
        assert np.abs(lam - lref[:k]).max() <= tol * np.abs(lref[:k]).max(), (k, lam, lref[:k])
        d = problem.degrees(W)
        op = SFairSCOperator(W, None, h, F=F)
        X = H * np.sqrt(d)[:, None]
        R = op.apply(X) - X * lam[None, :]
        assert (np.linalg.norm(R, axis=0) / np.linalg.norm(X, axis=0)).max() <= 1e-6 * op.sigma * 1.01
        inv_tol = 1e-9 if prec == "fp64" else 1e-5
        assert np.abs(F.T @ H).max() <= inv_tol * np.abs(F).sum(axis=0).max() * np.abs(H).max()
        assert info["fairness_err"] == pytest.approx(np.abs(F.T @ H).max(), rel=1e-6, abs=1e-12)
        assert np.abs((H.T * d) @ H - np.eye(k)).max() <= inv_tol
        assert lab.min() >= 0 and lab.max() < k


def test_group_constraints_as_dense_f(built_lib):
    """range(F) is all that matters: F_groups R (R invertible) reproduces the labelled problem."""
    from paper_2210_16435_gb300.solver import FairSC

    g = configs.msbm_n2000_k5_h2(scale=1.0)["graph"]
    cells_h = 2
    _, Fg, _ = problem.fairness_constraints(g.groups, cells_h)
    R = np.array([[2.5]])
    rp, ci, v, gr = graph_tensors(g)
    s = FairSC(rp, ci, v, gr, k=5, h=2, prec="fp64")
    lam_lab, _, _, _ = s.solve(want_labels=False)
    s.close()
    s = dense_ctx(g, Fg @ R, 5, "fp64")
    lam_d, _, _, _ = s.solve(want_labels=False)
    s.close()
    assert np.abs(lam_lab.cpu().numpy() - lam_d.cpu().numpy()).max() <= 1e-10


def test_no_constraint_columns_is_plain_sc(built_lib):
    from paper_2210_16435_gb300.solver import FairSC

    c = configs.random_laplacian(1200, 1, seed=4)
    g = c["graph"]
    rp, ci, v, gr = graph_tensors(g)
    s = FairSC(rp, ci, v, gr, k=4, h=1, prec="fp64")
    lam1, _, _, _ = s.solve(want_labels=False)
    s.close()
    s = dense_ctx(g, np.zeros((g.n, 0)), 4, "fp64")
    lam0, _, _, _ = s.solve(want_labels=False)
    s.close()
    np.testing.assert_allclose(lam0.cpu().numpy(), lam1.cpu().numpy(), atol=1e-12)
    lref, _ = fairsc.fairsc_dense(g.to_scipy(), np.zeros(g.n, int), 1, 4)
    assert np.abs(lam0.cpu().numpy() - lref).max() <= 1e-8


def test_dense_backward_matches_closed_form(built_lib):
    c = configs.random_laplacian(1500, 4, seed=5)
    g, F, h = c["graph"], c["F"], c["h"]
    k = 4
    lref, Href = fairsc.fairsc_dense(g.to_scipy(), None, h, k + 1, F=F)
    assert lref[k] - lref[k - 1] > 1e-4
    s = dense_ctx(g, F, k, "fp64", tol=1e-12)
    s.solve(want_labels=False)
    grad, _ = s.backward(torch.ones(k, dtype=torch.float64))
    s.close()
    gref = gradient.edge_gradient(g.row_ptr, g.col_idx, lref[:k], Href[:, :k])
    assert np.abs(grad.cpu().numpy() - gref).max() <= 1e-7 * np.abs(gref).max()
