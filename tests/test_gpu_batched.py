"""Batched form: many graphs in one persistent launch, each checked against the oracle.

Every graph's eigenvalues, residuals (with the oracle's FP64 operator), the
invariants F^T H = 0 and H^T D H = I, the eigenspace and the column signs are
compared with the oracle's dense s-FairSC solve (Algorithm 3), or, for the
larger graphs, with its sparse FP64 eigensolve.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

from conftest import graph_tensors
from msbm import category_probabilities, cell_sizes_equal, configs, sample_msbm
from oracle import fairsc, problem
from oracle.sfairsc import operator_from_graph, residual_norms, sign_normalize, smallest_eigenpairs

pytestmark = pytest.mark.gpu

STATUS_OK, BAD_CSR, ISOLATED, EMPTY_GROUP, NONFINITE, NOT_CONVERGED = 0, -2, -3, -4, -6, -7


def principal_angle(A, B):
    Qa, _ = np.linalg.qr(A)
    Qb, _ = np.linalg.qr(B)
    s = np.linalg.svd(Qa.T @ Qb, compute_uv=False)
    return float(np.arccos(np.clip(s.min(), -1.0, 1.0)))


def as_batch_entry(g, k, h):
    rp, ci, v, gr = graph_tensors(g, torch.float32)
    return {"row_ptr": rp, "col_idx": ci, "values": v, "groups": gr, "k": k, "h": h}


def oracle_reference(g, k):
    """Oracle eigenpairs of the graph (its 0/1 weights are exact in FP32)."""
    assert np.array_equal(g.values.astype(np.float32).astype(np.float64), g.values)
    W = g.to_scipy()
    op = operator_from_graph(g)
    if g.n <= 2500:
        lref, Href, _, _, _ = fairsc.sfairsc_dense(W, g.groups, g.h, k + 1)
    else:
        lref, Xref = smallest_eigenpairs(op, k + 1, tol=1e-13, method="eigsh")
        Href = Xref / np.sqrt(problem.degrees(W))[:, None]
    return W, op, lref, Href


def check_graph(g, k, lam, H, W, op, lref, Href):
    sigma = op.sigma
    # eigenvalues: relative error <= 1e-4 (absolute in units of sigma for lambda ~ 0)
    big = np.abs(lref[:k]) >= 1e-3 * sigma
    err = np.where(big, np.abs(lam - lref[:k]) / np.maximum(np.abs(lref[:k]), 1e-300), np.abs(lam - lref[:k]) / sigma)
    assert err.max() <= 1e-4, (lam, lref[:k])
    d = problem.degrees(W)
    X = H * np.sqrt(d)[:, None]
    res = residual_norms(op, lam, X)
    assert res.max() <= 1e-6 * sigma * 1.01, res.max() / sigma
    _, F, _ = problem.fairness_constraints(g.groups, g.h)
    if g.h > 1:
        assert np.abs(F.T @ H).max() <= 1e-5 * np.abs(H).sum(axis=0).max()
    G = (H.T * d) @ H
    assert np.abs(G - np.eye(k)).max() <= 1e-5
    gap = lref[k] - lref[k - 1]
    if gap > 100 * 1e-6 * sigma:
        Xr = Href[:, :k] * np.sqrt(d)[:, None]
        assert principal_angle(X, Xr) <= 1e-4
    # column signs: for simple, well separated eigenvalues H matches the oracle's sign convention
    Xr = sign_normalize(Href[:, :k] * np.sqrt(d)[:, None])
    for c in range(k):
        lo = lref[c] - lref[c - 1] if c > 0 else np.inf
        hi = lref[c + 1] - lref[c]
        if min(lo, hi) > 1e-3 * sigma:
            top = np.sort(np.abs(Xr[:, c]))[-2:]
            if top[1] - top[0] > 1e-6:
                assert float(X[:, c] @ Xr[:, c]) > 0.99, c


def small_batch(count, seed):
    """Uneven small m-SBM graphs in the shape of the batched workload (oracle-sized)."""
    rng = np.random.default_rng(seed)
    out = []
    for t in range(count):
        k = int(rng.integers(3, 11))
        h = int(rng.integers(2, 7))
        n = int(round(np.exp(rng.uniform(np.log(300), np.log(2400)))))
        n = max(n, 4 * k * h)
        deg = float(rng.uniform(16, 64))
        cells = cell_sizes_equal(n, k, h)
        probs = category_probabilities(cells, min(deg, 0.5 * n), configs.SPLIT)
        g = sample_msbm(cells, probs, seed=seed * 1000 + t)
        out.append((g, k, h))
    return out


def run_batch(items, autotune=False, **kw):
    from paper_2210_16435_gb300.solver import FairSCBatch

    b = FairSCBatch([as_batch_entry(g, k, h) for g, k, h in items], autotune=autotune, **kw)
    status, info = b.solve(allow_not_converged=True)
    lams = [x.cpu().numpy() for x in b.lam]
    Hs = [x.cpu().numpy() for x in b.H]
    b.close()
    return status, info, lams, Hs


def test_small_batch_vs_oracle(built_lib):
    items = small_batch(24, seed=11)
    status, info, lams, Hs = run_batch(items)
    assert status == [STATUS_OK] * len(items), status
    assert info["converged"] == len(items)
    assert info["max_resid"] <= 1e-6
    for (g, k, h), lam, H in zip(items, lams, Hs):
        W, op, lref, Href = oracle_reference(g, k)
        check_graph(g, k, lam, H, W, op, lref, Href)


def test_teams_split_large_graphs(built_lib):
    """A few large graphs among many small ones: the large ones are solved by teams of CTAs."""
    items = small_batch(40, seed=12)
    rng = np.random.default_rng(5)
    big = []
    for t in range(3):
        n = 20000 + 3000 * t
        k, h = 6 + t, 3 + t
        cells = cell_sizes_equal(n, k, h)
        probs = category_probabilities(cells, 48.0, configs.SPLIT)
        big.append((sample_msbm(cells, probs, seed=777 + t), k, h))
    order = list(rng.permutation(len(items) + len(big)))
    allg = items + big
    allg = [allg[i] for i in order]
    status, info, lams, Hs = run_batch(allg)
    assert status == [STATUS_OK] * len(allg), status
    assert sum(info["teams"][1:]) >= 1, info  # at least one team of 2+ CTAs
    for (g, k, h), lam, H in zip(allg, lams, Hs):
        if g.n > 10000:
            W, op, lref, Href = oracle_reference(g, k)
            check_graph(g, k, lam, H, W, op, lref, Href)
    # the small graphs, spot-checked
    for (g, k, h), lam, H in list(zip(allg, lams, Hs))[:6]:
        if g.n <= 2500:
            W, op, lref, Href = oracle_reference(g, k)
            check_graph(g, k, lam, H, W, op, lref, Href)


def test_team_results_match_single_cta(built_lib):
    """A graph solved by a team of 16 CTAs and by one CTA: the same eigenpairs to the solver tolerance."""
    from paper_2210_16435_gb300 import binding as B
    from paper_2210_16435_gb300.solver import FairSCBatch

    n, k, h = 16000, 5, 3
    cells = cell_sizes_equal(n, k, h)
    g = sample_msbm(cells, category_probabilities(cells, 40.0, configs.SPLIT), seed=4242)
    b = FairSCBatch([as_batch_entry(g, k, h)])
    B.sfairsc_batch_schedule(b.handle, 1, 16, 0.0)
    st, info = b.solve()
    assert st[0] == STATUS_OK and info["teams"][4] >= 1 and info["max_team"] == 16, info
    lam_team, H_team = b.lam[0].cpu().numpy(), b.H[0].cpu().numpy()
    B.sfairsc_batch_schedule(b.handle, 1, 1, 1.0)
    st1, info1 = b.solve()
    assert st1[0] == STATUS_OK and info1["teams"][1:] == [0, 0, 0, 0] and info1["max_team"] == 1, info1
    lam_one, H_one = b.lam[0].cpu().numpy(), b.H[0].cpu().numpy()
    b.close()
    W, op, lref, Href = oracle_reference(g, k)
    assert np.abs(lam_team - lam_one).max() <= 1e-6 * op.sigma
    check_graph(g, k, lam_team, H_team, W, op, lref, Href)
    check_graph(g, k, lam_one, H_one, W, op, lref, Href)


def test_autotune_and_graph_replay(built_lib):
    from paper_2210_16435_gb300.solver import FairSCBatch

    items = small_batch(20, seed=14)
    b = FairSCBatch([as_batch_entry(g, k, h) for g, k, h in items], autotune=True)
    st1, info1 = b.solve()
    lam1 = [x.cpu().numpy().copy() for x in b.lam]
    st2, info2 = b.solve()  # replay of the captured launch sequence
    lam2 = [x.cpu().numpy() for x in b.lam]
    b.close()
    assert info1["autotuned"] == 1 and info1["ms_autotune"] > 0
    assert st1 == st2 == [STATUS_OK] * len(items)
    for a, c in zip(lam1, lam2):  # same schedule and inputs: bitwise the same results
        assert np.array_equal(a, c)
    for (g, k, h), lam in list(zip(items, lam1))[:5]:
        W, op, lref, Href = oracle_reference(g, k)
        assert np.abs(lam - lref[:k]).max() <= 1e-6 * op.sigma


def test_h1_and_unit_groups(built_lib):
    """h = 1 (no fairness constraint: plain normalized spectral clustering) inside a batch."""
    items = small_batch(6, seed=15)
    n, k = 900, 4
    cells = cell_sizes_equal(n, k, 1)
    g1 = sample_msbm(cells, category_probabilities(cells, 30.0, configs.SPLIT), seed=99)
    items.append((g1, k, 1))
    status, info, lams, Hs = run_batch(items)
    assert status == [STATUS_OK] * len(items)
    for (g, k, h), lam, H in zip(items, lams, Hs):
        W, op, lref, Href = oracle_reference(g, k)
        check_graph(g, k, lam, H, W, op, lref, Href)


def test_per_graph_errors(built_lib):
    """Input errors found on the device are reported per graph; the other graphs still solve."""
    from paper_2210_16435_gb300.solver import FairSCBatch

    items = small_batch(5, seed=16)
    entries = [as_batch_entry(g, k, h) for g, k, h in items]
    g0, k0, h0 = items[0]
    # isolated vertex: drop every edge of vertex 0 (both directions)
    W = g0.to_scipy().tolil()
    W[0, :] = 0
    W[:, 0] = 0
    Wc = sp.csr_matrix(W)
    Wc.eliminate_zeros()
    iso = {"row_ptr": torch.as_tensor(Wc.indptr, dtype=torch.int32, device="cuda"),
           "col_idx": torch.as_tensor(Wc.indices, dtype=torch.int32, device="cuda"),
           "values": torch.as_tensor(Wc.data, dtype=torch.float32, device="cuda"),
           "groups": torch.as_tensor(g0.groups, dtype=torch.int32, device="cuda"), "k": k0, "h": h0}
    # column index out of range
    badcol = as_batch_entry(g0, k0, h0)
    badcol["col_idx"] = badcol["col_idx"].clone()
    badcol["col_idx"][3] = g0.n + 5
    # negative weight
    neg = as_batch_entry(g0, k0, h0)
    neg["values"] = neg["values"].clone()
    neg["values"][7] = -1.0
    # NaN weight
    nanw = as_batch_entry(g0, k0, h0)
    nanw["values"] = nanw["values"].clone()
    nanw["values"][2] = float("nan")
    # empty group: labels never use group h-1
    emp = as_batch_entry(g0, k0, h0)
    emp["groups"] = torch.zeros_like(emp["groups"])
    b = FairSCBatch(entries + [iso, badcol, neg, nanw, emp])
    from paper_2210_16435_gb300 import binding as B

    rc, st, info = B.sfairsc_batch_solve(b.handle, b.count, allow=(0, -2, -3, -4, -6, -7))
    b.close()
    assert st[:5] == [STATUS_OK] * 5
    assert st[5:] == [ISOLATED, BAD_CSR, BAD_CSR, NONFINITE, EMPTY_GROUP], st
    assert rc == ISOLATED


def test_host_argument_errors(built_lib):
    from paper_2210_16435_gb300 import binding as B
    from paper_2210_16435_gb300.solver import FairSCBatch

    g, k, h = small_batch(1, seed=17)[0]
    e = as_batch_entry(g, k, h)
    e["k"] = g.n  # k > n - h + 1
    with pytest.raises(B.SFairSCError) as ex:
        FairSCBatch([e])
    assert ex.value.status == -5
    e = as_batch_entry(g, k, h)
    e["h"] = 33
    with pytest.raises(B.SFairSCError) as ex:
        FairSCBatch([e])
    assert ex.value.status == -1


def test_batch_workload_scaled(built_lib):
    """The 256-graph workload at reduced size: every graph converges; sampled graphs vs the oracle."""
    c = configs.msbm_batch256(count=64, scale=0.15)
    items = [(x["graph"], x["k"], x["h"]) for x in c["graphs"]]
    status, info, lams, Hs = run_batch(items)
    assert status == [STATUS_OK] * len(items), status
    assert info["max_resid"] <= 1e-6
    idx = np.random.default_rng(0).choice(len(items), 6, replace=False)
    for i in idx:
        g, k, h = items[i]
        W, op, lref, Href = oracle_reference(g, k)
        check_graph(g, k, lams[i], Hs[i], W, op, lref, Href)
