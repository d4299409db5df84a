"""End-to-end s-FairSC solves (Algorithm 3) against the oracle."""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

from conftest import graph_tensors
from msbm import category_probabilities, cell_sizes_equal, configs, sample_msbm
from oracle import fairsc, metrics, problem
from oracle.kmeans import kmeans as oracle_kmeans
from oracle.sfairsc import operator_from_graph, residual_norms, smallest_eigenpairs

pytestmark = pytest.mark.gpu


def principal_angle(A, B):
    Qa, _ = np.linalg.qr(A)
    Qb, _ = np.linalg.qr(B)
    s = np.linalg.svd(Qa.T @ Qb, compute_uv=False)
    return float(np.arccos(np.clip(s.min(), -1.0, 1.0)))


def eig_rel_err(got, ref, sigma, tol):
    """Relative error when lambda >= 1e-3 sigma, absolute (in units of sigma) below."""
    big = np.abs(ref) >= 1e-3 * sigma
    rel = np.where(big, np.abs(got - ref) / np.maximum(np.abs(ref), 1e-300), np.abs(got - ref) / sigma)
    return rel.max()


def solve_and_check(g, k, prec, block=1, lam_tol=None, normalized=True, ref=None, vdt=torch.float64, basis=0,
                    **opts):
    from paper_2210_16435_gb300.solver import FairSC

    rp, ci, v, gr = graph_tensors(g, vdt)
    s = FairSC(rp, ci, v, gr, k=k, h=g.h, prec=prec, block=block, normalized=normalized, basis=basis, **opts)
    lam, H, lab, info = s.solve()
    lam, H, lab = lam.cpu().numpy(), H.cpu().numpy(), lab.cpu().numpy()
    W = sp.csr_matrix((v.double().cpu().numpy(), g.col_idx, g.row_ptr), shape=(g.n, g.n))
    op = operator_from_graph(g, normalized=normalized)
    op.A = op.A  # same graph
    if ref is None:
        if g.n <= 2500:
            lref, Href, Xref, _, _ = fairsc.sfairsc_dense(W, g.groups, g.h, k + 1, normalized=normalized)
        else:
            lref, Xref = smallest_eigenpairs(op, k + 1, tol=1e-13, method="eigsh")
            d = problem.degrees(W)
            Href = Xref / np.sqrt(d)[:, None] if normalized else Xref
    else:
        lref, Href = ref
    lam_tol = lam_tol or (1e-6 if prec == "fp64" else 1e-4)
    assert eig_rel_err(lam, lref[:k], op.sigma, lam_tol) <= lam_tol, (lam, lref[:k])
    # residual with the oracle's FP64 operator on the returned H (X = D^{1/2} H)
    d = problem.degrees(W)
    X = H * np.sqrt(d)[:, None] if normalized else H
    res = residual_norms(op, lam, X)
    assert res.max() <= 1e-6 * op.sigma * 1.01, res.max() / op.sigma
    # invariants: F^T H = 0 and H^T D H = I (eq. normal-prob-fair)
    _, F, _ = problem.fairness_constraints(g.groups, g.h)
    tol_inv = 1e-9 if prec == "fp64" else 1e-5
    if g.h > 1:
        assert np.abs(F.T @ H).max() <= tol_inv * np.abs(H).sum(axis=0).max()
    G = (H.T * d) @ H if normalized else H.T @ H
    assert np.abs(G - np.eye(k)).max() <= tol_inv
    # subspace: compare in the Euclidean-orthonormal X coordinates when the gap is clear
    gap = lref[k] - lref[k - 1]
    if gap > 100 * 1e-6 * op.sigma:
        Xr = Href[:, :k] * np.sqrt(d)[:, None] if normalized else Href[:, :k]
        ang = principal_angle(X, Xr)
        assert ang <= 1e-4, ang
    assert abs(info["sigma"] - op.sigma) <= 1e-12 * op.sigma
    assert info["max_resid"] <= 1e-6
    s.close()
    return lam, H, lab, info


def test_n2000_k5_h2_fp64(built_lib):
    c = configs.msbm_n2000_k5_h2()
    g = c["graph"]
    lam, H, lab, info = solve_and_check(g, 5, "fp64")
    # clusters: balance equal to the oracle's k-means on the oracle's embedding
    W = g.to_scipy()
    lref, Href, *_ = fairsc.sfairsc_dense(W, g.groups, 2, 5)
    oref, _, _ = oracle_kmeans(Href, 5, seed=0, n_init=1, max_iter=100)
    assert metrics.balance_multiset(lab, g.groups, 5, 2) == metrics.balance_multiset(oref, g.groups, 5, 2)
    # and exactly the oracle's labels when the oracle clusters the library's own H
    omine, _, _ = oracle_kmeans(H, 5, seed=0, n_init=1, max_iter=100)
    assert np.array_equal(omine, lab)


def test_n2000_k5_h2_mixed(built_lib):
    g = configs.msbm_n2000_k5_h2()["graph"]
    solve_and_check(g, 5, "mixed")


@pytest.mark.parametrize("block", [2, 4])
def test_block_lanczos(built_lib, block):
    g = configs.msbm_n2000_k5_h2()["graph"]
    solve_and_check(g, 5, "fp64", block=block)
    solve_and_check(g, 5, "mixed", block=block)


@pytest.mark.parametrize("prec,block", [("mixed", 4), ("fp64", 1)])
def test_wide_basis(built_lib, prec, block):
    """A 136-column basis: the Gram-Schmidt kernel's two-panels-per-lane variant
    (more than 128 basis columns) and its shorter row slices."""
    g = configs.msbm_n2000_k5_h2()["graph"]
    lam, H, lab, info = solve_and_check(g, 5, prec, block=block, basis=136)
    assert info["basis"] == 136


def test_n50k_shape_scaled(built_lib):
    """The n = 50,000, k = 20, h = 5 workload's shape at n = 5,000."""
    g = configs.msbm_n50k_k20_h5(scale=0.1)["graph"]
    solve_and_check(g, 20, "mixed", vdt=torch.float32)
    solve_and_check(g, 20, "fp64", vdt=torch.float32)


@pytest.mark.parametrize("block", [1, 4])
def test_n50k_k20_h5_full_size(built_lib, block):
    """m-SBM n = 50,000, k = 20, h = 5 at its stated size, FP32 values, mixed precision, against
    the oracle's eigsh (tol 1e-13): eigenvalues, residuals, invariants, principal angles, and the
    cluster balance of the library's labels against the oracle's k-means on the oracle's H."""
    c = configs.msbm_n50k_k20_h5()
    g, k, h = c["graph"], c["k"], c["h"]
    op = operator_from_graph(g)
    lref, Xref = smallest_eigenpairs(op, k + 1, tol=1e-13, method="eigsh")
    d = problem.degrees(g.to_scipy())
    Href = Xref / np.sqrt(d)[:, None]
    lam, H, lab, info = solve_and_check(g, k, "mixed", block=block, vdt=torch.float32, ref=(lref, Href))
    from oracle.sfairsc import sign_normalize

    oref, _, _ = oracle_kmeans(sign_normalize(Xref[:, :k]) / np.sqrt(d)[:, None], k, seed=0, n_init=1, max_iter=100)
    assert metrics.balance_multiset(lab, g.groups, k, h) == metrics.balance_multiset(oref, g.groups, k, h)
    omine, _, _ = oracle_kmeans(H, k, seed=0, n_init=1, max_iter=100)
    assert np.array_equal(omine, lab)


def test_h1_plain_sc(built_lib):
    cells = cell_sizes_equal(1500, 4, 1)
    probs = category_probabilities(cells, 40, (0.7, 0.0, 0.3, 0.0))
    g = sample_msbm(cells, probs, seed=3)
    solve_and_check(g, 4, "fp64")


def test_unnormalized_extension(built_lib):
    cells = cell_sizes_equal(1200, 3, 3)
    probs = category_probabilities(cells, 40, (0.5, 0.25, 0.15, 0.10))
    g = sample_msbm(cells, probs, seed=4)
    solve_and_check(g, 3, "fp64", normalized=False)


def sparse_fair_clusters(k=10, per=200, h=2, matchings=4, seed=0):
    """k clusters of `per` vertices, each the union of `matchings` random matchings (average degree
    about 2 matchings, an expander: a wide gap above the k smallest eigenvalues), groups alternating
    inside every cluster (each cluster is fair), consecutive clusters joined by one weak edge."""
    from msbm import graph_from_dense

    rng = np.random.default_rng(seed)
    n = k * per
    W = np.zeros((n, n))
    for c in range(k):
        base = c * per
        for _ in range(matchings):
            p = rng.permutation(per)
            for i in range(per):
                if p[i] != i:
                    W[base + i, base + p[i]] = W[base + p[i], base + i] = 1.0
        nb = ((c + 1) % k) * per
        W[base, nb] = W[nb, base] = 0.05
    return graph_from_dense(W, np.tile(np.arange(h), n // h), np.repeat(np.arange(k), per), k)


def test_low_degree_final_check_lanes(built_lib):
    """MIXED, k = 10, average degree below 8: the final check's double-float SpMV runs one launch
    of eight vectors and one of two with two lanes per row, so each lane forms several columns."""
    g = sparse_fair_clusters()
    assert len(g.col_idx) / g.n <= 8.0  # FP64 operator lanes per row: 2
    solve_and_check(g, 10, "mixed", block=4)


def test_fair_cliques_exact_recovery(built_lib):
    """Disjoint exactly-fair cliques joined weakly: k-means recovers them (Err = 0)."""
    k, h, per = 4, 2, 50
    n = k * per
    clusters = np.repeat(np.arange(k), per)
    groups = np.tile(np.arange(h), n // h)
    W = (clusters[:, None] == clusters[None, :]).astype(float) - np.eye(n)
    for c in range(k):
        a, b = c * per, ((c + 1) % k) * per
        W[a, b] = W[b, a] = 0.01
    from msbm import graph_from_dense

    g = graph_from_dense(W, groups, clusters, k)
    lam, H, lab, info = solve_and_check(g, k, "fp64")
    assert metrics.error_rate(lab, clusters, k) == 0.0


def test_errors_are_reported(built_lib):
    from paper_2210_16435_gb300 import binding as B
    from paper_2210_16435_gb300.solver import FairSC

    g = configs.msbm_n2000_k5_h2(scale=0.1)["graph"]
    rp, ci, v, gr = graph_tensors(g)
    bad = gr.clone()
    bad[0] = 7
    with pytest.raises(B.SFairSCError) as e:
        FairSC(rp, ci, v, bad, k=2, h=2)
    assert e.value.status == -1
    with pytest.raises(B.SFairSCError) as e:
        FairSC(rp, ci, v, gr, k=2, h=3)  # group 2 empty
    assert e.value.status == -4
    vn = v.clone()
    vn[3] = float("nan")
    with pytest.raises(B.SFairSCError) as e:
        FairSC(rp, ci, vn, gr, k=2, h=2)
    assert e.value.status == -6
    cb = ci.clone()
    cb[0] = g.n + 5
    with pytest.raises(B.SFairSCError) as e:
        FairSC(rp, cb, v, gr, k=2, h=2)
    assert e.value.status == -2
    with pytest.raises(B.SFairSCError) as e:
        FairSC(rp, ci, v, gr, k=g.n, h=2)
    assert e.value.status == -5


@pytest.mark.parametrize("block", [1, 2, 4])
@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_deferred_second_projection(built_lib, prec, block):
    """Both reorthogonalisation modes reach the oracle's pairs; the deferred one (default) passes over
    the basis twice per step, the DGKS one up to three times."""
    g = configs.msbm_n50k_k20_h5(scale=0.1)["graph"]
    ref_l, ref_X = smallest_eigenpairs(operator_from_graph(g), 21, tol=1e-13, method="eigsh")
    d = problem.degrees(g.to_scipy())
    ref = (ref_l, ref_X / np.sqrt(d)[:, None])
    _, _, _, i0 = solve_and_check(g, 20, prec, block=block, vdt=torch.float32, ref=ref, orth_mode=0)
    _, _, _, i1 = solve_and_check(g, 20, prec, block=block, vdt=torch.float32, ref=ref, orth_mode=1)
    # every launch after a block's first: two sweeps; the start / fresh-block launches may take three
    assert i0["orth_sweeps"] <= 2 * i0["n_orth"] + (i0["restarts"] + 1), i0
    assert i1["orth_sweeps"] >= i0["orth_sweeps"] or i1["matvecs"] != i0["matvecs"]


@pytest.mark.parametrize("orth_mode", [0, 1])
def test_tensor_core_restart(built_lib, orth_mode):
    """The thick restart on the tensor cores (three-pass TF32, the default for a MIXED basis with blocks
    of 4) and on the CUDA cores both reach the oracle's pairs, with the same restart counts give or take
    one; the tensor-core path carries the deferred correction of the last block (orth_mode 0)."""
    g = configs.msbm_n50k_k20_h5(scale=0.1)["graph"]
    ref_l, ref_X = smallest_eigenpairs(operator_from_graph(g), 21, tol=1e-13, method="eigsh")
    d = problem.degrees(g.to_scipy())
    ref = (ref_l, ref_X / np.sqrt(d)[:, None])
    l0, _, _, i0 = solve_and_check(g, 20, "mixed", block=4, vdt=torch.float32, ref=ref, orth_mode=orth_mode,
                                   restart_mode=0)
    l1, _, _, i1 = solve_and_check(g, 20, "mixed", block=4, vdt=torch.float32, ref=ref, orth_mode=orth_mode,
                                   restart_mode=1)
    assert i0["restarts"] > 0 and i0["restarts_tc"] == i0["restarts"], i0
    assert i1["restarts_tc"] == 0
    assert abs(i0["restarts"] - i1["restarts"]) <= 1, (i0["restarts"], i1["restarts"])
    assert i0["dorth_err"] <= 1e-6, i0["dorth_err"]
    assert eig_rel_err(l0, l1, float(i0["sigma"]), 1e-4) <= 1e-4


def test_solve_into_caller_buffers(built_lib):
    """solve(out=...) writes into caller-owned tensors (pinned host here, allocated once) the same
    values as a solve into fresh device tensors."""
    from paper_2210_16435_gb300.solver import FairSC

    g = configs.msbm_n2000_k5_h2()["graph"]
    rp, ci, v, gr = graph_tensors(g)
    s = FairSC(rp, ci, v, gr, k=5, h=2, prec="mixed", block=4)
    lam, H, lab, _ = s.solve()
    outs = (torch.empty(5, dtype=torch.float64).pin_memory(), torch.empty(g.n, 5, dtype=torch.float64).pin_memory(),
            torch.empty(g.n, dtype=torch.int32).pin_memory())
    for _ in range(2):
        l2, H2, lab2, _ = s.solve(out=outs)
        assert l2 is outs[0] and H2 is outs[1] and lab2 is outs[2]
        assert torch.equal(l2, lam.cpu()) and torch.equal(H2, H.cpu()) and torch.equal(lab2, lab.cpu())
    with pytest.raises(ValueError):
        s.solve(out=(outs[0], outs[1][:, :4], outs[2]))
    s.close()
