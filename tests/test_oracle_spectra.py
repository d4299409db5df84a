"""Pins of the oracle's eigen-solvers against the paper's propositions and closed forms."""
import numpy as np
import pytest
import scipy.sparse as sp

from msbm import cell_sizes_equal, graph_from_dense, sample_msbm
from oracle import fairsc, problem, sfairsc
from oracle.kmeans import kmeans
from oracle.metrics import error_rate


def random_graph(n, h, seed, density=0.3):
    rng = np.random.default_rng(seed)
    A = (rng.random((n, n)) < density) * rng.uniform(0.5, 2.0, (n, n))
    W = np.triu(A, 1)
    W = W + W.T
    # connect a ring so no vertex is isolated
    for i in range(n):
        j = (i + 1) % n
        W[i, j] = W[j, i] = max(W[i, j], 0.3)
    groups = rng.integers(0, h, n)
    groups[:h] = np.arange(h)
    return sp.csr_matrix(W), groups


@pytest.mark.parametrize("n,h,k,seed", [(40, 2, 3, 0), (50, 3, 4, 1), (60, 4, 5, 2), (45, 1, 3, 3)])
def test_three_formulations_same_spectrum(n, h, k, seed):
    """FairSC (Alg. 2), the first variant (eq. lveig) and s-FairSC (eq. asigma) agree (Prop. 3.3)."""
    W, groups = random_graph(n, h, seed)
    l1, H1 = fairsc.fairsc_dense(W, groups, h, k)
    l2, H2, _ = fairsc.variant_dense(W, groups, h, k)
    l3, H3, _, sigma, _ = fairsc.sfairsc_dense(W, groups, h, k)
    np.testing.assert_allclose(l1, l2, atol=1e-12)
    np.testing.assert_allclose(l1, l3, atol=1e-12)
    d = problem.degrees(W)
    # same subspace: principal angles between D^{1/2} H
    for Ha, Hb in [(H1, H3), (H2, H3)]:
        Qa, _ = np.linalg.qr(Ha * np.sqrt(d)[:, None])
        Qb, _ = np.linalg.qr(Hb * np.sqrt(d)[:, None])
        s = np.linalg.svd(Qa.T @ Qb, compute_uv=False)
        assert s.min() > 1 - 1e-10


@pytest.mark.parametrize("h", [2, 3, 5])
def test_prop31_projected_spectrum(h):
    """spec(P L_n P) = spec(L_n^v) plus h-1 zeros (Prop. 3.1, eq. blockAp)."""
    W, groups = random_graph(40, h, 10 + h)
    Ln = problem.normalized_laplacian(W).toarray()
    C = problem.constraint_matrix(W, groups, h)
    P = fairsc.projector(C)
    Lp = P @ Ln @ P
    _, _, lv_all = fairsc.variant_dense(W, groups, h, 1)
    lp = np.linalg.eigvalsh(0.5 * (Lp + Lp.T))
    expect = np.sort(np.concatenate([lv_all, np.zeros(h - 1)]))
    np.testing.assert_allclose(lp, expect, atol=1e-12)


def test_hotelling_shift_structure_and_invariance():
    """L_n^sigma = L_n^p + sigma U2 U2^T: eigenvalue sigma h-1 times on range(C); results do not depend on sigma."""
    h, k = 3, 4
    W, groups = random_graph(50, h, 21)
    As, sigma = fairsc.sfairsc_matrix(W, groups, h)
    C = problem.constraint_matrix(W, groups, h)
    np.testing.assert_allclose(As @ C, sigma * C, atol=1e-12)
    l1, H1, *_ = fairsc.sfairsc_dense(W, groups, h, k)
    l2, H2, *_ = fairsc.sfairsc_dense(W, groups, h, k, sigma=2 * sigma)
    np.testing.assert_allclose(l1, l2, atol=1e-12)
    # negative control: a shift below lambda_k lets sigma into the k smallest
    l3, *_ = fairsc.sfairsc_dense(W, groups, h, k, sigma=0.5 * l1[1] + 1e-3)
    assert np.any(np.abs(l3 - l1) > 1e-3)


def test_sigma_is_one_norm_and_bounds_spectrum():
    W, groups = random_graph(30, 2, 5)
    Ln = problem.normalized_laplacian(W).toarray()
    sigma = problem.sigma_one_norm(Ln)
    assert sigma == pytest.approx(np.abs(Ln).sum(axis=0).max())
    assert sigma >= np.linalg.eigvalsh(Ln).max() - 1e-12
    # label-free closed form of the 1-norm: 1 + max_j d_j^{-1/2} sum_i w_ij d_i^{-1/2}
    d = problem.degrees(W)
    Wd = W.toarray() / np.sqrt(np.outer(d, d))
    assert sigma == pytest.approx(1.0 + Wd.sum(axis=0).max(), rel=1e-14)


@pytest.mark.parametrize("n,h,k,seed", [(40, 2, 3, 0), (60, 3, 5, 4)])
def test_invariants(n, h, k, seed):
    """F^T H = 0, H^T D H = I (eq. normal-prob-fair) and tr(H^T L H) = sum of lambda (Theorem 2.1)."""
    W, groups = random_graph(n, h, seed)
    lam, H, *_ = fairsc.sfairsc_dense(W, groups, h, k)
    _, F, _ = problem.fairness_constraints(groups, h)
    D = np.diag(problem.degrees(W))
    L = problem.laplacian(W).toarray()
    assert np.abs(F.T @ H).max() < 1e-12
    np.testing.assert_allclose(H.T @ D @ H, np.eye(k), atol=1e-12)
    assert np.trace(H.T @ L @ H) == pytest.approx(lam.sum(), abs=1e-12)
    # lambda_1 = 0 with a constant eigenvector: 1^T F0 = 0 puts D^{1/2} 1 in null(C^T)
    assert abs(lam[0]) < 1e-12
    h1 = H[:, 0]
    assert np.ptp(h1) < 1e-10 * np.abs(h1).max()


def test_lemma21_rank():
    rng = np.random.default_rng(0)
    for h in [1, 2, 3, 7]:
        groups = rng.integers(0, h, 200)
        groups[:h] = np.arange(h)
        F0, F, z = problem.fairness_constraints(groups, h)
        assert np.linalg.matrix_rank(F0) == h - 1
        assert (np.linalg.matrix_rank(F) if h > 1 else 0) == h - 1
        np.testing.assert_allclose(F0 @ np.ones(h), 0, atol=1e-14)
        np.testing.assert_allclose(z, np.bincount(groups, minlength=h) / 200)


def test_lemma21_fairness_iff():
    """F^T H = 0 iff every cluster holds the groups in proportion (Lemma 2.1 (ii), eq. fair)."""
    groups = np.array([0, 0, 1, 1, 0, 0, 1, 1, 0, 1])
    fair = np.array([0, 0, 0, 0, 1, 1, 1, 1, 2, 2])
    unfair = np.array([0, 0, 1, 1, 0, 1, 1, 1, 2, 2])
    _, F, _ = problem.fairness_constraints(groups, 2)
    Hf = np.eye(3)[fair]
    Hu = np.eye(3)[unfair]
    assert np.abs(F.T @ Hf).max() < 1e-15
    assert np.abs(F.T @ Hu).max() > 0.1


def test_complete_graph_closed_form():
    """K_n: L_n = n/(n-1) I - J/(n-1): lambda = 0 once, then n/(n-1)."""
    n, h, k = 24, 3, 5
    W = sp.csr_matrix(np.ones((n, n)) - np.eye(n))
    groups = np.arange(n) % h
    lam, H, *_ = fairsc.sfairsc_dense(W, groups, h, k)
    assert abs(lam[0]) < 1e-12
    np.testing.assert_allclose(lam[1:], n / (n - 1), atol=1e-12)


def test_h1_is_plain_sc():
    """h = 1 drops the constraint: Algorithm 3 reduces to Algorithm 1."""
    W, _ = random_graph(40, 1, 8)
    lam, *_ = fairsc.sfairsc_dense(W, np.zeros(40, int), 1, 4)
    ref = np.linalg.eigvalsh(problem.normalized_laplacian(W).toarray())[:4]
    np.testing.assert_allclose(lam, ref, atol=1e-12)


def test_fair_cliques_zero_eigenvalues_and_exact_recovery():
    """Disjoint exactly-fair cliques: lambda_1..lambda_k = 0, k-means recovers them (Err = 0)."""
    k, h, per = 4, 2, 6
    n = k * per
    clusters = np.repeat(np.arange(k), per)
    groups = np.tile(np.arange(h), n // h)
    W = (clusters[:, None] == clusters[None, :]).astype(float) - np.eye(n)
    W = sp.csr_matrix(W)
    lam, H, *_ = fairsc.sfairsc_dense(W, groups, h, k)
    np.testing.assert_allclose(lam, 0, atol=1e-12)
    labels, _, _ = kmeans(H, k, seed=1, n_init=3)
    assert error_rate(labels, clusters, k) == 0.0


def test_matrix_free_operator_equals_dense_matrix():
    """The Sec. 3.4 matvec P(L_n(Pw)) - sigma P w + sigma w equals the dense eq. asigma."""
    for h in [1, 2, 4]:
        W, groups = random_graph(35, h, 30 + h)
        op = sfairsc.SFairSCOperator(W, groups, h)
        As, sigma = fairsc.sfairsc_matrix(W, groups, h)
        assert op.sigma == pytest.approx(sigma)
        np.testing.assert_allclose(op.apply(np.eye(35)), As, atol=1e-13)


def test_unnormalized_extension_invariants():
    h, k = 3, 4
    W, groups = random_graph(40, h, 40)
    lam, H, X, sigma, _ = fairsc.sfairsc_dense(W, groups, h, k, normalized=False)
    _, F, _ = problem.fairness_constraints(groups, h)
    assert np.abs(F.T @ H).max() < 1e-12
    np.testing.assert_allclose(H.T @ H, np.eye(k), atol=1e-12)
    assert sigma == pytest.approx(2 * problem.degrees(W).max())


def test_eigensolvers_agree_on_msbm():
    """Dense eigh, SciPy eigsh and the own thick-restart Lanczos on the same operator."""
    cells = cell_sizes_equal(300, 3, 3)
    pr = {(True, True): 0.3, (True, False): 0.2, (False, True): 0.08, (False, False): 0.04}
    g = sample_msbm(cells, pr, seed=11)
    op = sfairsc.operator_from_graph(g)
    k = 3
    ld, Xd = sfairsc.smallest_eigenpairs(op, k, method="dense")
    le, Xe = sfairsc.smallest_eigenpairs(op, k, method="eigsh")
    ll, Xl = sfairsc.smallest_eigenpairs(op, k, method="lanczos")
    np.testing.assert_allclose(le, ld, atol=1e-10)
    np.testing.assert_allclose(ll, ld, atol=1e-10)
    assert sfairsc.residual_norms(op, ll, Xl).max() < 1e-9 * op.sigma
    W = g.to_scipy()
    lf, _ = fairsc.fairsc_dense(W, g.groups, g.h, k)
    np.testing.assert_allclose(lf, ld, atol=1e-10)
