"""Pins of the oracle's unnormalized extension (L = D - W with the constraint F^T H = 0, H^T H = I).

The normalized problem of the paper reduces to the unnormalized one of the FairSC model it builds
on (Kleindessner, Samadi, Awasthi and Morgenstern, ICML 2019) when D is replaced by I: the fair
embedding is the k smallest eigenvectors of Z^T L Z with Z an orthonormal basis of null(F^T), and
s-FairSC's deflated operator P L P + sigma (I - P) must give the same spectrum and subspace (the
unnormalized reading of Prop. 3.3).  Every reference here is formed by a route the oracle does not
use: the nullspace and the projector from a complete QR factorisation of F (the oracle takes them
from an SVD and a Cholesky solve), and a closed form on the complete graph.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import fairsc, problem, sfairsc


def random_graph(n, h, seed, density=0.3):
    rng = np.random.default_rng(seed)
    A = (rng.random((n, n)) < density) * rng.uniform(0.5, 2.0, (n, n))
    W = np.triu(A, 1)
    W = W + W.T
    for i in range(n):  # a ring, so no vertex is isolated
        j = (i + 1) % n
        W[i, j] = W[j, i] = max(W[i, j], 0.3)
    groups = rng.integers(0, h, n)
    groups[:h] = np.arange(h)
    return sp.csr_matrix(W), groups


def qr_complement(F):
    """Orthonormal basis of null(F^T): the trailing n - r columns of a complete QR of F (rank r)."""
    Q, _ = np.linalg.qr(F, mode="complete")
    return Q[:, F.shape[1]:]


@pytest.mark.parametrize("n,h,k,seed", [(40, 2, 3, 0), (48, 3, 4, 1), (56, 4, 5, 2)])
def test_spectrum_and_subspace_equal_the_nullspace_formulation(n, h, k, seed):
    W, groups = random_graph(n, h, seed)
    lam, H, X, sigma, _ = fairsc.sfairsc_dense(W, groups, h, k, normalized=False)
    L = problem.laplacian(W).toarray()
    _, F, _ = problem.fairness_constraints(groups, h)
    Z = qr_complement(F)
    mu, Y = np.linalg.eigh(Z.T @ L @ Z)
    np.testing.assert_allclose(lam, mu[:k], atol=1e-11 * sigma)
    # same subspace when the k-th gap is clear: principal angles between H and Z Y_k (both orthonormal)
    assert mu[k] - mu[k - 1] > 1e-6 * sigma
    s = np.linalg.svd(H.T @ (Z @ Y[:, :k]), compute_uv=False)
    np.testing.assert_allclose(s, 1.0, atol=1e-10)
    # the unnormalized embedding is X itself (no D^{-1/2} scaling)
    np.testing.assert_array_equal(H, X)


@pytest.mark.parametrize("n,sizes", [(12, (4, 4, 4)), (15, (2, 6, 7)), (10, (5, 5))])
def test_complete_graph_closed_form(n, sizes):
    """K_n: L = n I - 1 1^T and F^T 1 = 0 for any groups, so on null(F^T) the spectrum is 0
    (the constant vector) and n; sigma = ||L||_1 = 2 (n - 1)."""
    groups = np.repeat(np.arange(len(sizes)), sizes)
    h = len(sizes)
    W = sp.csr_matrix(np.ones((n, n)) - np.eye(n))
    k = 4
    lam, H, _, sigma, _ = fairsc.sfairsc_dense(W, groups, h, k, normalized=False)
    assert sigma == pytest.approx(2.0 * (n - 1), rel=1e-15)
    np.testing.assert_allclose(lam, [0.0] + [float(n)] * (k - 1), atol=1e-11 * n)
    # the first column is the normalised constant vector, up to sign
    np.testing.assert_allclose(np.abs(H[:, 0]), 1.0 / np.sqrt(n), atol=1e-12)


@pytest.mark.parametrize("h", [2, 3, 5])
def test_matrix_free_operator_equals_projector_form(h):
    """The matrix-free P(L(P w)) - sigma P w + sigma w with P = I - Q Q^T, Q an orthonormal basis
    of range(F) from a QR factorisation, and sigma = ||L||_1 = 2 max_i d_i."""
    n = 36
    W, groups = random_graph(n, h, 70 + h)
    op = sfairsc.SFairSCOperator(W, groups, h, normalized=False)
    d = problem.degrees(W)
    assert op.sigma == pytest.approx(2.0 * d.max(), rel=1e-14)
    _, F, _ = problem.fairness_constraints(groups, h)
    Q, _ = np.linalg.qr(F)
    P = np.eye(n) - Q @ Q.T
    L = np.diag(d) - W.toarray()
    A = P @ L @ P - op.sigma * P + op.sigma * np.eye(n)
    np.testing.assert_allclose(op.apply(np.eye(n)), A, atol=1e-12 * op.sigma)
    # range(F) is the eigenspace of sigma (the unnormalized reading of Prop. 3.2)
    np.testing.assert_allclose(op.apply(F), op.sigma * F, atol=1e-12 * op.sigma * np.abs(F).max())
