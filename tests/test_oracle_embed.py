"""Pins of the oracle's embedding step (Algorithm 3 step 4) and of its end-to-end Algorithm 3.

sign_normalize: the column sign rule (largest |x| positive, lowest row on
ties), checked on hand-built matrices where the wrong rules (argmax of x
instead of |x|, highest row on ties) give different answers.
embed: H = D^{-1/2} X, checked on a triangle whose degrees are perfect
squares (exact expected values written out), through the generalized
eigenproblem L h = lambda D h that H must satisfy when X holds eigenvectors
of L_n (Algorithm 1 / Sec. 2.2), and through H^T D H = I, F^T H = 0.
sfairsc(): Algorithm 3 end to end on exactly fair cliques joined by weak
edges recovers the cliques (Err = 0, eq. err) with balance 1 (eq. bal).
"""
import numpy as np
import pytest
import scipy.sparse as sp

from msbm import graph_from_dense
from oracle import problem, sfairsc
from oracle.metrics import balance, error_rate


def test_sign_rule_largest_magnitude_lowest_row():
    X = np.array([
        [0.3, 0.1, -0.2, 1.0],
        [-0.9, -0.5, 0.7, -1.0],
        [0.1, 0.5, -0.7, 0.5],
        [0.2, 0.2, 0.0, 0.0],
    ])
    S = sfairsc.sign_normalize(X)
    # column 0: largest |x| is -0.9 (row 1), not the largest x (0.3, row 0): flipped
    np.testing.assert_array_equal(S[:, 0], [-0.3, 0.9, -0.1, -0.2])
    # column 1: |-0.5| = |0.5| tie at rows 1 and 2; the lower row (1) is negative: flipped
    np.testing.assert_array_equal(S[:, 1], [-0.1, 0.5, -0.5, -0.2])
    # column 2: tie at rows 1 (+0.7) and 2 (-0.7); the lower row is positive: unchanged
    np.testing.assert_array_equal(S[:, 2], X[:, 2])
    # column 3: tie between rows 0 (+1) and 1 (-1): unchanged
    np.testing.assert_array_equal(S[:, 3], X[:, 3])
    # the input is not modified
    assert X[1, 0] == -0.9


def test_sign_rule_is_idempotent_and_sign_invariant():
    rng = np.random.default_rng(3)
    X = rng.standard_normal((50, 6))
    S = sfairsc.sign_normalize(X)
    np.testing.assert_array_equal(sfairsc.sign_normalize(S), S)
    np.testing.assert_array_equal(sfairsc.sign_normalize(-X), S)
    assert np.all(S[np.argmax(np.abs(S), axis=0), np.arange(6)] > 0)


def _triangle():
    # degrees 9, 16, 16: D^{-1/2} = diag(1/3, 1/4, 1/4)
    W = np.array([[0.0, 4.5, 4.5], [4.5, 0.0, 11.5], [4.5, 11.5, 0.0]])
    return graph_from_dense(W, [0, 0, 0])


def test_embed_exact_values_on_square_degrees():
    g = _triangle()
    X = np.array([[3.0, -12.0], [8.0, 4.0], [-4.0, 8.0]])  # signs already normalized in column 0
    op = sfairsc.operator_from_graph(g)
    H = sfairsc.embed(op, X)
    # column 0: largest |x| is +8 (row 1) -> kept; column 1: -12 (row 0) -> flipped
    expect = np.array([[1.0, 4.0], [2.0, -1.0], [-1.0, -2.0]])
    np.testing.assert_array_equal(H, expect)
    op_u = sfairsc.operator_from_graph(g, normalized=False)
    np.testing.assert_array_equal(sfairsc.embed(op_u, X), [[3.0, 12.0], [8.0, -4.0], [-4.0, -8.0]])


def _graph(n, h, seed):
    rng = np.random.default_rng(seed)
    A = (rng.random((n, n)) < 0.25) * rng.uniform(0.5, 2.0, (n, n))
    W = np.triu(A, 1)
    W = W + W.T
    for i in range(n):
        j = (i + 1) % n
        W[i, j] = W[j, i] = max(W[i, j], 0.3)
    groups = rng.integers(0, h, n)
    groups[:h] = np.arange(h)
    return graph_from_dense(W, groups)


def test_embed_solves_generalized_problem_plain_sc():
    """h = 1: X eigenvectors of L_n  =>  H = D^{-1/2} X satisfies L H = D H diag(lambda) (Algorithm 1)."""
    g = _graph(40, 1, 4)
    op = sfairsc.operator_from_graph(g)
    lam, X = sfairsc.smallest_eigenpairs(op, 5, method="dense")
    H = sfairsc.embed(op, X)
    W = g.to_scipy()
    L = problem.laplacian(W).toarray()
    d = problem.degrees(W)
    np.testing.assert_allclose(L @ H, (d[:, None] * H) * lam[None, :], atol=1e-12)
    np.testing.assert_allclose((H.T * d) @ H, np.eye(5), atol=1e-12)


@pytest.mark.parametrize("h", [2, 4])
def test_embed_fair_invariants(h):
    """H^T D H = I and F^T H = 0 (eq. normal-prob-fair) for the oracle's embedding of the s-FairSC eigenvectors."""
    g = _graph(45, h, 10 + h)
    op = sfairsc.operator_from_graph(g)
    lam, X = sfairsc.smallest_eigenpairs(op, 4, method="dense")
    H = sfairsc.embed(op, X)
    W = g.to_scipy()
    d = problem.degrees(W)
    _, F, _ = problem.fairness_constraints(g.groups, h)
    np.testing.assert_allclose((H.T * d) @ H, np.eye(4), atol=1e-12)
    np.testing.assert_allclose(F.T @ H, 0.0, atol=1e-12)
    # the generalized problem restricted to null(F^T): Z^T (L - lambda D) h = 0 for Z spanning null(F^T)
    Z = np.linalg.svd(F, full_matrices=True)[0][:, h - 1:]
    L = problem.laplacian(W).toarray()
    for i in range(4):
        np.testing.assert_allclose(Z.T @ (L @ H[:, i] - lam[i] * d * H[:, i]), 0.0, atol=1e-11)


@pytest.mark.parametrize("method", ["dense", "eigsh", "lanczos"])
def test_algorithm3_end_to_end_recovers_fair_cliques(method):
    """Exactly fair cliques with weak links: Algorithm 3 returns the cliques (Err = 0) and balance 1."""
    k, h, per = 4, 2, 8
    n = k * per
    clusters = np.repeat(np.arange(k), per)
    groups = np.tile(np.arange(h), n // h)
    W = (clusters[:, None] == clusters[None, :]).astype(float) - np.eye(n)
    for c in range(k):  # one weak edge from each clique to the next keeps the graph connected
        a, b = c * per, ((c + 1) % k) * per + 1
        W[a, b] = W[b, a] = 0.01
    g = graph_from_dense(W, groups, clusters, k)
    out = sfairsc.sfairsc(g, k, method=method, n_init=3)
    assert error_rate(out["labels"], clusters, k) == 0.0
    np.testing.assert_array_equal(balance(out["labels"], groups, k, h), np.ones(k))
    # lambda_1 = 0 with a constant column of H (Sec. 3.3: D^{1/2} 1 lies in null(C^T))
    assert abs(out["eigenvalues"][0]) <= 1e-10
    h0 = out["H"][:, 0]
    np.testing.assert_allclose(h0, h0[0], rtol=1e-8)
    assert sp.issparse(g.to_scipy())
