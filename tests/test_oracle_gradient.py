"""The eigenvalue-sum gradient against central finite differences and scale invariance."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import fairsc, gradient


def graph(n, h, seed, density=0.35):
    rng = np.random.default_rng(seed)
    A = (rng.random((n, n)) < density) * rng.uniform(0.5, 1.5, (n, n))
    W = np.triu(A, 1)
    W = W + W.T
    for i in range(n):
        W[i, (i + 1) % n] = W[(i + 1) % n, i] = max(W[i, (i + 1) % n], 0.4)
    groups = rng.integers(0, h, n)
    groups[:h] = np.arange(h)
    M = sp.csr_matrix(W)
    return M.indptr.astype(np.int32), M.indices.astype(np.int32), M.data.copy(), groups


@pytest.mark.parametrize("h,k,seed", [(2, 3, 0), (3, 4, 1)])
def test_edge_gradient_vs_fd(h, k, seed):
    rp, ci, v, groups = graph(36, h, seed)
    W = sp.csr_matrix((v, ci, rp))
    lam, H, *_ = fairsc.sfairsc_dense(W, groups, h, k + 1)
    assert lam[k] - lam[k - 1] > 1e-3        # f differentiable: lambda_k simple at the boundary
    g = gradient.edge_gradient(rp, ci, lam[:k], H[:, :k])
    rng = np.random.default_rng(seed)
    rows = np.repeat(np.arange(36), np.diff(rp))
    for e in rng.choice(len(ci), 8, replace=False):
        a, b = rows[e], ci[e]
        fd = gradient.edge_gradient_fd(rp, ci, v, groups, h, k, a, b, step=1e-5)
        # both CSR entries carry half of the undirected derivative
        e2 = np.nonzero((rows == b) & (ci == a))[0][0]
        assert g[e] + g[e2] == pytest.approx(fd, abs=1e-7, rel=1e-5)


def test_scale_invariance_sum_w_g_is_zero():
    """f(cW) = f(W) for L_n, so sum_e w_e g_e = 0."""
    rp, ci, v, groups = graph(30, 2, 4)
    W = sp.csr_matrix((v, ci, rp))
    lam, H, *_ = fairsc.sfairsc_dense(W, groups, 2, 3)
    g = gradient.edge_gradient(rp, ci, lam, H)
    assert abs(np.dot(v, g)) < 1e-12 * np.abs(v * g).sum() * 100


def test_bandwidth_gradient_vs_fd():
    rng = np.random.default_rng(5)
    n, h, k, s = 30, 2, 3, 1.5
    x = rng.standard_normal((n, 3))
    rp, ci, _, groups = graph(n, h, 6, density=0.5)
    rows = np.repeat(np.arange(n), np.diff(rp))
    r2 = ((x[rows] - x[ci]) ** 2).sum(1)

    def f(bw):
        w = np.exp(-r2 / (2 * bw * bw))
        return gradient.eigsum_dense(rp, ci, w, groups, h, k)

    w = np.exp(-r2 / (2 * s * s))
    lam, H, *_ = fairsc.sfairsc_dense(sp.csr_matrix((w, ci, rp)), groups, h, k)
    g = gradient.edge_gradient(rp, ci, lam, H)
    ds = gradient.bandwidth_gradient(g, w, s)
    fd = (f(s + 1e-5) - f(s - 1e-5)) / 2e-5
    assert ds == pytest.approx(fd, rel=1e-5, abs=1e-8)
