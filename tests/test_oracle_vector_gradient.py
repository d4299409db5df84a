"""Pins of the oracle's eigenvector-level gradient (a loss on H, not only on the eigenvalues).

Checked against central differences of the embedding computed by another route (the dense
s-FairSC matrix of eq. asigma, not Algorithm 2's pencil), against the eigenvalue gradient when
the loss only sees the eigenvalues, and against homogeneity: scaling W by c scales D by c, so
H(cW) = H(W) / sqrt(c) (H^T D H = I) and, for a loss linear in H, sum_e w_e g_e = -loss / 2.
"""
import numpy as np
import pytest

from msbm import graph_from_dense
from oracle import gradient


def small(n, h, seed, density=0.35):
    rng = np.random.default_rng(seed)
    A = (rng.random((n, n)) < density) * rng.uniform(0.5, 2.0, (n, n))
    W = np.triu(A, 1)
    W = W + W.T
    for i in range(n):
        j = (i + 1) % n
        W[i, j] = W[j, i] = max(W[i, j], 0.3)
    groups = rng.integers(0, h, n)
    groups[:h] = np.arange(h)
    return graph_from_dense(W, groups)


@pytest.mark.parametrize("n,h,k,seed", [(40, 2, 3, 0), (50, 3, 4, 1), (36, 1, 3, 2)])
def test_vector_gradient_vs_central_differences(n, h, k, seed):
    g = small(n, h, seed)
    rng = np.random.default_rng(100 + seed)
    G = rng.standard_normal((n, k))
    gl = rng.standard_normal(k)
    grad, lam, H = gradient.vector_gradient(g.row_ptr, g.col_idx, g.values, g.groups, h, k, G, gbar_lam=gl)
    rows = np.repeat(np.arange(n), np.diff(g.row_ptr))
    for e in rng.choice(g.nnz, 5, replace=False):
        a, b = rows[e], g.col_idx[e]
        sel = ((rows == a) & (g.col_idx == b)) | ((rows == b) & (g.col_idx == a))
        fs = []
        for sgn in (1, -1):
            vals = g.values.copy()
            vals[sel] += sgn * 1e-6
            l2, H2 = gradient.embedding_dense(g.row_ptr, g.col_idx, vals, g.groups, h, k)
            fs.append(np.sum(G * H2) + np.dot(gl, l2))
        fd = (fs[0] - fs[1]) / 2e-6
        got = grad[sel].sum()
        assert abs(got - fd) <= 1e-6 * max(1.0, abs(fd)), (e, got, fd)


def test_reduces_to_eigenvalue_gradient():
    g = small(45, 3, 7)
    k = 4
    gl = np.array([1.0, -0.5, 2.0, 0.25])
    grad, lam, H = gradient.vector_gradient(g.row_ptr, g.col_idx, g.values, g.groups, 3, k, np.zeros((45, k)),
                                           gbar_lam=gl)
    rows = np.repeat(np.arange(45), np.diff(g.row_ptr))
    ha, hb = H[rows], H[g.col_idx]
    ref = 0.5 * (gl[None, :] * ((ha - hb) ** 2 - lam[None, :] * (ha ** 2 + hb ** 2))).sum(axis=1)
    np.testing.assert_allclose(grad, ref, atol=1e-14)
    ones = gradient.vector_gradient(g.row_ptr, g.col_idx, g.values, g.groups, 3, k, np.zeros((45, k)),
                                    gbar_lam=np.ones(k))[0]
    np.testing.assert_allclose(gradient.edge_gradient(g.row_ptr, g.col_idx, lam, H), ones, atol=1e-14)


def test_homogeneity_of_a_linear_loss():
    g = small(42, 2, 9)
    k = 3
    G = np.random.default_rng(3).standard_normal((42, k))
    grad, lam, H = gradient.vector_gradient(g.row_ptr, g.col_idx, g.values, g.groups, 2, k, G)
    assert np.dot(g.values, grad) == pytest.approx(-0.5 * np.sum(G * H), rel=1e-9)
