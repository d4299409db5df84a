"""The fair spectral clustering problem's matrices, written out literally (FP64).

Sec. 2.1: W symmetric, w_ij >= 0, w_ii = 0, no isolated vertex, d_i = sum_j w_ij.
eq. group-vec: G in {0,1}^{n x h}, g_is = 1 iff v_i in V_s.
eq. f0h: F0 = G - 1 z^T with z = G^T 1 / n.
Lemma 2.1: F = F0(:, 1:h-1) has rank h-1 and F^T H = 0 is group fairness.
Sec. 2.2 / Algorithm 1: L = D - W, L_n = D^{-1/2} L D^{-1/2}.
Sec. 3.2 (first variant): C = D^{-1/2} F.
App. C (Parameter sigma): sigma = ||L_n||_1.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def adjacency(row_ptr, col_idx, values, n=None):
    """W as a scipy CSR matrix (FP64)."""
    n = len(row_ptr) - 1 if n is None else n
    return sp.csr_matrix((np.asarray(values, np.float64), np.asarray(col_idx), np.asarray(row_ptr)), shape=(n, n))


def degrees(W) -> np.ndarray:
    """d_i = sum_j w_ij (Sec. 2.1)."""
    return np.asarray(W.sum(axis=1)).ravel()


def laplacian(W):
    """L = D - W (Algorithm 1 step 1, Algorithm 3 step 1)."""
    return sp.diags(degrees(W)) - W


def normalized_laplacian(W):
    """L_n = D^{-1/2} L D^{-1/2} (Algorithm 3 step 2)."""
    d = degrees(W)
    if np.any(d <= 0):
        raise ValueError("isolated vertex: D must be positive definite (Sec. 2.1)")
    s = sp.diags(1.0 / np.sqrt(d))
    return (s @ laplacian(W) @ s).tocsr()


def group_indicator(groups, h: int) -> np.ndarray:
    """G (eq. group-vec): g_is = 1 iff vertex i is in group s."""
    groups = np.asarray(groups)
    G = np.zeros((groups.size, h))
    G[np.arange(groups.size), groups] = 1.0
    return G


def fairness_constraints(groups, h: int):
    """(F0, F, z): F0 = G - 1 z^T, z = G^T 1 / n (eq. f0h), F = F0(:, 1:h-1) (Lemma 2.1)."""
    G = group_indicator(groups, h)
    n = G.shape[0]
    z = G.sum(axis=0) / n
    F0 = G - np.outer(np.ones(n), z)
    return F0, F0[:, : h - 1], z


def constraint_matrix(W, groups, h: int, normalized: bool = True, F=None) -> np.ndarray:
    """C = D^{-1/2} F (Sec. 3.2) for the normalized problem, F itself otherwise.

    F defaults to the group constraints of Lemma 2.1; a dense F (n x (h-1), full
    column rank) stands for any other linear constraint F^T H = 0 (the random
    Laplacian experiment, where F is a random matrix)."""
    if F is None:
        _, F, _ = fairness_constraints(groups, h)
    F = np.asarray(F, dtype=np.float64)
    if not normalized:
        return F
    return F / np.sqrt(degrees(W))[:, None]


def sigma_one_norm(A) -> float:
    """||A||_1 = max column sum of |a_ij| (App. C, Parameter sigma)."""
    A = sp.csc_matrix(A) if sp.issparse(A) else A
    if sp.issparse(A):
        return float(np.max(np.asarray(abs(A).sum(axis=0)).ravel()))
    return float(np.max(np.abs(A).sum(axis=0)))
