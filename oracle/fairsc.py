"""Dense reference solvers of the fair SC problem (eq. normal-prob-fair), FP64.

Three routes to the same minimiser, each written as the paper states it:

* fairsc_dense   -- Algorithm 2 (FairSC): explicit nullspace basis Z of F^T,
                    matrix square root Q = (Z^T D Z)^{1/2}, M = Q^-1 Z^T L Z Q^-1,
                    H = Z Q^-1 X.
* variant_dense  -- Sec. 3.2, first variant: V = null(C^T), L_n^v = V^T L_n V
                    (eq. lveig), H = D^{-1/2} V Y.
* sfairsc_dense  -- the explicitly formed s-FairSC matrix
                    L_n^sigma = P L_n P + sigma (I - P) (eq. asigma) with
                    P = I - C (C^T C)^{-1} C^T (eq. mv-Pw), H = D^{-1/2} X
                    (Algorithm 3 steps 3-4, Proposition 3.3).

These are O(n^3) and meant for n up to a few thousand.
"""
from __future__ import annotations

import numpy as np

from .problem import constraint_matrix, degrees, fairness_constraints, laplacian, normalized_laplacian, sigma_one_norm


def _dense(A):
    return A.toarray() if hasattr(A, "toarray") else np.asarray(A)


def nullspace_basis(F: np.ndarray) -> np.ndarray:
    """Orthonormal basis of null(F^T): trailing columns of U in the full SVD of F (Sec. 3.1)."""
    n, p = F.shape
    if p == 0:
        return np.eye(n)
    U, s, _ = np.linalg.svd(F, full_matrices=True)
    rank = int(np.sum(s > s[0] * max(n, p) * np.finfo(float).eps))
    return U[:, rank:]


def fairsc_dense(W, groups, h: int, k: int, F=None):
    """Algorithm 2 (FairSC).  Returns (eigenvalues[k], H[n, k]).  F: a dense constraint matrix
    (n x (h-1)) in place of the group constraints."""
    L = _dense(laplacian(W))
    D = np.diag(degrees(W))
    if F is None:
        _, F, _ = fairness_constraints(groups, h)
    Z = nullspace_basis(F)                                   # step 2
    mu, E = np.linalg.eigh(Z.T @ D @ Z)                      # step 3: Q = (Z^T D Z)^{1/2}
    Qinv = (E / np.sqrt(mu)) @ E.T                           #         Q^{-1}
    M = Qinv @ (Z.T @ L @ Z) @ Qinv                          # step 4
    M = 0.5 * (M + M.T)
    lam, X = np.linalg.eigh(M)                               # step 5
    H = Z @ Qinv @ X[:, :k]                                  # step 6
    return lam[:k], H


def variant_dense(W, groups, h: int, k: int):
    """Sec. 3.2 first variant (eq. tropt_null / tracemin1 / lveig).  Returns (eigenvalues[k], H)."""
    Ln = _dense(normalized_laplacian(W))
    C = constraint_matrix(W, groups, h)
    V = nullspace_basis(C)
    Lv = V.T @ Ln @ V
    lam, Y = np.linalg.eigh(0.5 * (Lv + Lv.T))
    H = (V @ Y[:, :k]) / np.sqrt(degrees(W))[:, None]
    return lam[:k], H, lam


def projector(C: np.ndarray) -> np.ndarray:
    """P = I - C (C^T C)^{-1} C^T (eq. mv-Pw)."""
    n = C.shape[0]
    if C.shape[1] == 0:
        return np.eye(n)
    return np.eye(n) - C @ np.linalg.solve(C.T @ C, C.T)


def sfairsc_matrix(W, groups, h: int, sigma: float | None = None, normalized: bool = True, F=None):
    """The explicit L_n^sigma = P L_n P + sigma (I - P) (eq. asigma) and its sigma.

    sigma defaults to ||L_n||_1 (App. C).  normalized=False uses L and
    P = I - F (F^T F)^{-1} F^T, an extension the paper does not define.
    """
    A = _dense(normalized_laplacian(W) if normalized else laplacian(W))
    C = constraint_matrix(W, groups, h, normalized, F)
    P = projector(C)
    if sigma is None:
        sigma = sigma_one_norm(A)
    n = A.shape[0]
    As = P @ A @ P + sigma * (np.eye(n) - P)
    return 0.5 * (As + As.T), sigma


def sfairsc_dense(W, groups, h: int, k: int, sigma: float | None = None, normalized: bool = True, F=None):
    """k smallest eigenpairs of the dense L_n^sigma, H = D^{-1/2} X (Algorithm 3).

    Returns (eigenvalues[k], H[n, k], X[n, k], sigma, all eigenvalues).
    """
    As, sigma = sfairsc_matrix(W, groups, h, sigma, normalized, F)
    lam, X = np.linalg.eigh(As)
    Xk = X[:, :k]
    H = Xk / np.sqrt(degrees(W))[:, None] if normalized else Xk
    return lam[:k], H, Xk, sigma, lam
