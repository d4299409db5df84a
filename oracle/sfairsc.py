"""s-FairSC (Algorithm 3) with the matrix-free operator of Sec. 3.4, FP64.

The operator is applied only through
    L_n^sigma w = P(L_n(P w)) - sigma P w + sigma w          (Sec. 3.4 (i))
with P w = w - C z, z = argmin ||C z - w||_2 solved directly through the
Cholesky factor of C^T C                                       (eq. mv-Pw)
and sigma = ||L_n||_1                                          (App. C).
F is formed explicitly from the group labels (Lemma 2.1), so this file is an
independent check of any label-based shortcut.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse.linalg as spla

from .problem import adjacency, constraint_matrix, degrees, laplacian, normalized_laplacian, sigma_one_norm


class SFairSCOperator:
    """w -> L_n^sigma w for the graph W and group labels (eq. asigma, Sec. 3.4)."""

    def __init__(self, W, groups, h: int, sigma: float | None = None, normalized: bool = True, F=None):
        """F: a dense n x (h-1) constraint matrix in place of the group constraints (groups unused)."""
        self.W = W
        self.n = W.shape[0]
        self.h = h
        self.normalized = normalized
        self.d = degrees(W)
        if np.any(self.d <= 0):
            raise ValueError("isolated vertex (Sec. 2.1 assumes D > 0)")
        self.A = normalized_laplacian(W) if normalized else laplacian(W).tocsr()
        self.C = constraint_matrix(W, groups, h, normalized, F)
        self.chol = sla.cho_factor(self.C.T @ self.C) if h > 1 else None   # Lemma 2.1: C^T C is SPD
        self.sigma = sigma_one_norm(self.A) if sigma is None else float(sigma)

    def project(self, w: np.ndarray) -> np.ndarray:
        """P w = w - C z, z = (C^T C)^{-1} C^T w (eq. mv-Pw)."""
        if self.chol is None:
            return w.copy()
        z = sla.cho_solve(self.chol, self.C.T @ w)
        return w - self.C @ z

    def apply(self, w: np.ndarray) -> np.ndarray:
        """P(L_n(P w)) - sigma P w + sigma w (Sec. 3.4 (i)); w may be n x b."""
        w = np.asarray(w, dtype=np.float64)
        y = self.project(w)
        return self.project(self.A @ y) - self.sigma * y + self.sigma * w

    def linear_operator(self):
        return spla.LinearOperator((self.n, self.n), matvec=self.apply, matmat=self.apply, dtype=np.float64)


def operator_from_graph(g, sigma=None, normalized=True) -> SFairSCOperator:
    W = adjacency(g.row_ptr, g.col_idx, g.values)
    return SFairSCOperator(W, g.groups, g.h, sigma, normalized)


def sign_normalize(X: np.ndarray) -> np.ndarray:
    """Flip each column so its largest-magnitude entry (lowest index on ties) is positive."""
    X = np.array(X, dtype=np.float64, copy=True)
    for c in range(X.shape[1]):
        i = int(np.argmax(np.abs(X[:, c])))
        if X[i, c] < 0:
            X[:, c] = -X[:, c]
    return X


def smallest_eigenpairs(op: SFairSCOperator, k: int, tol: float = 1e-12, seed: int = 0, method: str = "eigsh"):
    """k smallest eigenpairs of L_n^sigma (Algorithm 3 step 3), ascending."""
    if method == "dense":
        n = op.n
        M = op.apply(np.eye(n))
        lam, X = np.linalg.eigh(0.5 * (M + M.T))
        return lam[:k], X[:, :k]
    if method == "lanczos":
        from .lanczos import thick_restart_lanczos

        lam, X, _ = thick_restart_lanczos(op.apply, op.n, k, tol=tol, anorm=op.sigma, seed=seed)
        return lam, X
    v0 = np.random.default_rng(seed).standard_normal(op.n)
    lam, X = spla.eigsh(op.linear_operator(), k=k, which="SA", tol=tol, v0=v0, ncv=min(op.n, max(2 * k + 1, 20)))
    order = np.argsort(lam)
    return lam[order], X[:, order]


def embed(op: SFairSCOperator, X: np.ndarray) -> np.ndarray:
    """H = D^{-1/2} X (Algorithm 3 step 4); X for the unnormalized extension."""
    X = sign_normalize(X)
    return X / np.sqrt(op.d)[:, None] if op.normalized else X


def residual_norms(op: SFairSCOperator, lam: np.ndarray, X: np.ndarray) -> np.ndarray:
    """||L_n^sigma x_i - lambda_i x_i||_2 / ||x_i||_2 for each column."""
    R = op.apply(X) - X * lam[None, :]
    return np.linalg.norm(R, axis=0) / np.linalg.norm(X, axis=0)


def sfairsc(g, k: int, sigma=None, normalized=True, tol=1e-12, method="eigsh", kmeans_seed=0, n_init=10,
            max_iter=300):
    """Algorithm 3 end to end: eigenpairs, embedding, seeded k-means labels."""
    from .kmeans import kmeans

    op = operator_from_graph(g, sigma, normalized)
    lam, X = smallest_eigenpairs(op, k, tol=tol, method=method)
    H = embed(op, X)
    labels, _, _ = kmeans(H, k, seed=kmeans_seed, n_init=n_init, max_iter=max_iter)
    return {"eigenvalues": lam, "X": X, "H": H, "labels": labels, "sigma": op.sigma, "op": op}
