"""Plain thick-restart Lanczos with full reorthogonalisation (FP64).

A textbook stand-in for the implicitly restarted Lanczos of ARPACK / `eigs`
that the paper calls for its k smallest eigenpairs (Sec. 3.4 (i)); thick
restart with exact shifts is mathematically equivalent to implicit restart.
Each step orthogonalises A v_j against all basis vectors twice (classical
Gram-Schmidt, twice), the projected matrix T = V^T A V is kept in full, and
at a restart the K best Ritz vectors plus the residual direction become the
new basis.  Convergence: |beta_m y_{m,i}| <= tol * anorm for the k smallest.
"""
from __future__ import annotations

import numpy as np


def thick_restart_lanczos(apply, n: int, k: int, m: int | None = None, tol: float = 1e-12, anorm: float = 1.0,
                          seed: int = 0, max_restarts: int = 500, v0=None, on_cycle=None):
    """k smallest eigenpairs of the symmetric operator `apply` (ascending).

    v0: start vector (default: a seeded Gaussian vector).
    on_cycle: called as on_cycle(cycle, matvecs) after each restart cycle's
    Lanczos steps (a timing hook for the benchmark; it changes nothing).
    Returns (eigenvalues[k], X[n, k], info dict).
    """
    if m is None:
        m = max(2 * k, 20)
    m = min(m, n)
    if k >= m:
        m = min(n, k + 1)
    V = np.zeros((n, m + 1))
    T = np.zeros((m + 1, m + 1))
    v = np.random.default_rng(seed).standard_normal(n) if v0 is None else np.asarray(v0, dtype=np.float64)
    V[:, 0] = v / np.linalg.norm(v)
    j0 = 0
    matvecs = 0
    for restart in range(max_restarts):
        beta = 0.0
        for j in range(j0, m):
            w = apply(V[:, j])
            matvecs += 1
            for _ in range(2):
                c = V[:, : j + 1].T @ w
                w -= V[:, : j + 1] @ c
                T[: j + 1, j] += c
            beta = np.linalg.norm(w)
            T[j + 1, j] = beta
            if beta <= 1e-300:
                w = np.random.default_rng(seed + j + 1).standard_normal(n)
                for _ in range(2):
                    w -= V[:, : j + 1] @ (V[:, : j + 1].T @ w)
                beta_dir = np.linalg.norm(w)
                V[:, j + 1] = w / beta_dir
            else:
                V[:, j + 1] = w / beta
        if on_cycle is not None:
            on_cycle(restart, matvecs)
        Tm = np.triu(T[:m, :m]) + np.triu(T[:m, :m], 1).T
        theta, Y = np.linalg.eigh(Tm)
        resid = np.abs(beta * Y[m - 1, :])
        if np.all(resid[:k] <= tol * anorm) or m == n:
            X = V[:, :m] @ Y[:, :k]
            return theta[:k], X, {"restarts": restart, "matvecs": matvecs, "ritz_resid": resid[:k]}
        K = min(m - 1, k + (m - k) // 2)
        V[:, :K] = V[:, :m] @ Y[:, :K]
        V[:, K] = V[:, m]
        T[:] = 0.0
        T[np.arange(K), np.arange(K)] = theta[:K]
        T[K, :K] = beta * Y[m - 1, :K]
        j0 = K
    X = V[:, :m] @ Y[:, :k]
    return theta[:k], X, {"restarts": max_restarts, "matvecs": matvecs, "ritz_resid": resid[:k], "converged": False}
