"""Gradients of the fair problem's eigenvalues and eigenvectors with respect to the edge weights.

The eigenvalues of eq. normal-prob-fair are those of the pencil
(Z^T L Z, Z^T D Z) of Algorithm 2, where Z spans null(F^T) and does not depend
on W.  For a simple eigenvalue lambda with h = Z y, h^T D h = 1 (so H^T D H = I
as in eq. normal-prob-fair), first-order perturbation gives
d lambda = h^T (dL - lambda dD) h.  Moving w_ab = w_ba together by eps changes
L by eps (e_a - e_b)(e_a - e_b)^T and D by eps (e_a e_a^T + e_b e_b^T), so

    d lambda / d w_ab = (h_a - h_b)^2 - lambda (h_a^2 + h_b^2).

Each of the two CSR entries (a, b) and (b, a) reports half of this.  With
Gaussian weights w = exp(-r^2 / (2 s^2)), dw/ds = w r^2 / s^3 = w (-2 ln w) / s.
"""
from __future__ import annotations

import numpy as np

from .fairsc import sfairsc_dense
from .problem import adjacency


def edge_gradient(row_ptr, col_idx, lam, H) -> np.ndarray:
    """Per-CSR-entry d f / d w_e (half of the undirected derivative), f = sum lam."""
    n = len(row_ptr) - 1
    rows = np.repeat(np.arange(n), np.diff(row_ptr))
    cols = np.asarray(col_idx)
    ha, hb = H[rows], H[cols]
    per = (ha - hb) ** 2 - lam[None, :] * (ha ** 2 + hb ** 2)
    return 0.5 * per.sum(axis=1)


def bandwidth_gradient(grad_entries, values, bandwidth: float) -> float:
    """d f / d s = sum_e g_e * w_e * (-2 ln w_e) / s for w = exp(-r^2 / (2 s^2))."""
    w = np.asarray(values, dtype=np.float64)
    return float(np.sum(grad_entries * w * (-2.0 * np.log(w)) / bandwidth))


def eigsum_dense(row_ptr, col_idx, values, groups, h, k) -> float:
    W = adjacency(row_ptr, col_idx, values)
    lam, *_ = sfairsc_dense(W, groups, h, k)
    return float(lam.sum())


def edge_gradient_fd(row_ptr, col_idx, values, groups, h, k, a: int, b: int, step: float = 1e-6) -> float:
    """Central difference of f in the undirected weight w_ab = w_ba (dense solve)."""
    values = np.asarray(values, dtype=np.float64)
    n = len(row_ptr) - 1
    rows = np.repeat(np.arange(n), np.diff(row_ptr))
    sel = ((rows == a) & (np.asarray(col_idx) == b)) | ((rows == b) & (np.asarray(col_idx) == a))
    vp = values.copy(); vp[sel] += step
    vm = values.copy(); vm[sel] -= step
    return (eigsum_dense(row_ptr, col_idx, vp, groups, h, k) - eigsum_dense(row_ptr, col_idx, vm, groups, h, k)) / (2 * step)


def vector_gradient(row_ptr, col_idx, values, groups, h, k, Gbar, gbar_lam=None, F=None) -> np.ndarray:
    """Per-CSR-entry d loss / d w_e for a loss on H (upstream gradient Gbar, n x k) and optionally
    on the eigenvalues (gbar_lam, k), half of the undirected derivative per entry.

    The columns of H are the generalized eigenvectors h = Z y of (Z^T L Z) y = lambda (Z^T D Z) y
    with y^T (Z^T D Z) y = 1 (Algorithm 2; Z spans null(F^T), independent of W).  For simple
    eigenvalues first-order perturbation gives
        dh_i = sum_{j != i} h_j h_j^T (dL - lambda_i dD) h_i / (lambda_i - lambda_j) - (h_i^T dD h_i) h_i / 2,
    the sum running over every eigenpair of the pencil.  With v_i = sum_{j != i} h_j (h_j^T gbar_i)
    / (lambda_i - lambda_j) and c_i = gbar_i^T h_i, moving w_ab = w_ba by dw (dL = (e_a - e_b)(e_a - e_b)^T dw,
    dD = (e_a e_a^T + e_b e_b^T) dw) changes the loss by
        sum_i (v_ia - v_ib)(h_ia - h_ib) - lambda_i (v_ia h_ia + v_ib h_ib) - c_i (h_ia^2 + h_ib^2) / 2.
    Dense: every eigenpair from Algorithm 2's full eigendecomposition (small n only)."""
    from .fairsc import nullspace_basis
    from .problem import adjacency, degrees, fairness_constraints, laplacian

    W = adjacency(row_ptr, col_idx, values)
    L = laplacian(W).toarray()
    d = degrees(W)
    if F is None:
        _, F, _ = fairness_constraints(groups, h)
    Z = nullspace_basis(np.asarray(F, dtype=np.float64))
    K = Z.T @ L @ Z
    M = Z.T @ (d[:, None] * Z)
    mu, E = np.linalg.eigh(M)
    Mih = (E / np.sqrt(mu)) @ E.T                      # M^{-1/2}
    lam_all, Y = np.linalg.eigh(Mih @ K @ Mih)
    Hall = Z @ (Mih @ Y)                               # every generalized eigenvector, H^T D H = I
    lam = lam_all[:k]
    H = Hall[:, :k]
    Gbar = np.asarray(Gbar, dtype=np.float64)
    # the sign convention of the forward pass fixes each column (Gbar refers to it): the entry of
    # x = D^{1/2} h of largest magnitude (lowest row on ties) is positive
    for i in range(k):
        xi = H[:, i] * np.sqrt(d)
        if xi[np.argmax(np.abs(xi))] < 0:
            H[:, i] = -H[:, i]
            Hall[:, i] = H[:, i]
    V = np.zeros_like(H)
    for i in range(k):
        coef = Hall.T @ Gbar[:, i]
        den = lam[i] - lam_all
        den[i] = np.inf
        V[:, i] = Hall @ (coef / den)
    c = np.einsum("ri,ri->i", Gbar, H)
    n = len(row_ptr) - 1
    rows = np.repeat(np.arange(n), np.diff(row_ptr))
    cols = np.asarray(col_idx)
    ha, hb, va, vb = H[rows], H[cols], V[rows], V[cols]
    per = (va - vb) * (ha - hb) - lam[None, :] * (va * ha + vb * hb) - 0.5 * c[None, :] * (ha ** 2 + hb ** 2)
    if gbar_lam is not None:
        per = per + np.asarray(gbar_lam)[None, :] * ((ha - hb) ** 2 - lam[None, :] * (ha ** 2 + hb ** 2))
    return 0.5 * per.sum(axis=1), lam, H


def embedding_dense(row_ptr, col_idx, values, groups, h, k, F=None):
    """H (n x k) from the dense s-FairSC matrix for the given weights, with the sign rule of the
    embedding (largest-magnitude entry of x = D^{1/2} h positive)."""
    from .problem import degrees

    W = adjacency(row_ptr, col_idx, values)
    lam, H = sfairsc_dense(W, groups, h, k, F=F)[:2]
    sd = np.sqrt(degrees(W))
    for i in range(k):
        xi = H[:, i] * sd
        if xi[np.argmax(np.abs(xi))] < 0:
            H[:, i] = -H[:, i]
    return lam, H
