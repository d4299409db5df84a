"""Gradient of f(W) = sum of the k smallest eigenvalues of the fair problem.

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
