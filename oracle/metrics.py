"""Evaluation metrics of Sec. 4: error rate (eq. err) and balance (eq. bal, eq. avebal)."""
from __future__ import annotations

import numpy as np
from scipy.optimize import linear_sum_assignment


def indicator(labels, k: int) -> np.ndarray:
    """Cluster indicator matrix H in {0,1}^{n x k} (eq. H)."""
    labels = np.asarray(labels)
    H = np.zeros((labels.size, k))
    H[np.arange(labels.size), labels] = 1.0
    return H


def error_rate(computed, truth, k: int) -> float:
    """Err = (1/n) min over permutations J of ||H_hat J - H||_F^2 (eq. err).

    ||H_hat J - H||_F^2 = 2 * (number of rows whose permuted label differs),
    so the minimising J is the assignment maximising the label agreement.
    """
    computed = np.asarray(computed)
    truth = np.asarray(truth)
    n = truth.size
    conf = np.zeros((k, k))
    np.add.at(conf, (computed, truth), 1.0)
    r, c = linear_sum_assignment(-conf)
    agree = conf[r, c].sum()
    return 2.0 * (n - agree) / n


def misclustered_fraction(computed, truth, k: int) -> float:
    """Fraction of rows whose best-permuted label differs from the truth."""
    return 0.5 * error_rate(computed, truth, k)


def group_cluster_counts(labels, groups, k: int, h: int) -> np.ndarray:
    """k x h matrix of |V_s cap C_l| (rows: clusters), i.e. M^T of eq. mz."""
    M = np.zeros((k, h), dtype=np.int64)
    np.add.at(M, (np.asarray(labels), np.asarray(groups)), 1)
    return M


def balance(labels, groups, k: int, h: int) -> np.ndarray:
    """Balance(C_l) = min over s != s' of |V_s cap C_l| / |V_s' cap C_l| (eq. bal)."""
    M = group_cluster_counts(labels, groups, k, h).astype(np.float64)
    out = np.zeros(k)
    for l in range(k):
        row = M[l]
        if h < 2 or row.sum() == 0:
            out[l] = 1.0 if h < 2 else 0.0
            continue
        if np.any(row == 0):
            out[l] = 0.0
            continue
        out[l] = row.min() / row.max()
    return out


def average_balance(labels, groups, k: int, h: int) -> float:
    """Average_Balance = (1/k) sum_l Balance(C_l) (eq. avebal)."""
    return float(balance(labels, groups, k, h).mean())


def balance_multiset(labels, groups, k: int, h: int):
    """Rows of the cluster x group count matrix, sorted: equal iff equal up to label permutation."""
    M = group_cluster_counts(labels, groups, k, h)
    return sorted(map(tuple, M.tolist()))
