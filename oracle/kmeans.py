"""Seeded k-means on the rows of H (Algorithm 3 step 4), written plainly.

The paper only says "apply k-means clustering to the rows of H"; the
unstated details are fixed here so that any implementation can reproduce the
labels exactly:

* data: X = float32(H); all distances are squared Euclidean distances
  computed in float32 as  acc = 0; for c in 0..d-1: t = x_c - m_c; acc = acc + t*t
  (one rounding per operation, no fused multiply-add, dimension order);
* randomness: splitmix64 (Steele, Lea and Flood, 2014) used as a
  counter-based generator: draw q of seed s is mix(s + (q + 1) * 0x9E3779B97F4A7C15),
  which is the q-th output of the sequential generator started at state s;
  replicate r uses draws q = r*k + t, t = 0..k-1;
* seeding: k-means++ (Arthur and Vassilvitskii, 2007).  Center 0 is row
  floor(r64 * n / 2^64).  Center t > 0 is drawn with probability proportional
  to D^2 (distance to the nearest chosen center), with the D^2 values
  quantised to integers q_i = floor(D2_i * 2^S), S = 62 - bitlen(n) - e, where
  max D2 = f * 2^e, 1/2 <= f < 1; the pick is the first row whose integer
  prefix sum exceeds floor(r64 * total / 2^64);
* Lloyd: assign every row to the nearest float32(centroid) (lowest index on
  ties); stop when no label changes or after max_iter assignments; a centroid
  is the mean of its rows, summed exactly in the same fixed point
  (scale from max |X|) and divided once in float64; an empty cluster takes the
  row farthest from its own centroid (lowest index on ties), in cluster order;
* replicates: the one with the smallest inertia (sum of float32 distances,
  quantised like the D^2 weights) wins, lowest replicate index on ties.
"""
from __future__ import annotations

import math

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
MASK64 = (1 << 64) - 1


def splitmix64_mix(z: int) -> int:
    z &= MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def splitmix64_sequence(seed: int, count: int):
    """The sequential generator: state += gamma; output mix(state)."""
    state = seed & MASK64
    out = []
    for _ in range(count):
        state = (state + GAMMA) & MASK64
        out.append(splitmix64_mix(state))
    return out


def splitmix64_draw(seed: int, q: int) -> int:
    """Counter-based access: the q-th (0-based) output for seed."""
    return splitmix64_mix((seed + (q + 1) * GAMMA) & MASK64)


def dist2_f32(X32: np.ndarray, m32: np.ndarray) -> np.ndarray:
    """Squared distances of all rows of X32 to one float32 center, dimension order, no FMA."""
    acc = np.zeros(X32.shape[0], dtype=np.float32)
    for c in range(X32.shape[1]):
        t = X32[:, c] - m32[c]
        acc = acc + t * t
    return acc


def _scale_shift(maxval: float, n: int) -> int:
    """S such that floor(v * 2^S) < 2^(62 - bitlen(n)) for 0 <= v <= maxval."""
    _, e = math.frexp(float(maxval))
    return 62 - int(n).bit_length() - e


def quantise(v: np.ndarray, shift: int) -> np.ndarray:
    """Truncate v * 2^shift toward zero to int64 (exact scaling in float64)."""
    return np.trunc(np.ldexp(v.astype(np.float64), shift)).astype(np.int64)


def quantised_total(v32: np.ndarray) -> float:
    """Sum of nonnegative float32 values through the exact fixed point, as float64."""
    maxv = float(v32.max()) if v32.size else 0.0
    if maxv == 0.0:
        return 0.0
    s = _scale_shift(maxv, v32.size)
    return math.ldexp(float(int(quantise(v32, s).sum())), -s)


def kmeanspp(X32: np.ndarray, k: int, seed: int, replicate: int = 0) -> np.ndarray:
    """Indices of the k k-means++ seeds for one replicate."""
    n = X32.shape[0]
    q0 = replicate * k
    idx = [(splitmix64_draw(seed, q0) * n) >> 64]
    D2 = dist2_f32(X32, X32[idx[0]])
    for t in range(1, k):
        r64 = splitmix64_draw(seed, q0 + t)
        maxv = float(D2.max())
        if maxv == 0.0:
            nxt = (r64 * n) >> 64
        else:
            s = _scale_shift(maxv, n)
            w = quantise(D2, s)
            cum = np.cumsum(w)
            total = int(cum[-1])
            target = (r64 * total) >> 64
            nxt = int(np.searchsorted(cum, target, side="right"))
        idx.append(nxt)
        D2 = np.minimum(D2, dist2_f32(X32, X32[nxt]))
    return np.array(idx, dtype=np.int64)


def assign(X32: np.ndarray, M32: np.ndarray):
    """Nearest centroid per row (lowest index on ties) and its float32 distance."""
    best = dist2_f32(X32, M32[0])
    lab = np.zeros(X32.shape[0], dtype=np.int32)
    for c in range(1, M32.shape[0]):
        d = dist2_f32(X32, M32[c])
        better = d < best
        lab[better] = c
        best = np.where(better, d, best)
    return lab, best


def update(X32: np.ndarray, labels: np.ndarray, k: int, M32_used: np.ndarray, dist_used: np.ndarray,
           xshift: int) -> np.ndarray:
    """Exact fixed-point means; empty clusters take the farthest rows."""
    n, d = X32.shape
    Q = quantise(X32, xshift)
    counts = np.bincount(labels, minlength=k)
    mu = np.zeros((k, d))
    for c in range(k):
        if counts[c] > 0:
            sums = Q[labels == c].sum(axis=0)          # exact int64 sums
            mu[c] = np.array([math.ldexp(float(int(v)), -xshift) for v in sums]) / counts[c]
    empty = np.nonzero(counts == 0)[0]
    if empty.size:
        far = dist_used.astype(np.float32).copy()
        taken = np.zeros(n, dtype=bool)
        for c in empty:
            cand = np.where(taken, np.float32(-1.0), far)
            i = int(np.argmax(cand))
            taken[i] = True
            mu[c] = X32[i].astype(np.float64)
    return mu


def lloyd(X32: np.ndarray, centers: np.ndarray, max_iter: int):
    """Lloyd iterations from float64 centers; returns (labels, mu, iterations)."""
    n = X32.shape[0]
    k = centers.shape[0]
    xmax = float(np.max(np.abs(X32))) if X32.size else 0.0
    xshift = _scale_shift(xmax, n) if xmax > 0 else 0
    mu = centers.astype(np.float64).copy()
    labels = None
    it = 0
    for it in range(max_iter):
        M32 = mu.astype(np.float32)
        new, dist = assign(X32, M32)
        if labels is not None and np.array_equal(new, labels):
            break
        labels = new
        mu = update(X32, labels, k, M32, dist, xshift)
    return labels, mu, it + 1


def inertia(X32: np.ndarray, labels: np.ndarray, mu: np.ndarray) -> float:
    M32 = mu.astype(np.float32)
    dist = np.zeros(X32.shape[0], dtype=np.float32)
    for c in range(M32.shape[0]):
        sel = labels == c
        if sel.any():
            dist[sel] = dist2_f32(X32[sel], M32[c])
    return quantised_total(dist)


def kmeans(H: np.ndarray, k: int, seed: int = 0, n_init: int = 10, max_iter: int = 300):
    """Best-of-n_init seeded k-means on the rows of H.  Returns (labels, mu, inertia)."""
    X32 = np.ascontiguousarray(np.asarray(H, dtype=np.float64).astype(np.float32))
    best = None
    for r in range(n_init):
        seeds = kmeanspp(X32, k, seed, r)
        labels, mu, _ = lloyd(X32, X32[seeds].astype(np.float64), max_iter)
        val = inertia(X32, labels, mu)
        if best is None or val < best[2]:
            best = (labels, mu, val)
    return best
