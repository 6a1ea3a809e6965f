"""Downstream agreement of two distance matrices of the same samples: the
paper validates its FP32 mode by the statistics a user computes from the
matrix (Sec. 4: a Mantel test between the FP32 and FP64 results), so these
helpers compare the mixed-precision matrix with the FP64 one the same way.

Host-side numpy on condensed (upper-triangle, row-major) vectors; nothing
here is on the compute path.

- ``mantel``: Pearson correlation of the two condensed vectors (the Mantel
  statistic) and a one-sided permutation p-value from relabelling the
  samples of one matrix.
- ``pcoa``: principal coordinates (classical multidimensional scaling) of a
  distance matrix: eigenvectors of the double-centred -D^2 / 2, scaled by the
  square roots of their eigenvalues.
- ``procrustes``: disparity (sum of squared differences, both sides centred
  and scaled to unit norm) after the best orthogonal alignment of one
  coordinate set onto the other.
"""
from __future__ import annotations

import numpy as np

__all__ = ["square", "mantel", "pcoa", "procrustes"]


def _n_of(m: int) -> int:
    n = int(round((1 + np.sqrt(1 + 8 * m)) / 2))
    if n * (n - 1) // 2 != m:
        raise ValueError(f"{m} is not a condensed length n(n-1)/2")
    return n


def square(condensed) -> np.ndarray:
    """Symmetric n x n matrix with zero diagonal from a condensed vector."""
    c = np.asarray(condensed, dtype=np.float64)
    n = _n_of(c.size)
    d = np.zeros((n, n))
    i, j = np.triu_indices(n, 1)
    d[i, j] = c
    d[j, i] = c
    return d


def mantel(a, b, permutations: int = 99, seed: int = 0):
    """(r, p): Pearson r between the condensed vectors a and b, and the
    fraction of sample relabellings of b (plus the identity) whose r is at
    least the observed one."""
    x = np.asarray(a, dtype=np.float64)
    y = np.asarray(b, dtype=np.float64)
    if x.shape != y.shape:
        raise ValueError("condensed vectors of different lengths")

    def pearson(u, v):
        u = u - u.mean()
        v = v - v.mean()
        den = np.sqrt((u * u).sum() * (v * v).sum())
        return float((u * v).sum() / den) if den > 0 else 0.0

    r = pearson(x, y)
    if permutations <= 0:
        return r, None
    n = _n_of(x.size)
    yb = square(y)
    iu, ju = np.triu_indices(n, 1)
    rng = np.random.default_rng(seed)
    hits = 1
    for _ in range(permutations):
        p = rng.permutation(n)
        if pearson(x, yb[p][:, p][iu, ju]) >= r:
            hits += 1
    return r, hits / (permutations + 1)


def pcoa(condensed, k: int = 10) -> tuple[np.ndarray, np.ndarray]:
    """(coordinates n x k', eigenvalues k') of the k largest eigenvalues of
    the double-centred matrix -D^2 / 2 that are positive (above 1e-10 of the
    largest; smaller ones are rounding of zero)."""
    d = square(condensed)
    a = -0.5 * d * d
    a -= a.mean(axis=0, keepdims=True)
    a -= a.mean(axis=1, keepdims=True)
    w, v = np.linalg.eigh(a)
    order = np.argsort(w)[::-1][:k]
    w = w[order]
    v = v[:, order]
    keep = w > (w[0] * 1e-10 if w.size and w[0] > 0 else 0.0)
    coords = v[:, keep] * np.sqrt(w[keep])
    return coords, w[keep]


def procrustes(x, y) -> float:
    """Disparity of y aligned onto x: both centred and scaled to unit
    Frobenius norm, y rotated / reflected by the orthogonal matrix that
    minimises the sum of squared differences (from the SVD of x^T y)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    k = min(x.shape[1], y.shape[1])
    x = x[:, :k] - x[:, :k].mean(axis=0)
    y = y[:, :k] - y[:, :k].mean(axis=0)
    nx, ny = np.linalg.norm(x), np.linalg.norm(y)
    if nx == 0 or ny == 0:
        return 0.0 if nx == ny else 1.0
    x /= nx
    y /= ny
    u, s, vt = np.linalg.svd(x.T @ y)
    rot = (u @ vt).T
    return float(((x - y @ rot) ** 2).sum())
