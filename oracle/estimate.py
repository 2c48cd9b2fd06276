"""Parameter estimation of Sec. 2.6 ("Energy Levels & Partitioning"), written
plainly: TEST INFRASTRUCTURE ONLY (the tests and the benchmark's CPU baseline
may use it; the library never does).

- energy_n_eig: truncation to the least number of leading eigenvectors whose
  eigenvalues hold a given share of the energy (energy = sum of the positive
  eigenvalues).
- quantile_bounds: the equal-count partition used by the benchmark's
  pre-pass (levels split at the eigenvalue quantiles, each inner edge halfway
  between the two pooled values it separates).
- kmeans_1d / kmeans_bounds: k-means clustering of eigenvalues into level
  partitions. In one dimension the optimal clusters of sorted values are
  contiguous runs; the least within-cluster sum of squares is found by the
  textbook dynamic programme over (clusters, last index), O(k n^2), ties to the
  earliest start. Level bounds: level 0 is the highest cluster, inner edges
  halfway between neighbouring clusters, outer edges -inf / +inf.
"""
from __future__ import annotations

import math


def energy_n_eig(mu_desc, fraction):
    mu = [float(m) for m in mu_desc]
    total = sum(max(m, 0.0) for m in mu)
    acc = max(mu[0], 0.0)
    k = 1
    while k < len(mu) and acc < fraction * total:
        acc += max(mu[k], 0.0)
        k += 1
    return k


def _sse(x, i, j):
    seg = x[i:j + 1]
    m = sum(seg) / len(seg)
    return sum((v - m) ** 2 for v in seg)


def kmeans_1d(values, k):
    """Returns (sorted values, first index of each of the k clusters, cost)."""
    x = sorted(float(v) for v in values)
    n = len(x)
    inf = math.inf
    D = [[inf] * n for _ in range(k)]
    B = [[0] * n for _ in range(k)]
    for j in range(n):
        D[0][j] = _sse(x, 0, j)
    for c in range(1, k):
        for j in range(c, n):
            best, arg = inf, c
            for i in range(c, j + 1):
                v = D[c - 1][i - 1] + _sse(x, i, j)
                if v < best:
                    best, arg = v, i
            D[c][j], B[c][j] = best, arg
    starts = [0] * k
    j = n - 1
    for c in range(k - 1, -1, -1):
        starts[c] = 0 if c == 0 else B[c][j]
        j = starts[c] - 1
    return x, starts, D[k - 1][n - 1]


def kmeans_bounds(values, k):
    x, starts, _ = kmeans_1d(values, k)
    out = []
    for lev in range(k):
        c = k - 1 - lev
        lo = -math.inf if c == 0 else 0.5 * (x[starts[c] - 1] + x[starts[c]])
        hi = math.inf if c == k - 1 else 0.5 * (x[starts[c + 1] - 1] + x[starts[c + 1]])
        out.append((lo, hi))
    return out


def quantile_bounds(values, k):
    """Inner edge q (1 <= q < k) halfway between sorted values m-1 and m,
    m = round(q n / k) (half to even) clamped to [1, n-1]; outer edges -inf and
    +inf; returns k (lo, hi) pairs, level 0 holding the largest values."""
    x = sorted(float(v) for v in values)
    n = len(x)
    edges = []
    for q in range(1, k):
        m = min(max(int(round(q * n / k)), 1), n - 1)
        edges.append(0.5 * (x[m - 1] + x[m]))
    edges.sort()
    lows = [-math.inf] + edges
    highs = edges + [math.inf]
    return [(lows[c], highs[c]) for c in range(k - 1, -1, -1)]
