"""Parameter estimation of Sec. 2.6 (energy-fraction truncation, k-means level
partitions): the oracle against closed forms and brute force, then the
library's host functions against the oracle (CPU only)."""
from __future__ import annotations

import itertools
import math

import numpy as np
import pytest

import oracle
from oracle import estimate as oest
from paper_2310_09200_b300 import bipp_ss, inputs


# ---------------------------------------------------------------- oracle pins

def test_energy_fraction_closed_forms():
    mu = [4.0, 3.0, 2.0, 1.0, -1.0]  # positive energy 10
    assert oest.energy_n_eig(mu, 0.7) == 2   # 4 + 3 = 7 >= 7
    assert oest.energy_n_eig(mu, 0.71) == 3
    assert oest.energy_n_eig(mu, 0.4) == 1
    assert oest.energy_n_eig(mu, 1.0) == 4   # the negative eigenvalue adds no energy
    assert oest.energy_n_eig([-1.0, -2.0], 0.5) == 1


def test_kmeans_dp_is_the_brute_force_optimum():
    rng = np.random.default_rng(3)
    for trial in range(20):
        n, k = int(rng.integers(4, 10)), int(rng.integers(1, 4))
        vals = rng.normal(size=n) * 10 ** rng.uniform(-2, 2, size=n)
        x, starts, cost = oest.kmeans_1d(vals, k)
        best = math.inf
        for cuts in itertools.combinations(range(1, n), k - 1):
            edges = (0,) + cuts + (n,)
            c = sum(oest._sse(x, edges[q], edges[q + 1] - 1) for q in range(k))
            best = min(best, c)
        assert cost <= best * (1 + 1e-12) + 1e-300, (trial, cost, best)
        assert starts == sorted(starts) and starts[0] == 0


def test_kmeans_separated_clusters():
    vals = [1.0, 1.1, 0.9, 5.0, 5.2, 10.0, 10.5]
    b = oest.kmeans_bounds(vals, 3)
    assert b[0] == (7.6, math.inf)           # halfway between 5.2 and 10.0
    assert b[1] == (3.05, 7.6)               # halfway between 1.1 and 5.0
    assert b[2] == (-math.inf, 3.05)


def test_quantile_bounds_closed_forms():
    # 12 values 1..12 in 4 levels: edges between the 3rd/4th, 6th/7th and 9th/10th values
    b = oest.quantile_bounds(np.arange(1.0, 13.0), 4)
    assert b == [(9.5, math.inf), (6.5, 9.5), (3.5, 6.5), (-math.inf, 3.5)]
    # q n / k = 2.5 rounds half to even (to 2): the edge falls between the 2nd and 3rd values
    assert oest.quantile_bounds([10.0, 0.0, 20.0, 30.0, 40.0], 2) == [(15.0, math.inf), (-math.inf, 15.0)]
    # one level: the whole real line; a level count equal to n puts an edge between every pair
    assert oest.quantile_bounds([3.0], 1) == [(-math.inf, math.inf)]
    assert oest.quantile_bounds([1.0, 2.0, 4.0], 3) == [(3.0, math.inf), (1.5, 3.0), (-math.inf, 1.5)]


def test_quantile_bounds_split_into_equal_counts():
    rng = np.random.default_rng(8)
    for _ in range(20):
        n, k = int(rng.integers(8, 200)), int(rng.integers(1, 8))
        vals = rng.normal(size=n) * 10 ** rng.uniform(-2, 2)
        b = oest.quantile_bounds(vals, k)
        counts = [int(np.sum((vals >= lo) & (vals < hi))) for lo, hi in b]
        assert sum(counts) == n  # distinct values: every one in exactly one half-open level
        assert max(counts) - min(counts) <= 2, counts


# ---------------------------------------------------------------- library vs oracle

@pytest.mark.parametrize("k", [1, 2, 4, 7])
def test_library_quantile_bounds_match_oracle(k):
    rng = np.random.default_rng(20 + k)
    for n in (k, k + 1, 13, 257):
        vals = rng.lognormal(size=n) * rng.choice([-1.0, 1.0], size=n)
        got = bipp_ss.quantile_level_bounds(vals, k)
        want = np.array(oest.quantile_bounds(vals, k))
        np.testing.assert_array_equal(got, want)  # same sorted values, same halving: bit for bit


def test_library_energy_matches_oracle():
    rng = np.random.default_rng(5)
    for _ in range(50):
        mu = np.sort(rng.normal(size=int(rng.integers(1, 60))) * 3 + 1)[::-1]
        f = float(rng.uniform(0.05, 1.0))
        assert bipp_ss.bipp_ss_energy_neig(mu, f) == oest.energy_n_eig(mu, f)


@pytest.mark.parametrize("k", [1, 2, 4, 6])
def test_library_kmeans_matches_oracle(k):
    rng = np.random.default_rng(10 + k)
    vals = np.concatenate([rng.normal(c, 0.3 * (1 + c / 10), size=int(rng.integers(20, 60)))
                           for c in (0.0, 4.0, 9.0, 30.0)])
    got = bipp_ss.bipp_ss_kmeans_bounds(vals, k)
    want = np.array(oest.kmeans_bounds(vals, k))
    np.testing.assert_allclose(got, want, rtol=1e-13)


def test_library_kmeans_on_pooled_oracle_eigenvalues():
    inp = inputs.make_config(0, n_t=4)
    pooled = []
    for p, V in zip(inp.st_xyz, inp.vis):
        mu, _, _ = oracle.geneig(V, oracle.gram(p, inp.wl))
        pooled.extend(mu[: inp.n_eig])
    np.testing.assert_allclose(bipp_ss.bipp_ss_kmeans_bounds(pooled, 4), np.array(oest.kmeans_bounds(pooled, 4)),
                               rtol=1e-13)


@pytest.mark.parametrize("case", ["n_level0", "too_many", "nan", "fraction", "unordered", "q_too_many", "q_nan"])
def test_library_estimation_rejects_invalid_arguments(case):
    with pytest.raises(bipp_ss.BippError) as e:
        if case == "n_level0":
            bipp_ss.bipp_ss_kmeans_bounds([1.0, 2.0], 0)
        elif case == "too_many":
            bipp_ss.bipp_ss_kmeans_bounds([1.0, 2.0], 3)
        elif case == "nan":
            bipp_ss.bipp_ss_kmeans_bounds([1.0, np.nan], 1)
        elif case == "q_too_many":
            bipp_ss.quantile_level_bounds([1.0, 2.0], 3)
        elif case == "q_nan":
            bipp_ss.quantile_level_bounds([1.0, np.inf, 3.0], 2)
        elif case == "fraction":
            bipp_ss.bipp_ss_energy_neig([2.0, 1.0], 1.5)
        else:
            bipp_ss.bipp_ss_energy_neig([1.0, 2.0], 0.5)
    assert e.value.code == bipp_ss.BIPP_ERR_INVALID_ARG
