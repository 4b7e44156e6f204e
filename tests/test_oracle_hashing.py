"""Pins for the oracle's hashing (Eq. nc, Eq. TotalCost, Algorithms 1 and 2).

Each check compares the oracle with something other than itself: the paper's
worked example (Fig. 2), brute-force enumeration of all configurations, and
the binomial counts of the standard library.
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def brute_force_configs(N, M):
    """All occupation vectors with sum N, in ascending lexicographic order of
    the reversed vector (n_{M-1}, ..., n_0)."""
    out = [c for c in itertools.product(range(N + 1), repeat=M) if sum(c) == N]
    out.sort(key=lambda c: tuple(reversed(c)))
    return out


def test_fig2_worked_example():
    with open(os.path.join(GOLDEN, "fig2_hash_example.txt")) as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    for N, M, occ, idx, terms in rows:
        N, M, idx = int(N), int(M), int(idx)
        occ = [int(x) for x in occ.split(",")]
        assert oracle.rank(N, M, occ) == idx
        assert list(oracle.unrank(N, M, idx)) == occ
        # The caption's cost terms, each N_c(n, m) = C(n+m-1, m-1), add up to the index.
        total = 0
        for t in terms.split(";"):
            n, m = (int(x) for x in t.split(":"))
            assert oracle.nc(n, m) == math.comb(n + m - 1, m - 1)
            total += oracle.nc(n, m)
        assert total == idx


@pytest.mark.parametrize("N", range(0, 9))
@pytest.mark.parametrize("M", range(1, 8))
def test_count_matches_enumeration(N, M):
    assert oracle.nc(N, M) == len(brute_force_configs(N, M))


def test_count_conventions_and_large_values():
    assert oracle.nc(7, 0) == 0                     # N_c(n, 0) = 0 (Eq. TotalCost)
    assert oracle.nc(0, 4) == 1                     # no particles: one empty configuration
    assert oracle.nc(100, 6) == 96_560_646
    assert oracle.nc(30, 10) == 211_915_132
    assert oracle.nc(20, 8) == 888_030
    assert oracle.nc(5, 5) == 126
    assert oracle.nc(1000, 3) == math.comb(1002, 2)
    assert oracle.nc(10 ** 6, 40) == -1             # overflow is reported, not wrapped


@pytest.mark.parametrize("N,M", [(1, 1), (4, 1), (1, 5), (3, 5), (5, 5), (6, 4), (8, 3), (4, 7), (2, 9)])
def test_rank_is_brute_force_position(N, M):
    confs = brute_force_configs(N, M)
    occ = np.array(confs, dtype=np.int32)
    idx = oracle.rank_batch(N, M, occ)
    assert np.array_equal(idx, np.arange(len(confs)))
    back = oracle.unrank_batch(N, M, np.arange(len(confs)))
    assert np.array_equal(back, occ)


def test_rank_extremes_large_space():
    # index 0 holds every particle in orbital 0; the last index holds them in M-1.
    for N, M in [(100, 6), (30, 10), (200, 12)]:
        first = np.zeros(M, dtype=np.int32); first[0] = N
        last = np.zeros(M, dtype=np.int32); last[-1] = N
        n = math.comb(N + M - 1, M - 1)
        assert oracle.rank(N, M, first) == 0
        assert oracle.rank(N, M, last) == n - 1
        assert np.array_equal(oracle.unrank(N, M, n - 1), last)


def test_round_trip_sampled_large_space():
    rng = np.random.default_rng(7)
    N, M = 100, 6
    n = math.comb(N + M - 1, M - 1)
    idx = rng.integers(0, n, size=2000)
    occ = oracle.unrank_batch(N, M, idx)
    assert np.all(occ.sum(axis=1) == N) and np.all(occ >= 0)
    assert np.array_equal(oracle.rank_batch(N, M, occ), idx)
    # Order check against the reversed-lexicographic characterisation.
    order = np.argsort(idx)
    keys = [tuple(reversed(o)) for o in occ[order]]
    assert all(a < b for a, b in zip(keys, keys[1:]) if a != b)
