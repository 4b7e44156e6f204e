"""Pins for the oracle's single- and double-jump maps (Sec. 4, Fig. 4).

The maps are checked entry by entry against a dictionary from brute-force
enumeration (no call to Algorithm 1), and their sizes against the paper's
Fig. 4 counts and a closed form.
"""
import math
import os

import numpy as np
import pytest

import oracle
from tests.test_oracle_hashing import brute_force_configs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def index_dict(N, M):
    return {c: i for i, c in enumerate(brute_force_configs(N, M))}


@pytest.mark.parametrize("N,M", [(1, 3), (3, 3), (4, 5), (5, 4), (2, 6), (6, 2)])
def test_single_jump_map_by_enumeration(N, M):
    confs = brute_force_configs(N, M)
    d = index_dict(N, M)
    J1 = oracle.single_jump_map(N, M)
    for g, c in enumerate(confs):
        for k in range(M):
            for l in range(M):
                if c[k] == 0:
                    assert J1[g, k, l] == -1
                    continue
                t = list(c); t[k] -= 1; t[l] += 1
                assert J1[g, k, l] == d[tuple(t)]


@pytest.mark.parametrize("N,M", [(2, 3), (3, 3), (4, 5), (5, 4), (3, 6)])
def test_double_jump_map_by_enumeration(N, M):
    confs = brute_force_configs(N, M)
    d = index_dict(N, M)
    off, data = oracle.double_jump_map(N, M)
    for g, c in enumerate(confs):
        pos = off[g]
        for k in range(M):
            for q in range(k, M):
                ok = (c[k] >= 2) if k == q else (c[k] >= 1 and c[q] >= 1)
                if not ok:
                    continue
                for s in range(M):
                    for l in range(M):
                        t = list(c); t[k] -= 1; t[q] -= 1; t[s] += 1; t[l] += 1
                        assert data[pos + s * M + l] == d[tuple(t)]
                pos += M * M
        assert pos == off[g + 1]


@pytest.mark.parametrize("N,M", [(2, 3), (4, 5), (7, 4), (10, 3), (3, 8)])
def test_double_jump_map_size_closed_form(N, M):
    # Configurations with a removable pair {k <= q} biject with H(N-2, M), so
    # the rows hold M(M+1)/2 * N_c(N-2, M) strides of M^2 entries in total.
    off, _ = oracle.double_jump_map(N, M)
    P = M * (M + 1) // 2
    assert off[-1] == M * M * P * math.comb(N - 2 + M - 1, M - 1)


def test_fig4_counts():
    with open(os.path.join(GOLDEN, "fig4_double_jump_example.txt")) as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    for N, M, occ, pairs, real, naive, skips in rows:
        N, M = int(N), int(M)
        occ = [int(x) for x in occ.split(",")]
        assert oracle.removal_count(M, occ) == int(pairs)
        assert int(pairs) * M * M == int(real)
        assert M ** 4 == int(naive)
        # Position of the stride that removes the two highest-placed particles.
        parts = sorted(o for o, c in enumerate(occ) for _ in range(c))
        last_pair = (parts[-2], parts[-1])
        g = oracle.rank(N, M, occ)
        off, data = oracle.double_jump_map(N, M)
        strides = [(k, q) for k in range(M) for q in range(k, M)
                   if ((occ[k] >= 2) if k == q else (occ[k] >= 1 and occ[q] >= 1))]
        assert strides.index(last_pair) == int(skips)
        # the entry "put both back where they were" returns to gamma itself
        base = off[g] + int(skips) * M * M
        assert data[base + last_pair[0] * M + last_pair[1]] == g
        assert off[g + 1] - off[g] == int(real)
