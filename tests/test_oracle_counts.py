"""Pins for ``oracle.column_terms``: the number of operator strings of
Eqs. noninteracting and interacting with a nonzero coefficient that do not
annihilate one configuration |n> (before equal targets are merged).

The references are counting arguments, not the oracle's own string walk:

* a string a^dag_k a_l survives on |n> exactly when n_l >= 1, and
  a^dag_k a^dag_q a_s a_l survives exactly when n_l >= 1 and
  n_s - delta_sl >= 1 (creation operators never annihilate), so the count of a
  column is a sum of indicator functions of its occupations;
* summed over the whole basis, the configurations with n_l >= 1 are in
  bijection with H(N-1, M) (remove one particle from l), and those that allow
  the ordered removal (s, l) with H(N-2, M), so dense h and W give
  M^2 N_c(N-1, M) + M^4 N_c(N-2, M) strings in all (Eq. nc).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2005_13679_gb300 import inputs
from tests.test_oracle_hashing import brute_force_configs


def nc(n, m):
    return math.comb(n + m - 1, m - 1) if n >= 0 else 0


def survivors(n, h, W):
    M = len(n)
    one = sum(1 for k in range(M) for l in range(M) if h[k, l] != 0 and n[l] >= 1)
    two = 0
    if W is not None:
        for k in range(M):
            for q in range(M):
                for s in range(M):
                    for l in range(M):
                        if W[k, q, s, l] != 0 and n[l] >= 1 and n[s] - (s == l) >= 1:
                            two += 1
    return one + two


@pytest.mark.parametrize("N,M", [(1, 3), (2, 2), (3, 4), (4, 3), (5, 5)])
def test_column_terms_dense_operator(N, M):
    h, W = inputs.random_hermitian_hw(M, 31 + N)
    configs = brute_force_configs(N, M)
    total = 0
    for gamma, n in enumerate(configs):
        c = oracle.column_terms(N, M, h, W, gamma)
        assert c == survivors(n, h, W)
        total += c
    assert total == M * M * nc(N - 1, M) + M ** 4 * nc(N - 2, M)


@pytest.mark.parametrize("N,M", [(3, 5), (5, 5)])
def test_column_terms_lieb_liniger(N, M):
    # sparse pattern: diagonal h, W nonzero only when momentum is conserved
    h, W = inputs.lieb_liniger_hw(M, 1.0)
    configs = brute_force_configs(N, M)
    for gamma, n in enumerate(configs):
        assert oracle.column_terms(N, M, h, W, gamma) == survivors(n, h, W)


def test_column_terms_one_body_and_empty():
    M = 4
    h = np.zeros((M, M), dtype=np.complex128)
    h[0, 1] = h[1, 0] = 1.0
    h[2, 2] = 0.5
    for gamma, n in enumerate(brute_force_configs(3, M)):
        expect = (n[1] >= 1) + (n[0] >= 1) + (n[2] >= 1)
        assert oracle.column_terms(3, M, h, None, gamma) == expect
    # all-zero operator: no string survives
    Z = np.zeros((M, M), dtype=np.complex128)
    assert oracle.column_terms(3, M, Z, np.zeros((M,) * 4, dtype=np.complex128), 5) == 0
