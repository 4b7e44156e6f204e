"""Pins of the oracle's fixed-weight sectors (sum_i i n_i = Q; total momentum
for the plane-wave orbitals of Sec. 6) against facts that do not come from the
oracle's own sector code:

* sector sizes are the coefficients of the Gaussian binomial coefficient
  [N + M - 1 choose N]_q (partitions of Q into at most N parts no larger than
  M - 1), computed here from its product formula in exact integer arithmetic;
* membership and order against brute-force enumeration of occupation vectors,
  ordered by the reversed vector (the order Algorithm 1 induces);
* the restricted operator: a weight-conserving H maps a sector into itself,
  and the spectra of the dense sector blocks together are the spectrum of the
  dense full H; the Lieb-Liniger ground state lies in the zero-momentum sector.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_2005_13679_gb300 import inputs


def gaussian_binomial_coeffs(n, k):
    """Coefficients of [n choose k]_q = prod_{i=1..k} (1 - q^(n-k+i)) / (1 - q^i)."""
    num = [1]
    for i in range(1, k + 1):
        f = [0] * (n - k + i + 1)
        f[0], f[-1] = 1, -1
        num = _mul(num, f)
    for i in range(1, k + 1):
        num = _div(num, [1] + [0] * (i - 1) + [-1])
    return num


def _mul(a, b):
    out = [0] * (len(a) + len(b) - 1)
    for i, x in enumerate(a):
        for j, y in enumerate(b):
            out[i + j] += x * y
    return out


def _div(a, b):
    """Exact division of integer polynomials (b monic in its constant term)."""
    a = list(a)
    q = [0] * (len(a) - len(b) + 1)
    for i in range(len(q)):
        c = a[i] // b[0]
        q[i] = c
        for j, y in enumerate(b):
            a[i + j] -= c * y
    assert all(x == 0 for x in a), "inexact division"
    return q


def brute_sector(N, M, Q):
    occs = [c for c in itertools.product(range(N + 1), repeat=M)
            if sum(c) == N and sum(i * x for i, x in enumerate(c)) == Q]
    return sorted(occs, key=lambda c: tuple(reversed(c)))


@pytest.mark.parametrize("N,M", [(1, 1), (4, 1), (3, 4), (5, 5), (6, 4), (4, 7), (2, 9)])
def test_sector_sizes_are_gaussian_binomial_coefficients(N, M):
    coeffs = gaussian_binomial_coeffs(N + M - 1, N)
    assert len(coeffs) == N * (M - 1) + 1
    assert sum(coeffs) == oracle.nc(N, M)
    for Q, c in enumerate(coeffs):
        assert len(oracle.sector_indices(N, M, Q)) == c
    assert len(oracle.sector_indices(N, M, N * (M - 1) + 1)) == 0


@pytest.mark.parametrize("N,M,Q", [(5, 5, 10), (4, 6, 7), (6, 4, 0), (6, 4, 18), (3, 7, 9), (4, 1, 0)])
def test_sector_members_and_order_by_enumeration(N, M, Q):
    idx = oracle.sector_indices(N, M, Q)
    occ = oracle.unrank_batch(N, M, idx)
    assert np.all(np.diff(idx) > 0)
    assert [tuple(o) for o in occ] == brute_sector(N, M, Q)


@pytest.mark.parametrize("N,M,kind", [(4, 5, "ll"), (5, 4, "ll"), (4, 4, "wc"), (3, 6, "wc")])
def test_weight_conserving_operator_stays_in_sector(N, M, kind):
    h, W = inputs.lieb_liniger_hw(M, 0.7) if kind == "ll" else inputs.weight_conserving_hw(M, 3)
    rng = np.random.default_rng(5)
    for Q in range(0, N * (M - 1) + 1, 3):
        idx = oracle.sector_indices(N, M, Q)
        C = np.zeros(oracle.nc(N, M), dtype=np.complex128)
        C[idx] = rng.standard_normal(len(idx)) + 1j * rng.standard_normal(len(idx))
        out = oracle.apply_push(N, M, h, W, C)
        mask = np.ones(len(C), bool)
        mask[idx] = False
        assert np.all(out[mask] == 0)
        np.testing.assert_allclose(oracle.sector_apply(N, M, Q, h, W, C[idx]), out[idx], rtol=0, atol=0)


@pytest.mark.parametrize("N,M,kind", [(4, 4, "ll"), (3, 5, "wc"), (5, 3, "ll")])
def test_sector_spectra_make_up_the_full_spectrum(N, M, kind):
    h, W = inputs.lieb_liniger_hw(M, 1.3) if kind == "ll" else inputs.weight_conserving_hw(M, 8)
    full = np.linalg.eigvalsh(oracle.dense_hamiltonian(N, M, h, W))
    parts = []
    for Q in range(N * (M - 1) + 1):
        n = len(oracle.sector_indices(N, M, Q))
        if n == 0:
            continue
        Hs = np.stack([oracle.sector_apply(N, M, Q, h, W, np.eye(n)[j]) for j in range(n)], axis=1)
        np.testing.assert_allclose(Hs, Hs.conj().T, atol=1e-12)
        parts.append(np.linalg.eigvalsh(Hs))
    np.testing.assert_allclose(np.sort(np.concatenate(parts)), full, atol=1e-10)


def test_lieb_liniger_ground_state_in_zero_momentum_sector():
    N, M = 5, 5
    h, W = inputs.lieb_liniger_hw(M, 1.0)
    full = np.linalg.eigvalsh(oracle.dense_hamiltonian(N, M, h, W))[0]
    Q0 = N * (M // 2)
    n = len(oracle.sector_indices(N, M, Q0))
    Hs = np.stack([oracle.sector_apply(N, M, Q0, h, W, np.eye(n)[j]) for j in range(n)], axis=1)
    assert n == 12
    assert abs(np.linalg.eigvalsh(Hs)[0] - full) <= 1e-12 * abs(full)
