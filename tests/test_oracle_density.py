"""Pins of the oracle's density matrices (Eqs. rho1, rho2) against facts the
definitions imply, independent of the push apply the oracle uses: traces
fixed by the particle number, the contraction of rho2 to rho1, Hermiticity,
exchange symmetry of the boson operators, positive semidefiniteness, and the
explicit Appendix B element rules evaluated by brute-force enumeration."""
import numpy as np
import pytest

import oracle
from paper_2005_13679_gb300 import inputs

CASES = [(3, 3), (4, 4), (5, 3), (2, 5), (1, 4)]


@pytest.mark.parametrize("N,M", CASES)
def test_rho1_trace_hermitian_psd(N, M):
    C = inputs.random_state(oracle.nc(N, M), 31)
    r1 = oracle.rho1(N, M, C)
    norm2 = np.vdot(C, C).real
    assert abs(np.trace(r1) - N * norm2) < 1e-12 * N * norm2
    assert np.allclose(r1, r1.conj().T, atol=1e-13)
    assert np.linalg.eigvalsh(r1).min() > -1e-12


@pytest.mark.parametrize("N,M", [(3, 3), (4, 4), (5, 3), (2, 5)])
def test_rho2_trace_contraction_symmetry(N, M):
    C = inputs.random_state(oracle.nc(N, M), 33)
    r1 = oracle.rho1(N, M, C)
    r2 = oracle.rho2(N, M, C)
    norm2 = np.vdot(C, C).real
    # sum_{k,l} <a^dag_k a^dag_l a_l a_k> = N (N - 1) for an N-particle state
    assert abs(np.einsum("kllk->", r2) - N * (N - 1) * norm2) < 1e-11 * N * N * norm2
    # sum_q a^dag_k a^dag_q a_q a_l = a^dag_k (N - 1) a_l
    assert np.allclose(np.einsum("kqql->kl", r2), (N - 1) * r1, atol=1e-11)
    # bosonic exchange symmetry and Hermiticity
    assert np.allclose(r2, r2.transpose(1, 0, 2, 3), atol=1e-13)
    assert np.allclose(r2, r2.transpose(0, 1, 3, 2), atol=1e-13)
    assert np.allclose(r2, r2.transpose(3, 2, 1, 0).conj(), atol=1e-13)
    # as a matrix over (annihilated pair) x (annihilated pair) it is a Gram matrix
    G = r2.transpose(1, 0, 2, 3).reshape(M * M, M * M)
    assert np.linalg.eigvalsh(0.5 * (G + G.conj().T)).min() > -1e-11


def test_rho_elements_by_enumeration():
    # rho_kl and rho_ksql written out over an enumerated basis (Appendix B rules)
    N, M = 4, 4
    C = inputs.random_state(oracle.nc(N, M), 35)
    confs = [tuple(oracle.unrank(N, M, i)) for i in range(oracle.nc(N, M))]
    idx = {c: i for i, c in enumerate(confs)}
    r1 = oracle.rho1(N, M, C)
    r2 = oracle.rho2(N, M, C)
    k, s, q, l = 0, 1, 2, 3
    want1 = 0j
    want2 = 0j
    for b, c in enumerate(confs):
        n = np.array(c)
        if n[k] >= 1:                                    # beta_k^l
            t = list(c); t[k] -= 1; t[l] += 1
            want1 += np.conj(C[b]) * C[idx[tuple(t)]] * np.sqrt((n[l] + 1) * n[k])
        if n[k] >= 1 and n[s] >= 1:                      # beta_ks^ql
            t = list(c); t[k] -= 1; t[s] -= 1; t[q] += 1; t[l] += 1
            want2 += np.conj(C[b]) * C[idx[tuple(t)]] * np.sqrt(n[k] * n[s] * (n[q] + 1) * (n[l] + 1))
    assert abs(r1[k, l] - want1) < 1e-13
    # <a^dag_k a^dag_s a_q a_l> is rho2[k, s, q, l]
    assert abs(r2[k, s, q, l] - want2) < 1e-13
