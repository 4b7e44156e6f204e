"""Pins of the oracle's propagator exp(-i H dt) C against facts that do not
use its eigen-decomposition: unitarity, the phase of an eigenvector (from the
Lieb-Liniger closed forms), the group law, the small-dt limit -i H C (with
the push apply), and a Pade exponential of the dense matrix."""
import numpy as np
import pytest
import scipy.linalg

import oracle
from paper_2005_13679_gb300 import inputs


def hw(kind, M, seed=3):
    return inputs.lieb_liniger_hw(M, 0.7) if kind == "ll" else inputs.random_hermitian_hw(M, seed)


@pytest.mark.parametrize("N,M,kind", [(3, 4, "generic"), (4, 3, "ll"), (2, 5, "generic")])
def test_unitary_group_law_small_dt(N, M, kind):
    h, W = hw(kind, M)
    C = inputs.random_state(oracle.nc(N, M), 5)
    a = oracle.evolve(N, M, h, W, C, 0.3)
    assert abs(np.linalg.norm(a) - np.linalg.norm(C)) < 1e-12
    b = oracle.evolve(N, M, h, W, oracle.evolve(N, M, h, W, C, 0.1), 0.2)
    assert np.linalg.norm(a - b) < 1e-12
    assert np.linalg.norm(oracle.evolve(N, M, h, W, a, -0.3) - C) < 1e-12
    eps = 1e-5                                           # central difference: O(eps^2 ||H||^3)
    d = (oracle.evolve(N, M, h, W, C, eps) - oracle.evolve(N, M, h, W, C, -eps)) / (2 * eps)
    assert np.linalg.norm(d + 1j * oracle.apply_push(N, M, h, W, C)) < 1e-6 * np.linalg.norm(d)
    Hd = oracle.dense_hamiltonian(N, M, h, W)
    assert np.linalg.norm(scipy.linalg.expm(-1j * 0.3 * Hd) @ C - a) < 1e-11


def test_condensate_phase_at_zero_coupling():
    # g = 0: every configuration is an eigenvector with E = sum_k eps_k n_k
    N, M = 3, 5
    h, W = inputs.lieb_liniger_hw(M, 0.0)
    n = oracle.nc(N, M)
    for idx in (0, n // 2, n - 1):
        C = np.zeros(n, dtype=np.complex128)
        C[idx] = 1.0
        occ = oracle.unrank(N, M, idx)
        E = float(np.sum(np.real(np.diag(h)) * occ))
        out = oracle.evolve(N, M, h, W, C, 0.45)
        assert abs(out[idx] - np.exp(-1j * E * 0.45)) < 1e-12
        assert np.linalg.norm(out) - 1.0 < 1e-13
