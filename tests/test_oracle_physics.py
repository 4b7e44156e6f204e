"""Pins for the oracle's Lanczos solver and Bethe-ansatz energy (Sec. 6).

* Lanczos against LAPACK's dense Hermitian eigen-solver on the oracle's dense H;
* the Bethe-ansatz solver against three independent facts: the two-body ring
  problem solved directly (tan(q L / 2) = g / (2 q), E = q^2), the
  Tonks-Girardeau limit (free fermions with I_j = j - (N+1)/2), and
  first-order perturbation theory at weak coupling (E ~ g N (N-1) / 2L);
* exact diagonalisation of the Lieb-Liniger ring converging from above to the
  Bethe-ansatz energy as orbitals are added (variational, nested subspaces).
"""
import numpy as np
import pytest
from scipy.optimize import brentq

import oracle
from paper_2005_13679_gb300 import inputs


@pytest.mark.parametrize("N,M,kind", [(5, 5, "ll"), (3, 4, "generic"), (4, 5, "generic"), (6, 3, "ll")])
def test_lanczos_matches_dense(N, M, kind):
    h, W = inputs.lieb_liniger_hw(M, 1.0) if kind == "ll" else inputs.random_hermitian_hw(M, 9)
    n = oracle.nc(N, M)
    H = oracle.dense_hamiltonian(N, M, h, W)
    E_dense = np.linalg.eigvalsh(H)[0]
    E, v, it = oracle.lanczos_ground(lambda x: oracle.apply_push(N, M, h, W, x),
                                     inputs.random_state(n, 101), max_iter=n)
    assert abs(E - E_dense) <= 1e-10 * max(1.0, abs(E_dense))
    assert np.linalg.norm(H @ v - E * v) < 1e-6


@pytest.mark.parametrize("g", [0.1, 1.0, 7.5])
def test_bethe_two_body_closed_form(g):
    E, k = oracle.bethe_ground_energy(2, g)
    q = brentq(lambda x: np.tan(x / 2.0) - g / (2.0 * x), 1e-12, np.pi - 1e-12)
    assert abs(E - q * q) < 1e-12 * max(1.0, q * q)
    assert abs(k[0] + k[1]) < 1e-13


@pytest.mark.parametrize("N", [2, 3, 4, 5, 6])
def test_bethe_tonks_girardeau_limit(N):
    I = np.arange(1, N + 1) - (N + 1) / 2.0
    E_tg = 0.5 * float(np.sum((2 * np.pi * I) ** 2))
    E, _ = oracle.bethe_ground_energy(N, 1e9)
    assert abs(E - E_tg) / E_tg < 1e-7
    assert oracle.bethe_ground_energy(N, 50.0)[0] < E_tg


@pytest.mark.parametrize("N", [2, 5, 8])
def test_bethe_weak_coupling(N):
    g = 1e-6
    E, _ = oracle.bethe_ground_energy(N, g)
    assert abs(E / (g * N * (N - 1) / 2.0) - 1.0) < 1e-5


def test_ll_exact_diagonalisation_converges_to_bethe():
    N, g = 5, 1.0
    E_bethe, _ = oracle.bethe_ground_energy(N, g)
    energies = []
    for M in (3, 5, 7, 9):
        h, W = inputs.lieb_liniger_hw(M, g)
        H = oracle.dense_hamiltonian(N, M, h, W)
        energies.append(np.linalg.eigvalsh(H)[0])
    assert all(a > b for a, b in zip(energies, energies[1:]))
    assert energies[-1] > E_bethe
    # Tonks-Girardeau energy bounds every finite-g ground state from above
    assert energies[0] < 0.5 * (2 * np.pi) ** 2 * 10


def test_bose_hubbard_limits():
    """Bose-Hubbard ring (inputs.bose_hubbard_hw) through the oracle: with U = 0
    the ground energy is N times the lowest ring mode, -2J; with J = 0 the
    Hamiltonian is diagonal with (U/2) sum_k n_k (n_k - 1)."""
    N, M = 4, 5
    h, W = inputs.bose_hubbard_hw(M, J=0.7, U=0.0)
    E = np.linalg.eigvalsh(oracle.dense_hamiltonian(N, M, h, W))
    assert abs(E[0] - N * (-2 * 0.7)) < 1e-12
    h, W = inputs.bose_hubbard_hw(M, J=0.0, U=1.7)
    H = oracle.dense_hamiltonian(N, M, h, W)
    assert np.allclose(H, np.diag(np.diag(H)), atol=1e-14)
    for i in range(oracle.nc(N, M)):
        n = oracle.unrank(N, M, i)
        assert abs(H[i, i] - 0.5 * 1.7 * np.sum(n * (n - 1))) < 1e-12
