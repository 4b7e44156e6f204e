"""GPU one- and two-body density matrices (Eqs. rho1, rho2) through the C ABI:
element by element against the oracle on small spaces, and at full size
(N = 100, M = 6) against the particle-number traces, the rho2-to-rho1
contraction and rho1 entries evaluated as <C| h_kl C> with the library's
native FP64 apply of a unit one-body operator (an independent code path).

When both matrices are asked for, the library forms rho1 as the partial
trace of rho2 (sum_x rho2[k][x][x][l] = (N - 1) rho1[k][l]); asked for
alone, rho1 comes from its own Gram reduction over the (N-1)-particle space.
Both forms are checked against the oracle, and the contraction identity is
checked on the direct form.

Tolerance 1e-12 relative to the largest element: products are FP32 pairs
(48-bit significands) summed over 32 configurations, then in FP64."""
import numpy as np
import pytest

import oracle
from paper_2005_13679_gb300 import fock, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    fock.load()
    return t


SMALL = [(1, 4), (2, 5), (3, 3), (4, 4), (5, 3), (6, 2), (3, 6), (2, 8), (7, 1), (4, 5)]


@pytest.mark.parametrize("N,M", SMALL)
def test_density_matrices_against_oracle(torch, N, M):
    n = oracle.nc(N, M)
    C = inputs.random_state(n, 41 + N + M)
    sp = fock.Space(N, M)
    r1, r2 = fock.fock_density_matrices(sp.handle, torch.from_numpy(C).cuda(), M)
    d1, none = fock.fock_density_matrices(sp.handle, torch.from_numpy(C).cuda(), M, want_rho2=False)
    assert none is None
    o1 = oracle.rho1(N, M, C)
    scale1 = max(np.abs(o1).max(), 1e-300)
    assert np.abs(r1 - o1).max() <= 1e-12 * scale1
    assert np.abs(d1 - o1).max() <= 1e-12 * scale1
    if M <= 6:
        o2 = oracle.rho2(N, M, C)
        scale2 = max(np.abs(o2).max(), 1e-300)
        assert np.abs(r2 - o2).max() <= 1e-12 * scale2
    # identities hold at any size
    norm2 = np.vdot(C, C).real
    assert abs(np.trace(r1).real - N * norm2) <= 1e-12 * N * norm2
    if N >= 2:
        assert np.allclose(np.einsum("kqql->kl", r2), (N - 1) * d1, rtol=0, atol=1e-12 * N * scale1)


def test_density_matrices_full_size(torch):
    w = inputs.WORKLOADS["generic_n100_m6"]
    N, M = w.N, w.M
    sp = fock.Space(N, M)
    Cd = torch.from_numpy(w.state()).cuda()
    r1, r2 = fock.fock_density_matrices(sp.handle, Cd, M)
    d1, _ = fock.fock_density_matrices(sp.handle, Cd, M, want_rho2=False)    # direct Gram over N-1 particles
    norm2 = torch.vdot(Cd, Cd).real.item()
    assert abs(np.trace(r1).real - N * norm2) <= 1e-12 * N * norm2
    assert abs(np.trace(d1).real - N * norm2) <= 1e-12 * N * norm2
    assert abs(np.einsum("kllk->", r2).real - N * (N - 1) * norm2) <= 1e-12 * N * N * norm2
    scale1 = np.abs(r1).max()
    assert np.abs(np.einsum("kqql->kl", r2) - (N - 1) * d1).max() <= 1e-11 * N * scale1
    assert np.abs(r1 - d1).max() <= 1e-12 * scale1
    assert np.allclose(r1, r1.conj().T, rtol=0, atol=1e-14 * scale1)
    # entries of rho1 by the native FP64 apply of unit one-body operators
    for k, l in [(0, 0), (2, 3), (5, 1), (4, 4)]:
        h = np.zeros((M, M), dtype=np.complex128)
        h[k, l] += 0.5
        h[l, k] += 0.5                                   # Hermitian: (E_kl + E_lk) / 2
        H = fock.Hamiltonian(sp, h, None)
        s = H.apply(Cd, precision=fock.FOCK_PREC_F64_NATIVE)
        want = torch.vdot(Cd, s).item()                  # Re rho1_kl (= (rho1_kl + rho1_lk) / 2)
        assert abs(want - 0.5 * (r1[k, l] + r1[l, k])) <= 1e-12 * scale1
