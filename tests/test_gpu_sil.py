"""GPU short-iterative-Lanczos step C <- exp(-i H dt) C through the C ABI:
against the oracle's exact propagator on small spaces, and at full size
(generic N = 100, M = 6) unitarity, conservation of <H> and reversibility
(a step of -dt undoes a step of dt).

Tolerances: the Krylov space grows until the neglected weight is below tol =
1e-12, so the step agrees with the exact propagator to ~1e-11 relative."""
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


@pytest.mark.parametrize("N,M,kind,dt", [(4, 4, "generic", 0.2), (5, 3, "ll", 0.05), (3, 6, "generic", 0.5),
                                          (6, 2, "ll", 0.1), (1, 5, "generic", 0.3)])
def test_sil_step_against_exact(torch, N, M, kind, dt):
    h, W = inputs.lieb_liniger_hw(M, 1.3) if kind == "ll" else inputs.random_hermitian_hw(M, 9)
    C = inputs.random_state(oracle.nc(N, M), 12)
    sp = fock.Space(N, M)
    H = fock.Hamiltonian(sp, h, W)
    Cd = torch.from_numpy(C).cuda()
    m, err, st = fock.fock_sil_step(sp.handle, H.handle, Cd, dt, max_krylov=64, tol=1e-12)
    assert st == fock.FOCK_OK and err < 1e-12
    ref = oracle.evolve(N, M, h, W, C, dt)
    assert np.linalg.norm(Cd.cpu().numpy() - ref) <= 1e-10 * np.linalg.norm(ref)


def test_sil_full_size_invariants(torch):
    w = inputs.WORKLOADS["generic_n100_m6"]
    h, W = w.hamiltonian()
    sp = fock.Space(w.N, w.M)
    H = fock.Hamiltonian(sp, h, W)
    C0 = torch.from_numpy(w.state()).cuda()
    C0 /= torch.linalg.norm(C0)
    e0 = torch.vdot(C0, H.apply(C0)).real.item()
    C = C0.clone()
    dt = 2e-3
    m, err, st = fock.fock_sil_step(sp.handle, H.handle, C, dt, max_krylov=40, tol=1e-11)
    assert st == fock.FOCK_OK
    assert abs(torch.linalg.norm(C).item() - 1.0) < 1e-12
    e1 = torch.vdot(C, H.apply(C)).real.item()
    assert abs(e1 - e0) <= 1e-10 * abs(e0)
    assert torch.linalg.norm(C - C0).item() > 1e-3        # it moved
    m2, err2, st2 = fock.fock_sil_step(sp.handle, H.handle, C, -dt, max_krylov=40, tol=1e-11)
    assert st2 == fock.FOCK_OK
    assert torch.linalg.norm(C - C0).item() <= 1e-9
