"""GPU Lanczos ground state (Sec. 6) against the oracle's dense diagonalisation
and Lanczos, through the C ABI.  Energies must match to 1e-10 relative."""
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


@pytest.mark.parametrize("prec", [fock.FOCK_PREC_F64, fock.FOCK_PREC_F64_NATIVE, fock.FOCK_PREC_F32_MIXED])
def test_ll_n5_m5_against_dense(torch, prec):
    w = inputs.WORKLOADS["ll_n5_m5"]
    h, W = w.hamiltonian()
    E_dense = np.linalg.eigvalsh(oracle.dense_hamiltonian(w.N, w.M, h, W))[0]
    sp = fock.Space(w.N, w.M)
    H = fock.Hamiltonian(sp, h, W)
    E, res, it, vec, st = fock.fock_lanczos_ground(sp.handle, H.handle, max_iter=400, restart_len=40,
                                                   tol=1e-12, seed=w.lanczos_seed, precision=prec,
                                                   want_vector=True)
    assert st == fock.FOCK_OK
    assert abs(E - E_dense) <= 1e-10 * abs(E_dense)
    assert res <= 1e-8 * abs(E_dense)
    v = vec.cpu().numpy()
    Hd = oracle.dense_hamiltonian(w.N, w.M, h, W)
    assert np.linalg.norm(Hd @ v - E * v) <= 1e-8 * abs(E)


@pytest.mark.parametrize("N,M,kind,restart", [(6, 6, "generic", 20), (10, 5, "ll", 12), (4, 9, "ll", 30)])
def test_restarted_against_oracle(torch, N, M, kind, restart):
    h, W = inputs.lieb_liniger_hw(M, 0.7) if kind == "ll" else inputs.random_hermitian_hw(M, 3)
    n = oracle.nc(N, M)
    E_ref = np.linalg.eigvalsh(oracle.dense_hamiltonian(N, M, h, W))[0]
    sp = fock.Space(N, M)
    H = fock.Hamiltonian(sp, h, W)
    start = torch.from_numpy(inputs.random_state(n, 8)).cuda()
    E, res, it, _, st = fock.fock_lanczos_ground(sp.handle, H.handle, max_iter=2000, restart_len=restart,
                                                 tol=1e-12, precision=fock.FOCK_PREC_F64, start=start)
    assert st == fock.FOCK_OK
    assert abs(E - E_ref) <= 1e-10 * max(1.0, abs(E_ref))


def test_noninteracting_closed_form(torch):
    # g = 0: ground energy 0 (all bosons at zero momentum)
    h, W = inputs.lieb_liniger_hw(7, 0.0)
    sp = fock.Space(6, 7)
    H = fock.Hamiltonian(sp, h, W)
    E, res, it, _, st = fock.fock_lanczos_ground(sp.handle, H.handle, max_iter=500, restart_len=30,
                                                 tol=1e-12, seed=3)
    assert abs(E) <= 1e-10


def test_max_iter_reports_noconv(torch):
    w = inputs.WORKLOADS["ll_n5_m5"]
    h, W = w.hamiltonian()
    sp = fock.Space(w.N, w.M)
    H = fock.Hamiltonian(sp, h, W)
    E, res, it, _, st = fock.fock_lanczos_ground(sp.handle, H.handle, max_iter=3, restart_len=10,
                                                 tol=1e-14, seed=1)
    assert st == fock.FOCK_ERR_NOCONV and it == 3 and np.isfinite(E)


def test_ll_n30_m10_precision_forms(torch):
    """212M configurations: FP32-mixed products with FP64 orthogonalisation and
    final FP64 refinement give the FP64 ground energy to 1e-10 relative.  No
    oracle runs at this size; the energy is bracketed by the Bethe-ansatz energy
    (variational bound, the plane-wave space is a subspace) and by the energy of
    the condensate in the zero-momentum orbital, g N (N - 1) / 2L."""
    w = inputs.WORKLOADS["ll_n30_m10"]
    h, W = w.hamiltonian()
    sp = fock.Space(w.N, w.M)
    H = fock.Hamiltonian(sp, h, W)
    runs = {}
    for prec in (fock.FOCK_PREC_F64, fock.FOCK_PREC_F32_MIXED):
        E, res, it, vec, st = fock.fock_lanczos_ground(sp.handle, H.handle, max_iter=300, restart_len=24,
                                                       tol=1e-9, seed=w.lanczos_seed, precision=prec,
                                                       want_vector=(prec == fock.FOCK_PREC_F64))
        assert st == fock.FOCK_OK, (prec, E, res, it)
        assert res <= 1e-6 * abs(E)
        runs[prec] = (E, vec)
    E64, v = runs[fock.FOCK_PREC_F64]
    Emix = runs[fock.FOCK_PREC_F32_MIXED][0]
    assert abs(Emix - E64) <= 1e-10 * abs(E64)
    E_bethe, _ = oracle.bethe_ground_energy(w.N, w.g)
    assert E_bethe < E64 < w.g * w.N * (w.N - 1) / 2.0
    # error of one FP32-mixed product against the FP64-class product on the ground vector
    s64 = H.apply(v, precision=fock.FOCK_PREC_F64)
    s32 = H.apply(v.to(torch.complex64), precision=fock.FOCK_PREC_F32_MIXED).to(torch.complex128)
    assert (torch.linalg.norm(s32 - s64) / torch.linalg.norm(s64)).item() <= 5e-6
