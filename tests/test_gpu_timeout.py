"""The bounded-wait abort path of the tensor-core phase 1, run without a fault
or a hang.

Every wait of the kernel's producer, MMA-issue and epilogue roles polls an
mbarrier a bounded number of times.  With the process-wide test hook
fock_debug_set_wait_polls(0) each of those waits gives up at once: the MMA
role returns before issuing anything, the other roles leave their loops, the
status word is set and phase 2 writes NaN.  The final wait that lets issued
MMAs finish before tensor memory is released keeps its full budget (here
nothing was issued).  The test checks the reported status on every entry
point, then that the next apply with the default budget is correct again.
"""
import numpy as np
import pytest

import oracle
from paper_2005_13679_gb300 import fock, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    fock.load()
    yield t
    fock.fock_debug_set_wait_polls(-1)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("prec", [fock.FOCK_PREC_F64, fock.FOCK_PREC_F32_MIXED])
def test_wait_budget_exhausted_then_recovers(torch, prec):
    N, M = 12, 6
    h, W = inputs.random_hermitian_hw(M, 17)
    sp = fock.Space(N, M)
    H = fock.Hamiltonian(sp, h, W)
    assert fock.PATH_NAMES[fock.fock_apply_path(sp.handle, H.handle, 1, prec)] == "twophase_tc"
    C = inputs.random_state(sp.nc, 3)
    ref = oracle.apply_push(N, M, h, W, C)
    dt = torch.complex64 if prec == fock.FOCK_PREC_F32_MIXED else torch.complex128
    tol = 5e-6 if prec == fock.FOCK_PREC_F32_MIXED else 1e-12
    Ch = torch.from_numpy(C).to(dt).pin_memory()
    Sh = torch.empty_like(Ch).pin_memory()
    Cd = Ch.cuda()
    try:
        fock.fock_debug_set_wait_polls(0)
        # host buffers: the call itself reports the timeout
        st = fock.load().fock_apply_H_host(sp.handle, H.handle, fock.ctypes.c_void_p(Ch.data_ptr()),
                                           fock.ctypes.c_void_p(Sh.data_ptr()), 1, prec, fock.FOCK_ARM_AUTO,
                                           fock._stream(None))
        assert st == fock.FOCK_ERR_TIMEOUT
        assert np.all(np.isnan(Sh.numpy()))
        # device buffers: the apply returns before the device work ends; the
        # check reads the status word of the Hamiltonian's workspace
        out = H.apply(Cd, precision=prec)
        assert fock.fock_apply_check(sp.handle, H.handle) == fock.FOCK_ERR_TIMEOUT
        assert np.all(np.isnan(out.cpu().numpy()))
    finally:
        fock.fock_debug_set_wait_polls(-1)
    # default budget again: the same objects give the right answer
    out = H.apply(Cd, precision=prec)
    assert fock.fock_apply_check(sp.handle, H.handle) == fock.FOCK_OK
    assert rel(out.cpu().numpy().astype(np.complex128), ref) <= tol
    fock.fock_apply_H_host(sp.handle, H.handle, Ch, Sh, 1, prec)
    assert rel(Sh.numpy().astype(np.complex128), ref) <= tol
    torch.cuda.synchronize()


def test_check_without_tensor_core_path(torch):
    # a path without the tensor-core phase 1 never reports a timeout, even with
    # the budget at zero (its kernels have no such waits)
    N, M = 8, 8
    h, W = inputs.random_hermitian_hw(M, 19)
    sp = fock.Space(N, M)
    H = fock.Hamiltonian(sp, h, W)
    assert fock.PATH_NAMES[fock.fock_apply_path(sp.handle, H.handle)] != "twophase_tc"
    C = inputs.random_state(sp.nc, 4)
    try:
        fock.fock_debug_set_wait_polls(0)
        out = H.apply(torch.from_numpy(C).cuda())
        assert fock.fock_apply_check(sp.handle, H.handle) == fock.FOCK_OK
    finally:
        fock.fock_debug_set_wait_polls(-1)
    assert rel(out.cpu().numpy(), oracle.apply_push(N, M, h, W, C)) <= 1e-12
    with pytest.raises(fock.FockError):
        fock.fock_debug_set_wait_polls(1 << 40)
