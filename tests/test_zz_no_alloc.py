"""The allocation-free apply, for callers that must not let the library
allocate device memory (their memory belongs to another allocator, or a
cudaMalloc would synchronise a device they keep busy).

It must give the same sigma as fock_apply_H with FOCK_PREC_F64, within the
1e-12 relative-norm tolerance used for that precision, on consecutive calls
that share the fixed scratch array, agree with the CPU oracle directly, leave
the device's free memory unchanged on a Hamiltonian that never ran the
allocating entry point, and refuse requests larger than that array.  This file
is collected last on purpose.
"""
import numpy as np
import pytest

import oracle
from paper_2005_13679_gb300 import fock, inputs

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_noalloc_matches_apply_on_consecutive_calls():
    import torch
    fock.load()
    cases = [(8, 6, "generic", 1), (10, 5, "ll", 1), (8, 6, "generic", 3)]
    for N, M, kind, nrhs in cases:
        h, W = inputs.lieb_liniger_hw(M, 0.8) if kind == "ll" else inputs.random_hermitian_hw(M, 6)
        sp = fock.Space(N, M)
        H = fock.Hamiltonian(sp, h, W)
        # two calls in a row with different inputs (and magnitudes) through the
        # shared scratch; each compared with the allocating entry point
        for seed, scale in ((21, 1.0), (22, 3e-7)):
            B = inputs.random_block(sp.nc, range(seed, seed + nrhs)) * scale
            C = torch.from_numpy(B if nrhs > 1 else B[:, 0].copy()).cuda()
            ref = fock.fock_apply_H(sp.handle, H.handle, C, nrhs=nrhs, precision=fock.FOCK_PREC_F64)
            out, st = fock.fock_apply_H_noalloc(sp.handle, H.handle, C, nrhs=nrhs)
            torch.cuda.synchronize()
            assert st == fock.FOCK_OK
            assert rel(out.cpu().numpy(), ref.cpu().numpy()) <= 1e-12


def test_noalloc_refuses_oversized_requests():
    import torch
    fock.load()
    N, M = 100, 5                    # 4,598,126 configurations: above the 4,194,288 limit
    sp = fock.Space(N, M)
    assert sp.nc * 16 + 256 > fock.FOCK_NOALLOC_SCRATCH_BYTES
    h, W = inputs.random_hermitian_hw(M, 1)
    H = fock.Hamiltonian(sp, h, W)
    C = torch.zeros(sp.nc, dtype=torch.complex128, device="cuda")
    out = torch.empty_like(C)
    _, st = fock.fock_apply_H_noalloc(sp.handle, H.handle, C, out, check=False)
    assert st == fock.FOCK_ERR_SCRATCH_LIMIT
    assert "no-allocation" in fock.fock_strerror(st)


def test_noalloc_first_call_allocates_nothing():
    import torch
    fock.load()
    N, M = 9, 6
    h, W = inputs.random_hermitian_hw(M, 23)
    sp = fock.Space(N, M)
    C = torch.from_numpy(inputs.random_state(sp.nc, 31)).cuda()
    out = torch.empty_like(C)
    # a warm-up call on another Hamiltonian of the same shape lets CUDA load the
    # kernels' modules (lazy loading), which is a driver allocation
    warm = fock.Hamiltonian(sp, h, W)
    _, st = fock.fock_apply_H_noalloc(sp.handle, warm.handle, C, out)
    torch.cuda.synchronize()
    H = fock.Hamiltonian(sp, h, W)                     # fresh: no workspace of its own yet
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        _, st = fock.fock_apply_H_noalloc(sp.handle, H.handle, C, out)
        assert st == fock.FOCK_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert fock.fock_apply_check(sp.handle, H.handle, noalloc=True) == fock.FOCK_OK
    ref = oracle.apply_push(N, M, h, W, C.cpu().numpy())
    assert rel(out.cpu().numpy(), ref) <= 1e-12
