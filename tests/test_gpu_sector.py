"""GPU parity of the fixed-weight (total-momentum) sectors, through the C ABI.

Hash: bit-exact against the oracle's sector enumeration (the full space's
order restricted to the configurations of weight Q).  Apply: relative 2-norm
of the difference against the oracle's embed / push apply / restrict, with the
tolerances of the full-space apply (1e-12 FP64-class and native, 5e-6 FP32-
mixed).  Lanczos: the sector's lowest eigenvalue against the oracle's dense
sector matrix, and the zero-momentum sector against the full-space ground
state of the Lieb-Liniger ring.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2005_13679_gb300 import fock, inputs

pytestmark = pytest.mark.gpu

TOL = {fock.FOCK_PREC_F64: 1e-12, fock.FOCK_PREC_F64_NATIVE: 1e-12, fock.FOCK_PREC_F32_MIXED: 5e-6}
PRECS = list(TOL)


@pytest.fixture(scope="module")
def torch():
    import torch as t
    fock.load()
    return t


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def hw(kind, M):
    if kind == "ll":
        return inputs.lieb_liniger_hw(M, 0.7)
    if kind == "wc":
        return inputs.weight_conserving_hw(M, 13)
    h, _ = inputs.weight_conserving_hw(M, 13)
    return h, None                       # diagonal one-body operator only


def dev(torch, x, prec=fock.FOCK_PREC_F64):
    t = torch.from_numpy(np.ascontiguousarray(x))
    if prec == fock.FOCK_PREC_F32_MIXED:
        t = t.to(torch.complex64)
    return t.cuda()


# (N, M, Q): extremes (one configuration), M = 1 and 2, the zero-momentum
# sectors of several rings (Q = N floor(M/2)), several tiles with a ragged tail.
HASH_CASES = [(5, 5, 10), (8, 6, 15), (6, 4, 0), (6, 4, 18), (3, 12, 16), (9, 1, 0), (7, 2, 3),
              (10, 7, 30), (14, 8, 56), (12, 8, 40)]


@pytest.mark.parametrize("N,M,Q", HASH_CASES)
def test_sector_hash_against_oracle(torch, N, M, Q):
    sp = fock.Space(N, M)
    sec = fock.Sector(sp, Q)
    idx = oracle.sector_indices(N, M, Q)
    assert sec.size == len(idx)
    ref_occ = oracle.unrank_batch(N, M, idx)
    occ, _ = fock.fock_sector_unrank(sec.handle, torch.arange(sec.size, dtype=torch.int64, device="cuda"), M)
    assert np.array_equal(occ.cpu().numpy(), ref_occ)
    back, _ = fock.fock_sector_rank(sec.handle, torch.from_numpy(ref_occ).cuda())
    assert np.array_equal(back.cpu().numpy(), np.arange(sec.size))


def test_sector_hash_errors(torch):
    sp = fock.Space(5, 4)
    sec = fock.Sector(sp, 6)
    bad = np.array([[5, 0, 0, 0],          # weight 0
                    [1, 1, 1, 2],          # weight 9
                    [-1, 3, 2, 1],         # negative entry
                    [1, 2, 1, 0],          # four particles
                    [2, 1, 1, 1]], dtype=np.int32)   # a sector member (weight 6)
    idx, st = fock.fock_sector_rank(sec.handle, torch.from_numpy(bad).cuda(), check=False)
    assert st == fock.FOCK_ERR_INVALID_CONFIG
    ref = oracle.sector_indices(5, 4, 6)
    pos = int(np.nonzero(ref == oracle.rank(5, 4, bad[4]))[0][0])
    assert idx.cpu().numpy().tolist() == [-1, -1, -1, -1, pos]
    occ, st = fock.fock_sector_unrank(sec.handle, torch.tensor([0, sec.size, -1], dtype=torch.int64,
                                                               device="cuda"), 4, check=False)
    assert st == fock.FOCK_ERR_RANGE
    o = occ.cpu().numpy()
    assert np.all(o[1:] == -1) and np.array_equal(o[0], oracle.unrank(5, 4, ref[0]))
    with pytest.raises(fock.FockError):
        fock.Sector(sp, 16)                # above N (M - 1) = 15
    with pytest.raises(fock.FockError):
        fock.Sector(sp, -1)


# Apply cases: Lieb-Liniger, a random complex weight-conserving W, and a
# diagonal one-body operator; sectors of one to thousands of configurations.
APPLY_CASES = [(10, 7, 30, "ll"), (14, 8, 56, "ll"), (12, 8, 40, "wc"), (9, 6, 27, "wc"),
               (6, 4, 0, "ll"), (7, 5, 12, "onebody"), (1, 6, 4, "ll"), (8, 1, 0, "wc"), (6, 12, 30, "ll")]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("N,M,Q,kind", APPLY_CASES)
def test_sector_apply_against_oracle(torch, N, M, Q, kind, prec):
    h, W = hw(kind, M)
    sp = fock.Space(N, M)
    sec = fock.Sector(sp, Q)
    H = fock.Hamiltonian(sp, h, W)
    C = inputs.random_state(sec.size, 31)
    ref = oracle.sector_apply(N, M, Q, h, W, C)
    out = sec.apply(H, dev(torch, C, prec), precision=prec).cpu().numpy().astype(np.complex128)
    assert rel(out, ref) <= TOL[prec]


@pytest.mark.parametrize("prec", PRECS)
def test_sector_block_rhs(torch, prec):
    N, M, Q, nrhs = 12, 8, 48, 3
    h, W = hw("wc", M)
    sp = fock.Space(N, M)
    sec = fock.Sector(sp, Q)
    H = fock.Hamiltonian(sp, h, W)
    Cb = np.stack([inputs.random_state(sec.size, 50 + j) for j in range(nrhs)], axis=1)
    out = sec.apply(H, dev(torch, Cb, prec), nrhs=nrhs, precision=prec).cpu().numpy().astype(np.complex128)
    for j in range(nrhs):
        ref = oracle.sector_apply(N, M, Q, h, W, Cb[:, j])
        assert rel(out[:, j], ref) <= TOL[prec]


def test_sector_rejects_non_conserving_operators(torch):
    sp = fock.Space(5, 5)
    sec = fock.Sector(sp, 10)
    C = dev(torch, inputs.random_state(sec.size, 1))
    for h, W in (inputs.random_hermitian_hw(5, 3), inputs.bose_hubbard_hw(5, 1.0, 2.0)):
        H = fock.Hamiltonian(sp, h, W)
        with pytest.raises(fock.FockError) as e:
            sec.apply(H, C)
        assert e.value.status == fock.FOCK_ERR_NOT_CONSERVING
        with pytest.raises(fock.FockError) as e:
            fock.fock_sector_terms(sec.handle, H.handle)
        assert e.value.status == fock.FOCK_ERR_NOT_CONSERVING


def test_sector_terms_add_up_to_the_full_space(torch):
    """Every (N-2)-configuration has exactly one weight, so the terms of all
    sectors add up to (listed removal-addition pairs) x N_c(N - 2, M)."""
    N, M = 9, 6
    h, W = inputs.lieb_liniger_hw(M, 0.7)
    sp = fock.Space(N, M)
    H = fock.Hamiltonian(sp, h, W)
    pairs = {}
    for k in range(M):
        for q in range(M):
            for s in range(M):
                for l in range(M):
                    if W[k, q, s, l] != 0 or (q == s and h[k, l] != 0):
                        pairs[(min(k, q), max(k, q), min(s, l), max(s, l))] = 1
    sectors = [fock.Sector(sp, Q) for Q in range(N * (M - 1) + 1)]     # alive across the calls
    total = sum(fock.fock_sector_terms(sec.handle, H.handle) for sec in sectors)
    assert total == len(pairs) * math.comb(N - 2 + M - 1, M - 1)


@pytest.mark.parametrize("N,M,Q,kind", [(6, 7, 18, "ll"), (9, 6, 27, "wc"), (8, 6, 20, "ll")])
def test_sector_lanczos_against_dense_sector(torch, N, M, Q, kind):
    h, W = hw(kind, M)
    sp = fock.Space(N, M)
    sec = fock.Sector(sp, Q)
    H = fock.Hamiltonian(sp, h, W)
    n = sec.size
    Hs = np.stack([oracle.sector_apply(N, M, Q, h, W, np.eye(n)[j]) for j in range(n)], axis=1)
    E_ref = np.linalg.eigvalsh(Hs)[0]
    E0, res, it, vec, st = fock.fock_sector_lanczos_ground(sec.handle, H.handle, max_iter=400, restart_len=40,
                                                          tol=1e-12, want_vector=True)
    assert st == fock.FOCK_OK
    assert abs(E0 - E_ref) <= 1e-10 * max(abs(E_ref), 1.0)
    v = vec.cpu().numpy()
    r = oracle.sector_apply(N, M, Q, h, W, v) - E0 * v
    assert np.linalg.norm(r) <= 1e-6 * max(abs(E0), 1.0)


def test_zero_momentum_sector_holds_the_lieb_liniger_ground_state(torch):
    N, M = 8, 7
    h, W = inputs.lieb_liniger_hw(M, 1.0)
    sp = fock.Space(N, M)
    H = fock.Hamiltonian(sp, h, W)
    E_full = fock.fock_lanczos_ground(sp.handle, H.handle, max_iter=600, restart_len=40, tol=1e-12)[0]
    sec = fock.Sector(sp, N * (M // 2))
    for prec in (fock.FOCK_PREC_F64, fock.FOCK_PREC_F32_MIXED):
        E0, _, _, _, st = fock.fock_sector_lanczos_ground(sec.handle, H.handle, max_iter=600, restart_len=40,
                                                          tol=1e-12, precision=prec)
        assert st == fock.FOCK_OK
        assert abs(E0 - E_full) <= 1e-10 * abs(E_full)


def test_full_size_zero_momentum_sector_sampled_rows(torch):
    """Lieb-Liniger N = 30, M = 10, total momentum 0: 2,462,733 of the
    211,915,132 configurations.  Sampled rows of the FP64-class apply against
    the oracle's rows of the full operator on the embedded vector."""
    N, M = 30, 10
    Q = N * (M // 2)
    h, W = inputs.lieb_liniger_hw(M, 0.5)
    sp = fock.Space(N, M)
    sec = fock.Sector(sp, Q)
    assert sec.size == 2462733
    H = fock.Hamiltonian(sp, h, W)
    C = inputs.random_state(sec.size, 3)
    out = sec.apply(H, dev(torch, C)).cpu().numpy()
    occ, _ = fock.fock_sector_unrank(sec.handle, torch.arange(sec.size, dtype=torch.int64, device="cuda"), M)
    occ = occ.cpu().numpy()
    assert np.all(occ.astype(np.int64) @ np.arange(M) == Q) and np.all(occ.sum(axis=1) == N)
    full_idx = oracle.rank_batch(N, M, occ)
    assert np.all(np.diff(full_idx) > 0)          # the full space's order, restricted
    Cf = np.zeros(oracle.nc(N, M), dtype=np.complex128)
    Cf[full_idx] = C
    rng = np.random.Generator(np.random.PCG64(17))
    rows = np.unique(np.concatenate([rng.integers(0, sec.size, 200), [0, 1, sec.size - 2, sec.size - 1]]))
    ref = oracle.apply_rows(N, M, h, W, Cf, full_idx[rows])
    assert rel(out[rows], ref) <= 1e-12
