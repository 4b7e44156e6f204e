"""GPU parity of the hash (Algorithms 1 and 2) and the jump maps (Sec. 4)
against the oracle, through the C ABI.  Bit-exact."""
import math

import numpy as np
import pytest

import oracle
from paper_2005_13679_gb300 import fock

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    fock.load()
    return t


SMALL = [(1, 1), (7, 1), (1, 6), (3, 5), (5, 5), (6, 6), (10, 3), (4, 12), (2, 11)]


@pytest.mark.parametrize("N,M", SMALL)
def test_rank_unrank_all_indices(torch, N, M):
    sp = fock.Space(N, M)
    assert sp.nc == oracle.nc(N, M)
    idx = np.arange(sp.nc, dtype=np.int64)
    ref_occ = oracle.unrank_batch(N, M, idx)
    occ, _ = fock.fock_unrank(sp.handle, torch.from_numpy(idx).cuda(), M)
    assert np.array_equal(occ.cpu().numpy(), ref_occ)
    back, _ = fock.fock_rank(sp.handle, torch.from_numpy(ref_occ).cuda())
    assert np.array_equal(back.cpu().numpy(), idx)


@pytest.mark.parametrize("N,M", [(100, 6), (30, 10), (20, 8), (200, 12), (1000, 3), (45, 10)])
def test_rank_unrank_sampled_large(torch, N, M):
    sp = fock.Space(N, M)
    nc = oracle.nc(N, M)
    assert sp.nc == nc
    rng = np.random.default_rng(N * 100 + M)
    idx = np.concatenate([np.arange(min(nc, 512)), nc - 1 - np.arange(min(nc, 512)),
                          rng.integers(0, nc, size=200_000, dtype=np.int64)]).astype(np.int64)
    ref = oracle.unrank_batch(N, M, idx)
    occ, _ = fock.fock_unrank(sp.handle, torch.from_numpy(idx).cuda(), M)
    assert np.array_equal(occ.cpu().numpy(), ref)
    back, _ = fock.fock_rank(sp.handle, torch.from_numpy(ref).cuda())
    assert np.array_equal(back.cpu().numpy(), idx)


def test_invalid_inputs_are_flagged(torch):
    sp = fock.Space(5, 4)
    occ = torch.tensor([[5, 0, 0, 0], [2, 2, 2, 0], [-1, 3, 3, 0], [0, 0, 0, 5]], dtype=torch.int32).cuda()
    idx, st = fock.fock_rank(sp.handle, occ, check=False)
    assert st == fock.FOCK_ERR_INVALID_CONFIG
    assert idx.cpu().tolist() == [0, -1, -1, sp.nc - 1]
    bad = torch.tensor([0, -1, sp.nc, sp.nc - 1], dtype=torch.int64).cuda()
    occ2, st = fock.fock_unrank(sp.handle, bad, 4, check=False)
    assert st == fock.FOCK_ERR_RANGE
    o = occ2.cpu().numpy()
    assert o[1].tolist() == [-1] * 4 and o[2].tolist() == [-1] * 4
    assert o[3].tolist() == [0, 0, 0, 5]


def test_space_limits(torch):
    with pytest.raises(fock.FockError):
        fock.fock_space_create(0, 3)
    with pytest.raises(fock.FockError):
        fock.fock_space_create(3, 13)
    with pytest.raises(fock.FockError) as e:
        fock.fock_space_create(2 ** 30, 12)
    assert e.value.status == fock.FOCK_ERR_OVERFLOW


@pytest.mark.parametrize("N,M", [(1, 3), (3, 3), (4, 5), (5, 4), (6, 6), (2, 7), (9, 2)])
def test_jump_maps_exact(torch, N, M):
    sp = fock.Space(N, M)
    which = fock.FOCK_MAP_SINGLE | fock.FOCK_MAP_DOUBLE
    need = fock.fock_build_jump_maps(sp.handle, which, dry_run=True)
    P = M * (M + 1) // 2
    assert need == 4 * sp.nc * (M * M + P * P)
    fock.fock_build_jump_maps(sp.handle, which)
    torch.cuda.synchronize()
    J1 = fock.fock_jump_map_get(sp.handle, fock.FOCK_MAP_SINGLE).cpu().numpy()
    ref1 = oracle.single_jump_map(N, M)                      # [g][k][l]
    assert np.array_equal(J1, ref1.reshape(sp.nc, M * M).T)
    if N < 2:
        with pytest.raises(fock.FockError):
            fock.fock_jump_map_get(sp.handle, fock.FOCK_MAP_DOUBLE)
        return
    J2 = fock.fock_jump_map_get(sp.handle, fock.FOCK_MAP_DOUBLE).cpu().numpy()  # [r*P+a][g]
    off, data = oracle.double_jump_map(N, M)
    pairs = [(k, q) for k in range(M) for q in range(k, M)]
    occ = oracle.unrank_batch(N, M, np.arange(sp.nc))
    for g in range(sp.nc):
        pos = off[g]
        for r, (k, q) in enumerate(pairs):
            ok = occ[g, k] >= 2 if k == q else (occ[g, k] >= 1 and occ[g, q] >= 1)
            if not ok:
                assert np.all(J2[r * P:(r + 1) * P, g] == -1)
                continue
            stride = data[pos:pos + M * M].reshape(M, M)
            for a, (s, l) in enumerate(pairs):
                assert J2[r * P + a, g] == stride[s, l] == stride[l, s]
            pos += M * M
        assert pos == off[g + 1]


def test_jump_maps_sampled_n20_m8(torch):
    N, M = 20, 8
    sp = fock.Space(N, M)
    fock.fock_build_jump_maps(sp.handle, fock.FOCK_MAP_SINGLE | fock.FOCK_MAP_DOUBLE)
    J1 = fock.fock_jump_map_get(sp.handle, fock.FOCK_MAP_SINGLE)
    J2 = fock.fock_jump_map_get(sp.handle, fock.FOCK_MAP_DOUBLE)
    rng = np.random.default_rng(3)
    gs = np.concatenate([[0, 1, sp.nc - 1], rng.integers(0, sp.nc, 300)])
    occ = oracle.unrank_batch(N, M, gs)
    P = M * (M + 1) // 2
    pairs = [(k, q) for k in range(M) for q in range(k, M)]
    j1 = J1[:, torch.from_numpy(gs).cuda()].cpu().numpy()
    j2 = J2[:, torch.from_numpy(gs).cuda()].cpu().numpy()
    for i, g in enumerate(gs):
        n = occ[i]
        for k in range(M):
            for l in range(M):
                if n[k] == 0:
                    assert j1[k * M + l, i] == -1
                else:
                    t = n.copy(); t[k] -= 1; t[l] += 1
                    assert j1[k * M + l, i] == oracle.rank(N, M, t)
        for r, (k, q) in enumerate(pairs):
            ok = n[k] >= 2 if k == q else (n[k] >= 1 and n[q] >= 1)
            for a, (s, l) in enumerate(pairs):
                v = j2[r * P + a, i]
                if not ok:
                    assert v == -1
                    continue
                t = n.copy(); t[k] -= 1; t[q] -= 1; t[s] += 1; t[l] += 1
                assert v == oracle.rank(N, M, t)


def test_jump_map_memory_report_large(torch):
    # Dry run only: N = 100, M = 6 (96,560,646 configurations)
    sp = fock.Space(100, 6)
    b = fock.fock_build_jump_maps(sp.handle, fock.FOCK_MAP_SINGLE | fock.FOCK_MAP_DOUBLE, dry_run=True)
    assert b == 4 * sp.nc * (36 + 21 * 21)
    assert math.isclose(b / 1e9, 184.2, rel_tol=1e-3)
