"""Every kernel path of the apply against the oracle, and the autotuner.

Each path is pinned with fock_apply_set_path; fock_apply_path reports whether
it serves the call (a path that cannot serve it falls back to the built-in
order, which the test detects and skips).  Tolerances as for the apply:
1e-12 FP64-class and native, 5e-6 FP32-mixed (relative 2-norm).
"""
import numpy as np
import pytest

import oracle
from paper_2005_13679_gb300 import fock, inputs

pytestmark = pytest.mark.gpu

TOL = {fock.FOCK_PREC_F64: 1e-12, fock.FOCK_PREC_F64_NATIVE: 1e-12, fock.FOCK_PREC_F32_MIXED: 5e-6}
PATHS = [fock.FOCK_PATH_TWOPHASE_TC, fock.FOCK_PATH_TWOPHASE, fock.FOCK_PATH_TWOPHASE_BLOCK, fock.FOCK_PATH_NN,
         fock.FOCK_PATH_DENSE, fock.FOCK_PATH_SPARSE, fock.FOCK_PATH_LIST]


@pytest.fixture(scope="module")
def torch():
    import torch as t
    fock.load()
    return t


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def dev(torch, C, prec):
    t = torch.from_numpy(np.ascontiguousarray(C))
    return (t.to(torch.complex64) if prec == fock.FOCK_PREC_F32_MIXED else t).cuda()


def pair_weight_hw(M, seed):
    """A complex operator that conserves the pair weight (W_kqsl = 0 unless
    k + q = s + l) with a complex diagonal-free h = 0: the random symmetrised
    W masked by the selection rule, plus real site energies."""
    h, W = inputs.random_hermitian_hw(M, seed)
    k, q, s_, l = np.meshgrid(*(np.arange(M),) * 4, indexing="ij")
    W = np.where(k + q == s_ + l, W, 0.0)
    return np.diag(np.diag(h).real).astype(np.complex128), W


def hw(kind, M):
    if kind == "generic":
        return inputs.random_hermitian_hw(M, 21)
    if kind == "ll":
        return inputs.lieb_liniger_hw(M, 0.9)
    if kind == "llc":
        return pair_weight_hw(M, 23)
    return inputs.nearest_neighbour_hw(M, 4, True, True)


# (N, M, kind, the paths that must serve FP64-class single-vector applies)
CASES = [
    (9, 6, "generic", {fock.FOCK_PATH_TWOPHASE_TC, fock.FOCK_PATH_TWOPHASE, fock.FOCK_PATH_DENSE,
                       fock.FOCK_PATH_SPARSE, fock.FOCK_PATH_LIST}),
    (6, 8, "generic", {fock.FOCK_PATH_TWOPHASE, fock.FOCK_PATH_DENSE, fock.FOCK_PATH_SPARSE, fock.FOCK_PATH_LIST}),
    (10, 5, "ll", {fock.FOCK_PATH_TWOPHASE_BLOCK, fock.FOCK_PATH_SPARSE, fock.FOCK_PATH_LIST}),
    (7, 10, "ll", {fock.FOCK_PATH_TWOPHASE_BLOCK, fock.FOCK_PATH_SPARSE, fock.FOCK_PATH_LIST}),
    (6, 12, "llc", {fock.FOCK_PATH_TWOPHASE_BLOCK, fock.FOCK_PATH_SPARSE, fock.FOCK_PATH_LIST}),
    (7, 6, "nn", {fock.FOCK_PATH_NN, fock.FOCK_PATH_SPARSE, fock.FOCK_PATH_LIST}),
]


@pytest.mark.parametrize("prec", list(TOL))
@pytest.mark.parametrize("N,M,kind,must", CASES)
def test_every_path_against_oracle(torch, N, M, kind, must, prec):
    h, W = hw(kind, M)
    sp = fock.Space(N, M)
    H = fock.Hamiltonian(sp, h, W)
    C = inputs.random_state(sp.nc, 8)
    ref = oracle.apply_push(N, M, h, W, C)
    served = set()
    for p in PATHS:
        fock.fock_apply_set_path(H.handle, 1, prec, p)
        if fock.fock_apply_path(sp.handle, H.handle, 1, prec) != p:
            continue
        served.add(p)
        out = H.apply(dev(torch, C, prec), precision=prec).cpu().numpy().astype(np.complex128)
        assert rel(out, ref) <= TOL[prec], fock.PATH_NAMES[p]
    fock.fock_apply_set_path(H.handle, 1, prec, fock.FOCK_PATH_AUTO)
    if prec == fock.FOCK_PREC_F64:
        assert served == must
    assert fock.FOCK_PATH_LIST in served
    if prec == fock.FOCK_PREC_F64_NATIVE:
        assert not served & {fock.FOCK_PATH_TWOPHASE_TC, fock.FOCK_PATH_TWOPHASE, fock.FOCK_PATH_TWOPHASE_BLOCK,
                             fock.FOCK_PATH_DENSE}


def test_path_query_without_workspace_and_with_maps(torch):
    N, M = 9, 6
    h, W = hw("generic", M)
    sp = fock.Space(N, M)
    H = fock.Hamiltonian(sp, h, W)
    # without the (N-2)-space workspace the two-phase paths cannot serve
    assert fock.fock_apply_path(sp.handle, H.handle, 1, fock.FOCK_PREC_F64,
                                workspace_bytes=0) == fock.FOCK_PATH_DENSE
    with pytest.raises(fock.FockError) as e:
        fock.fock_apply_path(sp.handle, H.handle, 1, fock.FOCK_PREC_F64, fock.FOCK_ARM_MAPS)
    assert e.value.status == fock.FOCK_ERR_NOT_BUILT
    fock.fock_build_jump_maps(sp.handle, fock.FOCK_MAP_SINGLE | fock.FOCK_MAP_DOUBLE)
    assert fock.fock_apply_path(sp.handle, H.handle, 1, fock.FOCK_PREC_F64, fock.FOCK_ARM_MAPS) == \
        fock.FOCK_PATH_DENSE


@pytest.mark.parametrize("prec", [fock.FOCK_PREC_F64, fock.FOCK_PREC_F32_MIXED])
def test_autotune_chooses_a_serving_path_and_caches_it(torch, tmp_path, prec):
    N, M = 20, 6
    h, W = hw("generic", M)
    sp = fock.Space(N, M)
    fock.fock_build_jump_maps(sp.handle, fock.FOCK_MAP_SINGLE | fock.FOCK_MAP_DOUBLE)
    H = fock.Hamiltonian(sp, h, W)
    cache = str(tmp_path / "tune.txt")
    t = fock.fock_autotune(sp.handle, H.handle, 1, prec, cache)
    assert t.from_cache == 0 and t.candidates >= 6 and t.ms > 0
    assert t.arm in (fock.FOCK_ARM_HASH, fock.FOCK_ARM_MAPS)
    assert fock.fock_apply_path(sp.handle, H.handle, 1, prec, t.arm) == t.path
    C = inputs.random_state(sp.nc, 9)
    ref = oracle.apply_rows(N, M, h, W, C, np.arange(0, sp.nc, 97))
    out = H.apply(dev(torch, C, prec), precision=prec).cpu().numpy().astype(np.complex128)
    assert rel(out[::97], ref) <= TOL[prec]
    # a second operator of the same shape takes the cached choice without timing
    H2 = fock.Hamiltonian(sp, h, W)
    t2 = fock.fock_autotune(sp.handle, H2.handle, 1, prec, cache)
    assert t2.from_cache == 1 and t2.candidates == 0 and (t2.path, t2.arm) == (t.path, t.arm)
    assert abs(t2.ms - t.ms) <= 1e-5 * t.ms + 1e-6
    lines = open(cache).read().strip().splitlines()
    assert len(lines) == 1 and lines[0].startswith(f"N={N} M={M} ")
    # a choice on the map arm lapses when the maps are freed
    fock.fock_apply_set_path(H.handle, 1, prec, fock.FOCK_PATH_LIST, fock.FOCK_ARM_MAPS)
    assert fock.fock_apply_path(sp.handle, H.handle, 1, prec) == fock.FOCK_PATH_LIST
    fock.fock_jump_maps_free(sp.handle)
    assert fock.fock_apply_path(sp.handle, H.handle, 1, prec) == fock.FOCK_PATH_TWOPHASE_TC
    out = H.apply(dev(torch, C, prec), precision=prec).cpu().numpy().astype(np.complex128)
    assert rel(out[::97], ref) <= TOL[prec]
    # clearing the choice restores the built-in order
    fock.fock_apply_set_path(H.handle, 1, prec, fock.FOCK_PATH_AUTO)
    assert fock.fock_apply_path(sp.handle, H.handle, 1, prec) == fock.FOCK_PATH_TWOPHASE_TC


def test_autotune_block_rhs_and_nearest_neighbour(torch):
    N, M = 12, 8
    h, W = hw("nn", M)
    sp = fock.Space(N, M)
    H = fock.Hamiltonian(sp, h, W)
    t = fock.fock_autotune(sp.handle, H.handle, 3, fock.FOCK_PREC_F64)
    assert t.candidates == 3 and t.path in (fock.FOCK_PATH_NN, fock.FOCK_PATH_SPARSE, fock.FOCK_PATH_LIST)
    # the single-vector class keeps the built-in order
    assert fock.fock_apply_path(sp.handle, H.handle, 1, fock.FOCK_PREC_F64) == fock.FOCK_PATH_NN
    Cb = np.stack([inputs.random_state(sp.nc, 60 + j) for j in range(3)], axis=1)
    out = H.apply(dev(torch, Cb, fock.FOCK_PREC_F64), nrhs=3).cpu().numpy()
    for j in range(3):
        rows = np.arange(j, sp.nc, 211)
        ref = oracle.apply_rows(N, M, h, W, Cb[:, j], rows)
        assert rel(out[rows, j], ref) <= 1e-12


def test_operator_forms(torch):
    """The structure the library finds in an operator: generic dense W, the
    Lieb-Liniger contact interaction (pair weight conserved, rank one inside
    every pair-momentum block), a pair-weight operator that is not of contact
    form, and the Bose-Hubbard ring."""
    F = fock
    sp = fock.Space(6, 5)
    h, W = inputs.random_hermitian_hw(5, 3)
    assert fock.Hamiltonian(sp, h, W).forms & F.FOCK_FORM_DENSE
    h, W = inputs.lieb_liniger_hw(5, 0.7)
    f = fock.Hamiltonian(sp, h, W).forms
    assert f & F.FOCK_FORM_PAIR_WEIGHT and f & F.FOCK_FORM_PAIR_MOMENTUM and not f & F.FOCK_FORM_DENSE
    W2 = W.copy()
    # one coupling of the block K = 4 ({0,4}, {1,3}, {2,2}) changed: k + q = s + l
    # still holds, the block is no longer rank one off its diagonal
    for k, q, s, l in ((0, 4, 1, 3), (1, 3, 0, 4)):
        W2[k, q, s, l] = W2[q, k, l, s] = W2[k, q, l, s] = W2[q, k, s, l] = 0.3
    f2 = fock.Hamiltonian(sp, h, W2).forms
    assert f2 & F.FOCK_FORM_PAIR_WEIGHT and not f2 & F.FOCK_FORM_PAIR_MOMENTUM
    h, W = inputs.bose_hubbard_hw(5, 1.0, 4.0)
    assert fock.Hamiltonian(sp, h, W).forms & F.FOCK_FORM_NEAREST_NEIGHBOUR
