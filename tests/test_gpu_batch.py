"""Uneven batches (one persistent launch over the small problems, an apply of
its own for each large one) through the C ABI: the batched apply against the
oracle and against single-problem applies, the autotuner, and the batched
Lanczos against dense diagonalisation and the single-problem solver."""
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


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def small_problems():
    # uneven sizes, M from 4 to 12, one generic complex problem and one
    # one-body problem among Lieb-Liniger rings
    probs = []
    for N, M, g in [(6, 4, 0.3), (9, 5, 2.0), (4, 12, 1.0), (7, 6, 7.5), (3, 9, 0.1), (12, 3, 1.0)]:
        h, W = inputs.lieb_liniger_hw(M, g)
        probs.append((N, M, h, W))
    h, W = inputs.random_hermitian_hw(5, 8)
    probs.append((6, 5, h, W))
    h1, _ = inputs.random_hermitian_hw(4, 9)
    probs.append((5, 4, h1, None))
    return probs


@pytest.mark.parametrize("prec", [fock.FOCK_PREC_F64, fock.FOCK_PREC_F32_MIXED])
def test_batch_apply_matches_oracle_and_single(torch, prec):
    probs = small_problems()
    B = fock.Batch(probs)
    C = np.concatenate([inputs.random_state(oracle.nc(N, M), 100 + i) for i, (N, M, _, _) in enumerate(probs)])
    dt = torch.complex128 if prec == fock.FOCK_PREC_F64 else torch.complex64
    Cd = torch.from_numpy(C).to(dt).cuda()
    out = B.apply(Cd, precision=prec).cpu().numpy().astype(np.complex128)
    tol = 1e-12 if prec == fock.FOCK_PREC_F64 else 5e-6
    for i, (N, M, h, W) in enumerate(probs):
        a, b = B.offsets[i], B.offsets[i + 1]
        ref = oracle.apply_push(N, M, h, W, C[a:b])
        assert rel(out[a:b], ref) <= tol, i
        sp = fock.Space(N, M)
        H = fock.Hamiltonian(sp, h, W)
        one = H.apply(Cd[a:b].contiguous(), precision=prec).cpu().numpy().astype(np.complex128)
        assert rel(out[a:b], one) <= tol
    assert B.terms == sum(fock.Hamiltonian(fock.Space(N, M), h, W).terms for N, M, h, W in probs)


@pytest.mark.parametrize("prec", [fock.FOCK_PREC_F64, fock.FOCK_PREC_F32_MIXED])
def test_batch_own_and_shared_instances(torch, prec):
    """Instances of 2^18 configurations or more whose default path is a
    two-phase one are applied by that path (a generic M = 6 problem on the
    tensor-core phase 1, a Lieb-Liniger ring on the pair-weight form), the
    rest by the persistent launch; both against the oracle on sampled rows
    (every row of the small instances) and against the single-problem apply."""
    probs = small_problems()[:3]
    h, W = inputs.random_hermitian_hw(6, 21)
    probs.append((30, 6, h, W))                               # 324632 configurations
    probs.append((30, 7) + inputs.lieb_liniger_hw(7, 1.3))   # 1947792 configurations
    B = fock.Batch(probs)
    assert list(B.own) == [False, False, False, True, True]
    C = np.concatenate([inputs.random_state(oracle.nc(N, M), 200 + i) for i, (N, M, _, _) in enumerate(probs)])
    C[B.offsets[3]:B.offsets[4]] *= 1e5                       # scaled on its own
    dt = torch.complex128 if prec == fock.FOCK_PREC_F64 else torch.complex64
    Cd = torch.from_numpy(C).to(dt).cuda()
    out = B.apply(Cd, precision=prec).cpu().numpy().astype(np.complex128)
    tol = 1e-12 if prec == fock.FOCK_PREC_F64 else 5e-6
    rng = np.random.default_rng(3)
    for i, (N, M, h, W) in enumerate(probs):
        a, b = B.offsets[i], B.offsets[i + 1]
        if b - a <= 20000:
            rows = np.arange(b - a)
        else:
            rows = np.unique(np.concatenate([rng.integers(0, b - a, 800), np.arange(100), np.arange(b - a - 100, b - a)]))
        ref = oracle.apply_rows(N, M, h, W, C[a:b], rows)
        assert rel(out[a:b][rows], ref) <= tol, i
        sp = fock.Space(N, M)
        H = fock.Hamiltonian(sp, h, W)
        one = H.apply(Cd[a:b].contiguous(), precision=prec).cpu().numpy().astype(np.complex128)
        assert rel(out[a:b], one) <= tol, i


def test_batch_autotune_keeps_results(torch, tmp_path):
    probs = small_problems()
    B = fock.Batch(probs)
    C = torch.from_numpy(inputs.random_state(B.total, 3)).cuda()
    before = B.apply(C)
    out = torch.empty_like(C)
    t, b = B.autotune(C, out, cache_path=tmp_path / "tune.txt")
    assert t in (1, 2, 4, 8, 16, 32) and b in (0, 1, 2, 3)
    after = B.apply(C)
    assert torch.equal(before, after)        # item order never changes a configuration's sum
    assert (tmp_path / "tune.txt").read_text().count("tiles") == 1
    t2, b2 = B.autotune(C, out, cache_path=tmp_path / "tune.txt")   # served from the cache
    assert (t2, b2) == (t, b)


def test_batch_lanczos_against_dense(torch):
    probs = [p for p in small_problems() if oracle.nc(p[0], p[1]) <= 1500]
    B = fock.Batch(probs)
    E, R, it, st = B.lanczos_ground(max_iter=600, restart_len=16, tol=1e-12, seed=5)
    assert st == fock.FOCK_OK
    for i, (N, M, h, W) in enumerate(probs):
        Ed = np.linalg.eigvalsh(oracle.dense_hamiltonian(N, M, h, W))[0]
        assert abs(E[i] - Ed) <= 1e-10 * max(1.0, abs(Ed)), (i, E[i], Ed)
        assert R[i] <= 1e-6 * max(1.0, abs(Ed))


def test_batch_lanczos_uneven_ll(torch):
    """Uneven Lieb-Liniger instances (cap 10^6 configurations; all but one
    with an apply of their own, stopping at different cycles): every energy
    matches the single-problem solver to 1e-10 and lies between the
    Bethe-ansatz energy and the zero-momentum condensate energy."""
    inst = inputs.uneven_ll_batch(count=12, seed=5, cap=10 ** 6)
    probs = [(x.N, x.M) + inputs.lieb_liniger_hw(x.M, x.g) for x in inst]
    B = fock.Batch(probs)
    assert B.own.sum() == len(inst) - 1      # the 286-configuration instance stays in the shared launch
    E, R, it, st = B.lanczos_ground(max_iter=400, restart_len=12, tol=1e-10, seed=9)
    assert st == fock.FOCK_OK
    for i, x in enumerate(inst):
        Eb, _ = oracle.bethe_ground_energy(x.N, x.g)
        assert Eb < E[i] <= x.g * x.N * (x.N - 1) / 2.0 + 1e-9
        assert R[i] <= 1e-5 * abs(E[i])
    for i in (0, len(inst) - 1):
        x = inst[i]
        sp = fock.Space(x.N, x.M)
        H = fock.Hamiltonian(sp, *inputs.lieb_liniger_hw(x.M, x.g))
        E1, _, _, _, st1 = fock.fock_lanczos_ground(sp.handle, H.handle, max_iter=600, restart_len=24, tol=1e-10,
                                                    seed=4)
        assert st1 == fock.FOCK_OK
        assert abs(E[i] - E1) <= 1e-10 * abs(E1)
