"""GPU parity of sigma = H C (Eq. Haction) against the oracle, through the C ABI.

Tolerances (relative 2-norm of the difference, ||sigma - sigma_ref|| / ||sigma_ref||):
  FOCK_PREC_F64 (FP32-pair arithmetic) and FOCK_PREC_F64_NATIVE: 1e-12, the
  target the FP64 apply must meet; FP32-pair values carry 48-bit significands,
  so the expected error is a few 1e-15.
  FOCK_PREC_F32_MIXED: 5e-6; inputs rounded to complex64 carry 2^-24 relative
  error each and FP32 products add the same order, so a few 1e-7 is expected.
"""
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


def dev_vec(torch, C, prec):
    t = torch.from_numpy(np.ascontiguousarray(C))
    if prec == fock.FOCK_PREC_F32_MIXED:
        t = t.to(torch.complex64)
    return t.cuda()


def hw(kind, M, seed=7, g=1.0):
    if kind == "ll":
        return inputs.lieb_liniger_hw(M, g)
    if kind == "bh":
        return inputs.bose_hubbard_hw(M, 1.0, 3.0, 0.3)
    if kind == "onebody":
        h, _ = inputs.random_hermitian_hw(M, seed)
        return h, None
    return inputs.random_hermitian_hw(M, seed)


# (N, M, kind): several tiles of 128 configurations with a ragged tail, the
# degenerate spaces (N = 1, M = 1, N = 2) and both sparse and dense W.
SMALL = [
    (6, 6, "generic"),      # 462 configurations
    (8, 6, "generic"),      # 1287
    (10, 5, "ll"),          # 1001
    (5, 10, "ll"),          # 2002, most orbitals empty
    (7, 4, "generic"),      # 120
    (1, 7, "generic"),      # one particle: one-body part only
    (2, 5, "generic"),      # smallest N with a two-body part
    (9, 1, "generic"),      # one orbital, one configuration
    (12, 3, "onebody"),     # W absent
    (4, 12, "ll"),          # largest M
    (3, 9, "generic"),
]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("N,M,kind", SMALL)
def test_apply_full_vector(torch, N, M, kind, prec):
    h, W = hw(kind, M)
    sp = fock.Space(N, M)
    H = fock.Hamiltonian(sp, h, W)
    C = inputs.random_state(sp.nc, 11)
    ref = oracle.apply_push(N, M, h, W, C)
    out = H.apply(dev_vec(torch, C, prec), precision=prec)
    torch.cuda.synchronize()
    assert rel(out.cpu().numpy().astype(np.complex128), ref) <= TOL[prec]


@pytest.mark.parametrize("prec", PRECS)
def test_apply_scale_invariance(torch, prec):
    # The FP32-pair path rescales C by a power of two; extreme magnitudes
    # must not lose accuracy (FP32 storage has its own range, tested at 1e-20).
    N, M = 6, 5
    h, W = hw("generic", M)
    sp = fock.Space(N, M)
    H = fock.Hamiltonian(sp, h, W)
    C = inputs.random_state(sp.nc, 5)
    ref = oracle.apply_push(N, M, h, W, C)
    scales = [1e-20, 1e20] if prec == fock.FOCK_PREC_F32_MIXED else [1e-250, 1e-40, 1e40, 1e250]
    for s in scales:
        out = H.apply(dev_vec(torch, C * s, prec), precision=prec).cpu().numpy().astype(np.complex128)
        assert rel(out / s, ref) <= TOL[prec], s
    zero = H.apply(dev_vec(torch, np.zeros_like(C), prec), precision=prec).cpu().numpy()
    assert np.all(zero == 0)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("nrhs", [1, 3, 16])
def test_block_rhs_matches_single(torch, prec, nrhs):
    N, M = 8, 6
    h, W = hw("generic", M, seed=4)
    sp = fock.Space(N, M)
    H = fock.Hamiltonian(sp, h, W)
    B = inputs.random_block(sp.nc, range(40, 40 + nrhs))
    out = H.apply(dev_vec(torch, B, prec), nrhs=nrhs, precision=prec).cpu().numpy().astype(np.complex128)
    for j in range(nrhs):
        ref = oracle.apply_push(N, M, h, W, B[:, j])
        assert rel(out[:, j], ref) <= TOL[prec]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("N,M,kind", [(6, 6, "generic"), (10, 5, "ll"), (1, 5, "generic"), (12, 3, "onebody")])
def test_maps_arm_equals_hash_arm(torch, N, M, kind, prec):
    h, W = hw(kind, M)
    sp = fock.Space(N, M)
    H = fock.Hamiltonian(sp, h, W)
    C = dev_vec(torch, inputs.random_state(sp.nc, 9), prec)
    with pytest.raises(fock.FockError) as e:
        H.apply(C, precision=prec, arm=fock.FOCK_ARM_MAPS)
    assert e.value.status == fock.FOCK_ERR_NOT_BUILT
    fock.fock_build_jump_maps(sp.handle, fock.FOCK_MAP_SINGLE | fock.FOCK_MAP_DOUBLE)
    a = H.apply(C, precision=prec, arm=fock.FOCK_ARM_HASH)
    b = H.apply(C, precision=prec, arm=fock.FOCK_ARM_MAPS)
    ref = oracle.apply_push(N, M, h, W, C.cpu().numpy().astype(np.complex128))
    for out in (a, b):
        assert rel(out.cpu().numpy().astype(np.complex128), ref) <= TOL[prec]
    if kind == "ll":
        # the sparse kernel on both arms: same arithmetic order, bit-identical
        # sums (left to itself the hash arm takes the pair-weight two-phase
        # path, and the one-body M = 3 case the nearest-neighbour kernel:
        # every pair of three sites neighbours on a ring)
        fock.fock_apply_set_path(H.handle, 1, prec, fock.FOCK_PATH_SPARSE, fock.FOCK_ARM_HASH)
        a = H.apply(C, precision=prec, arm=fock.FOCK_ARM_HASH)
        fock.fock_apply_set_path(H.handle, 1, prec, fock.FOCK_PATH_AUTO)
        assert torch.equal(a, b)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("N,M", [(6, 4), (4, 7), (9, 3), (3, 12)])
def test_bose_hubbard_against_oracle(torch, N, M, prec):
    h, W = inputs.bose_hubbard_hw(M, J=1.0, U=3.5, mu=0.2)
    sp = fock.Space(N, M)
    H = fock.Hamiltonian(sp, h, W)
    C = inputs.random_state(sp.nc, 23)
    ref = oracle.apply_push(N, M, h, W, C)
    out = H.apply(dev_vec(torch, C, prec), precision=prec)
    assert rel(out.cpu().numpy().astype(np.complex128), ref) <= TOL[prec]


# Nearest-neighbour operators take their own kernel (one diagonal term and two
# hops per bond); chains and rings, real and complex hops, M = 2 (one bond),
# M = 3 (every pair neighbouring), several tiles with a ragged tail.
NN_CASES = [
    (9, 6, True, True),     # 2002 configurations
    (9, 6, False, False),
    (10, 8, True, False),   # 19448
    (5, 2, False, True),
    (7, 3, True, True),
    (3, 12, True, True),
    (1, 5, True, True),
    (6, 1, False, False),   # one site: no bond, generic path
]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("N,M,ring,cplx", NN_CASES)
def test_nearest_neighbour_against_oracle(torch, N, M, ring, cplx, prec):
    h, W = inputs.nearest_neighbour_hw(M, 11 + N + M, ring, cplx)
    sp = fock.Space(N, M)
    H = fock.Hamiltonian(sp, h, W)
    C = inputs.random_state(sp.nc, 29)
    ref = oracle.apply_push(N, M, h, W, C)
    out = H.apply(dev_vec(torch, C, prec), precision=prec)
    assert rel(out.cpu().numpy().astype(np.complex128), ref) <= TOL[prec]
    # without W: one-body hops and site energies only
    H1 = fock.Hamiltonian(sp, h, None)
    ref1 = oracle.apply_push(N, M, h, None, C)
    out1 = H1.apply(dev_vec(torch, C, prec), precision=prec)
    assert rel(out1.cpu().numpy().astype(np.complex128), ref1) <= TOL[prec]


@pytest.mark.parametrize("prec", PRECS)
def test_nearest_neighbour_block_and_maps(torch, prec):
    """Block right-hand sides against single applies, and the hash arm (the
    nearest-neighbour kernel) against the jump-map arm (the generic kernels)."""
    N, M, nrhs = 8, 7, 3
    h, W = inputs.nearest_neighbour_hw(M, 5, True, True)
    sp = fock.Space(N, M)
    fock.fock_build_jump_maps(sp.handle, fock.FOCK_MAP_SINGLE | fock.FOCK_MAP_DOUBLE)
    H = fock.Hamiltonian(sp, h, W)
    Cb = np.stack([inputs.random_state(sp.nc, 40 + j) for j in range(nrhs)], axis=1)
    out = H.apply(dev_vec(torch, Cb, prec), nrhs=nrhs, precision=prec).cpu().numpy().astype(np.complex128)
    for j in range(nrhs):
        one = H.apply(dev_vec(torch, Cb[:, j], prec), precision=prec).cpu().numpy().astype(np.complex128)
        assert rel(out[:, j], one) <= TOL[prec]
        maps = H.apply(dev_vec(torch, Cb[:, j], prec), precision=prec, arm=fock.FOCK_ARM_MAPS)
        assert rel(one, maps.cpu().numpy().astype(np.complex128)) <= TOL[prec]


def test_alias_and_argument_errors(torch):
    sp = fock.Space(5, 5)
    h, W = hw("ll", 5)
    H = fock.Hamiltonian(sp, h, W)
    C = dev_vec(torch, inputs.random_state(sp.nc, 1), fock.FOCK_PREC_F64)
    with pytest.raises(fock.FockError) as e:
        H.apply(C, sigma=C)
    assert e.value.status == fock.FOCK_ERR_ALIAS
    with pytest.raises(fock.FockError):
        H.apply(C, nrhs=17)
    with pytest.raises(fock.FockError) as e:
        fock.Hamiltonian(sp, h + np.triu(np.ones((5, 5)), 1), W)
    assert e.value.status == fock.FOCK_ERR_NOT_HERMITIAN


def test_terms_count_matches_oracle_columns(torch):
    for N, M, kind in [(6, 6, "generic"), (10, 5, "ll"), (1, 7, "generic")]:
        h, W = hw(kind, M)
        sp = fock.Space(N, M)
        H = fock.Hamiltonian(sp, h, W)
        # Column term counts of the oracle count ordered operator strings; the
        # library counts one term per distinct (removal, addition) multiset
        # pair, plus the diagonal and the off-diagonal one-body jumps.
        P = M * (M + 1) // 2
        Ws = np.zeros((P, P), dtype=np.complex128)
        pairs = {(k, q): i for i, (k, q) in enumerate((k, q) for k in range(M) for q in range(k, M))}
        if W is not None and N >= 2:
            for k in range(M):
                for q in range(M):
                    for s in range(M):
                        for l in range(M):
                            Ws[pairs[(min(k, q), max(k, q))], pairs[(min(s, l), max(s, l))]] += W[k, q, s, l]
        nz = int(np.count_nonzero(Ws))
        offh = int(np.count_nonzero(h - np.diag(np.diag(h))))
        expect = sp.nc + oracle.nc(N - 1, M) * offh + (oracle.nc(N - 2, M) * nz if N >= 2 else 0)
        assert H.terms == expect


@pytest.mark.parametrize("prec", [fock.FOCK_PREC_F64, fock.FOCK_PREC_F32_MIXED])
@pytest.mark.parametrize("N,M,kind,nrhs,pinned", [
    (8, 6, "generic", 1, True),      # two-phase on the tensor cores, sigma copied out by chunks
    (9, 6, "generic", 3, False),     # several right-hand sides, pageable host memory
    (6, 8, "generic", 1, True),      # two-phase with FP32 phase 1
    (10, 5, "ll", 2, True),          # pair-weight two-phase: input and sigma copied by chunks
    (16, 10, "ll", 1, True),
    (9, 6, "bh", 1, True),           # nearest-neighbour kernel, sigma copied out by chunks
    (8, 7, "bh", 3, False),
])
def test_host_buffer_entry_point(torch, N, M, kind, nrhs, pinned, prec):
    h, W = hw(kind, M)
    sp = fock.Space(N, M)
    H = fock.Hamiltonian(sp, h, W)
    C = np.stack([inputs.random_state(sp.nc, 2 + j) for j in range(nrhs)], axis=1)
    Ch = torch.from_numpy(np.ascontiguousarray(C))
    if prec == fock.FOCK_PREC_F32_MIXED:
        Ch = Ch.to(torch.complex64)
    out = torch.empty_like(Ch)
    if pinned:
        Ch, out = Ch.pin_memory(), out.pin_memory()
    fock.fock_apply_H_host(sp.handle, H.handle, Ch, out, nrhs=nrhs, precision=prec)
    dev_out = H.apply(Ch.cuda(), nrhs=nrhs, precision=prec).cpu()
    assert torch.equal(out, dev_out)              # same kernels, same sums
    for j in range(nrhs):
        ref = oracle.apply_push(N, M, h, W, C[:, j])
        assert rel(out.numpy().reshape(sp.nc, nrhs)[:, j].astype(np.complex128), ref) <= TOL[prec]


@pytest.mark.parametrize("scale", [1e-30, 1e9])
def test_host_buffer_outside_the_unscaled_band(torch, scale):
    # the host-buffer apply splits C chunk by chunk without a scale, which is
    # exact while the largest magnitude lies in [2^-20, 2^21); outside it the
    # call applies again from its device copy with the scaled split, so it
    # still equals the device apply bit for bit
    N, M = 8, 6
    h, W = hw("generic", M)
    sp = fock.Space(N, M)
    H = fock.Hamiltonian(sp, h, W)
    C = inputs.random_state(sp.nc, 12) * scale
    Ch = torch.from_numpy(C).pin_memory()
    out = torch.empty_like(Ch).pin_memory()
    fock.fock_apply_H_host(sp.handle, H.handle, Ch, out)
    assert torch.equal(out, H.apply(Ch.cuda()).cpu())
    assert rel(out.numpy(), oracle.apply_push(N, M, h, W, C)) <= 1e-12


# ---------------------------------------------------------------------------
# Full-size workloads in the launch configuration of the benchmark: sampled
# rows against the oracle's row form, plus properties at full size.
# ---------------------------------------------------------------------------
def sampled_rows(nc, seed, count):
    rng = np.random.default_rng(seed)
    edge = np.concatenate([np.arange(min(512, nc)), nc - 1 - np.arange(min(512, nc))])
    return np.unique(np.concatenate([edge, rng.integers(0, nc, count)])).astype(np.int64)


@pytest.mark.parametrize("name", ["generic_n100_m6", "ll_n30_m10", "ll_n5_m5", "bh_n20_m12"])
def test_full_size_sampled_rows(torch, name):
    w = inputs.WORKLOADS[name]
    h, W = w.hamiltonian()
    sp = fock.Space(w.N, w.M)
    H = fock.Hamiltonian(sp, h, W)
    C = w.state()
    rows = sampled_rows(sp.nc, 1, 3000)
    ref = oracle.apply_rows(w.N, w.M, h, W, C, rows)
    Cd = torch.from_numpy(C).cuda()
    del C
    sig = H.apply(Cd, precision=fock.FOCK_PREC_F64)
    got = sig[torch.from_numpy(rows).cuda()].cpu().numpy()
    assert rel(got, ref) <= 1e-12
    # Hermiticity at full size: <C, H C> is real
    q = torch.vdot(Cd, sig).item()
    assert abs(q.imag) <= 1e-12 * abs(q)
    del sig
    sig32 = H.apply(Cd.to(torch.complex64), precision=fock.FOCK_PREC_F32_MIXED)
    got32 = sig32[torch.from_numpy(rows).cuda()].cpu().numpy().astype(np.complex128)
    assert rel(got32, ref) <= 5e-6


def test_full_size_block_rhs_n20_m8(torch):
    w = inputs.WORKLOADS["generic_n20_m8_rhs16"]
    h, W = w.hamiltonian()
    sp = fock.Space(w.N, w.M)
    H = fock.Hamiltonian(sp, h, W)
    B = w.state()
    rows = sampled_rows(sp.nc, 2, 1500)
    Bd = torch.from_numpy(B).cuda()
    blk = H.apply(Bd, nrhs=16, precision=fock.FOCK_PREC_F64)
    for j in (0, 7, 15):
        ref = oracle.apply_rows(w.N, w.M, h, W, B[:, j], rows)
        got = blk[:, j][torch.from_numpy(rows).cuda()].cpu().numpy()
        assert rel(got, ref) <= 1e-12
        one = H.apply(Bd[:, j].contiguous(), precision=fock.FOCK_PREC_F64)
        assert torch.allclose(one, blk[:, j], rtol=0, atol=1e-13)


def test_full_vector_fp32_pair_against_native(torch):
    """All 8,259,888 rows of the generic N = 60, M = 6 workload: the FP64-class
    path (tensor-core phase 1, FP32-pair phase 2, integer conversions at both
    ends) against the native FP64 arm, which the small cases pin to the oracle.
    Every row is checked, so a rare failure (a cancellation, a rounding carry,
    an extreme exponent) cannot hide between sampled rows."""
    w = inputs.WORKLOADS["generic_n60_m6"]
    h, W = w.hamiltonian()
    sp = fock.Space(w.N, w.M)
    H = fock.Hamiltonian(sp, h, W)
    Cd = torch.from_numpy(w.state()).cuda()
    a = H.apply(Cd, precision=fock.FOCK_PREC_F64)
    b = H.apply(Cd, precision=fock.FOCK_PREC_F64_NATIVE)
    scale = b.abs().max().item()
    assert (torch.linalg.norm(a - b) / torch.linalg.norm(b)).item() <= 1e-12
    assert (a - b).abs().max().item() <= 1e-11 * scale

