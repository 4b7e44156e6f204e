"""Accuracy of the FP64-class apply (FOCK_PREC_F64) where the product cancels.

sigma = H C (Eq. Haction) factors through the (N-2)-particle configurations
n' = gamma - r of the removal pairs r = {k, q}:

    sigma_gamma = sum_r A_r(gamma) Y_r(n'),   Y_r(n') = sum_a R[r][a] X_a(n'),
    X_a(n') = B_a(n') C[n' + a],  A_r = sqrt(n_k (n_q - d_kq)),  B_a = sqrt((n'_s + 1)(n'_l + 1 + d_sl)),

with R the operator reduced to pairs of multisets (W summed over the
orderings, halved, and h folded in through sum_x a^dag_k a^dag_x a_x a_l =
(N - 1) a^dag_k a_l).  The tensor-core phase 1 has the a-priori bound
|dY| <= 2^-40.5 ||R~_r||_1 max_k |X_k(n')| per real component (R~ the real
form of R, X_k the 2P real parts of the column), so sqrt(2) times that for
the complex entry, and phase 2 adds in FP32 pairs (below 2^-46 B), so every
entry must satisfy

    |sigma^ - sigma| <= 2^-39.9 B_gamma + 2^-44 (|H| |C|)_gamma,
    B_gamma = sum_r |A_r(gamma)| ||R~_r||_1 max_k |X_k(gamma - r)|,

the second term covering the oracle's own FP64 rounding.  B is computed here
from h, W and C alone (the reduction is checked against the oracle first).
The cases are built so that |sigma| is far below B: an operator shifted by
its ground energy applied to its ground vector, a reduced coefficient row with
one dominant entry, and C spanning thirty orders of magnitude.  The bound is a
worst case (it adds every term's error with the same sign): on a random state
it implies a few 1e-11 normwise, while the measured error is 1e-13.  So
the normwise 1e-12 of the apply's contract is asserted on the measured error
for the cases where sigma does not cancel (random, dominant row, wide range),
and the shifted ground vector, where |sigma| is 10^-3..10^-14 of |H||C|, is
held to the element-wise bound alone.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_2005_13679_gb300 import fock, inputs

pytestmark = pytest.mark.gpu

FP64_PATHS = [fock.FOCK_PATH_TWOPHASE_TC, fock.FOCK_PATH_TWOPHASE, fock.FOCK_PATH_DENSE, fock.FOCK_PATH_SPARSE,
              fock.FOCK_PATH_LIST]


@pytest.fixture(scope="module")
def torch():
    import torch as t
    fock.load()
    return t


def pairs_of(M):
    return [(k, q) for k in range(M) for q in range(k, M)]


def reduced(N, M, h, W):
    pr = pairs_of(M)
    idx = {p: i for i, p in enumerate(pr)}
    R = np.zeros((len(pr), len(pr)), dtype=np.complex128)
    key = lambda a, b: idx[(min(a, b), max(a, b))]
    for k, q, s, l in itertools.product(range(M), repeat=4):
        R[key(k, q), key(s, l)] += 0.5 * W[k, q, s, l]
    for k, x, l in itertools.product(range(M), repeat=3):
        R[key(k, x), key(x, l)] += h[k, l] / (N - 1)
    return pr, R


def factored(N, M, h, W, C, rows):
    """sigma on `rows` by the factorisation (used only to check `reduced`), and
    the bound B on the same rows."""
    pr, R = reduced(N, M, h, W)
    Rn = np.sum(np.abs(R.real) + np.abs(R.imag), axis=1)
    occ = oracle.unrank_batch(N, M, rows)
    sig = np.zeros(len(rows), dtype=np.complex128)
    B = np.zeros(len(rows))
    for ri, (k, q) in enumerate(pr):
        npr = occ.copy()
        npr[:, k] -= 1
        npr[:, q] -= 1
        ok = np.all(npr >= 0, axis=1)
        A = np.sqrt(np.where(ok, occ[:, k] * (occ[:, q] - (k == q)), 0).astype(np.float64))
        safe = np.where(ok[:, None], npr, 0)
        safe[:, 0] += np.where(ok, 0, N - 2)                # any valid (N-2)-configuration
        Y = np.zeros(len(rows), dtype=np.complex128)
        mx = np.zeros(len(rows))
        for ai, (s, l) in enumerate(pr):
            t = safe.copy()
            t[:, s] += 1
            t[:, l] += 1
            amp = np.sqrt((safe[:, s] + 1.0) * (safe[:, l] + 1.0 + (s == l)))
            x = amp * C[oracle.rank_batch(N, M, t)]
            Y += R[ri, ai] * x
            mx = np.maximum(mx, np.maximum(np.abs(x.real), np.abs(x.imag)))
        sig += A * Y
        B += A * Rn[ri] * mx
    return sig, B


def tolerance(N, M, h, W, C, rows):
    sig_f, B = factored(N, M, h, W, C, rows)
    absHC = oracle.apply_rows(N, M, np.abs(h), np.abs(W), np.abs(C), rows).real
    return sig_f, 2.0 ** -39.9 * B + 2.0 ** -44 * absHC


def check(torch, N, M, h, W, C, rows=None, paths=FP64_PATHS, normwise=True):
    """Every FP64-class path that serves the apply, element by element within
    the bound and (normwise=True) within 1e-12 in relative 2-norm; returns
    {path: (worst error / tolerance, normwise error, bound-implied normwise
    error)}."""
    sp = fock.Space(N, M)
    H = fock.Hamiltonian(sp, h, W)
    if rows is None:
        rows = np.arange(sp.nc)
        ref = oracle.apply_push(N, M, h, W, C)
    else:
        ref = oracle.apply_rows(N, M, h, W, C, rows)
    sig_f, tol = tolerance(N, M, h, W, C, rows)
    assert np.linalg.norm(sig_f - ref) <= 1e-12 * max(np.linalg.norm(ref), 1e-300) + np.linalg.norm(tol)
    out = {}
    for p in paths:
        fock.fock_apply_set_path(H.handle, 1, fock.FOCK_PREC_F64, p)
        if fock.fock_apply_path(sp.handle, H.handle, 1, fock.FOCK_PREC_F64) != p:
            continue
        got = H.apply(torch.from_numpy(C).cuda(), precision=fock.FOCK_PREC_F64).cpu().numpy()[rows]
        err = np.abs(got - ref)
        worst = float(np.max(err / tol))
        assert worst <= 1.0, (fock.PATH_NAMES[p], worst)
        nref = np.linalg.norm(ref)
        out[p] = (worst, float(np.linalg.norm(err) / nref) if nref > 0 else 0.0,
                  float(np.linalg.norm(tol) / nref) if nref > 0 else np.inf)
    fock.fock_apply_set_path(H.handle, 1, fock.FOCK_PREC_F64, fock.FOCK_PATH_AUTO)
    assert fock.FOCK_PATH_TWOPHASE_TC in out or M > 6
    for p, (worst, rel, implied) in out.items():
        print(f"{fock.PATH_NAMES[p]}: worst err/bound {worst:.2e}, normwise {rel:.2e}, bound-implied {implied:.2e}")
        if normwise:
            assert rel <= 1e-12, (fock.PATH_NAMES[p], rel)
    return out


def shifted_ground(N, M, seed, delta):
    """h shifted on the diagonal by -(E0 - delta)/N, so that H - E0 + delta
    acts on the ground vector C0 of H as delta C0 (sum_k a^dag_k a_k = N)."""
    h, W = inputs.random_hermitian_hw(M, seed)
    Hd = oracle.dense_hamiltonian(N, M, h, W)
    w, v = np.linalg.eigh(Hd)
    hs = h - np.eye(M) * (w[0] - delta) / N
    return hs, W, np.ascontiguousarray(v[:, 0])


def test_random_state_small(torch):
    N, M = 8, 6
    h, W = inputs.random_hermitian_hw(M, 41)
    check(torch, N, M, h, W, inputs.random_state(oracle.nc(N, M), 5))


@pytest.mark.parametrize("delta_rel", [0.0, 1e-6, 1e-3])
def test_shifted_ground_vector(torch, delta_rel):
    N, M = 8, 6
    h, W = inputs.random_hermitian_hw(M, 43)
    E0 = np.linalg.eigvalsh(oracle.dense_hamiltonian(N, M, h, W))[0]
    hs, W, C0 = shifted_ground(N, M, 43, delta_rel * abs(E0))
    check(torch, N, M, hs, W, C0, normwise=False)


def dominant_row_operator(M, seed, big=1.0, small=1e-6):
    """A Hermitian, boson-symmetric W whose reduced row {0, 1} is one entry
    ({2, 3}, and its conjugate) of size `big`, everything else `small` times
    a random symmetrised draw; h likewise small."""
    h, W = inputs.random_hermitian_hw(M, seed)
    h = h * small
    W = W * small
    z = big * np.exp(0.7j)
    for k, q in ((0, 1), (1, 0)):
        for s, l in ((2, 3), (3, 2)):
            W[k, q, s, l] += z
            W[s, l, k, q] += np.conj(z)
    return h, W


def test_dominant_coefficient_row(torch):
    N, M = 9, 6
    h, W = dominant_row_operator(M, 45)
    check(torch, N, M, h, W, inputs.random_state(oracle.nc(N, M), 6))


def wide_range_state(nc, seed, decades=30):
    rng = np.random.default_rng(seed)
    C = (rng.standard_normal(nc) + 1j * rng.standard_normal(nc)) * 10.0 ** rng.uniform(-decades, 0, nc)
    return C / np.linalg.norm(C)


def test_wide_range_state(torch):
    N, M = 9, 6
    h, W = inputs.random_hermitian_hw(M, 47)
    check(torch, N, M, h, W, wide_range_state(oracle.nc(N, M), 7))


@pytest.mark.parametrize("kind", ["random", "dominant", "wide"])
def test_n60_sampled_rows(torch, kind):
    N, M = 60, 6
    if kind == "dominant":
        h, W = dominant_row_operator(M, 49)
    else:
        h, W = inputs.random_hermitian_hw(M, 2)
    nc = oracle.nc(N, M)
    C = wide_range_state(nc, 9) if kind == "wide" else inputs.random_state(nc, 9)
    rng = np.random.default_rng(11)
    rows = np.unique(np.concatenate([rng.integers(0, nc, 1500), np.arange(200), np.arange(nc - 200, nc)]))
    check(torch, N, M, h, W, C, rows=rows, paths=[fock.FOCK_PATH_TWOPHASE_TC])
