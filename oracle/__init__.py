"""Plain, slow CPU oracle for the bosonic Fock-space Hamiltonian apply.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The product
library (``paper_2005_13679_gb300``) never imports it and shares no code with
it; the two meet only through the seeded input generators, which hold none of
the method's arithmetic.

Contents (Andriati & Gammal, arXiv:2005.13679):

* ``nc``, ``rank``, ``unrank`` -- Eq. nc, Algorithm 1, Algorithm 2 (C, in
  ``fock_oracle.c``);
* ``single_jump_map``, ``double_jump_map`` -- the jump maps of Sec. 4, built by
  definition (unrank, move particles, rank);
* ``apply_push``, ``apply_rows``, ``dense_hamiltonian`` -- sigma = H C of
  Eq. Haction from the operator strings of Eqs. noninteracting/interacting;
* ``column_terms`` -- the number of those operator strings that survive on one
  configuration (the per-configuration operation count);
* ``rho1``, ``rho2`` -- the one- and two-body density matrices of Eqs. rho1
  and rho2, each element by its definition <C| O C> with O the unit one- or
  two-body operator applied by ``apply_push``;
* ``evolve`` -- exp(-i H dt) C through the eigen-decomposition of the dense H
  (the exact propagator that a short-iterative-Lanczos step approximates);
* ``sector_indices``, ``sector_apply`` -- the configurations of one total
  orbital weight sum_i i n_i (total momentum for plane waves) in the order of
  the full space, and sigma = H C restricted to them (embed, push, restrict);
* ``lanczos_ground`` -- Lanczos with complete re-orthogonalisation and a
  tridiagonal eigen-solve, as in Sec. 6;
* ``bethe_ground_energy`` -- the Lieb-Liniger ground state from the Bethe
  equations (Eqs. LLsystem and LLE0), by Newton's method.

Every function is pinned by tests in ``tests/test_oracle_*.py`` against
brute-force enumeration, a textbook matrix construction of the operators,
closed forms and the paper's worked examples.  ``bethe_ground_energy`` is
pinned by the two-body closed form and the Tonks-Girardeau and weak-coupling
limits.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fock_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``fock_oracle.c`` into ``liboracle.so`` next to it (gcc)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        i64, i32, p = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
        lib.oracle_nc.restype = i64
        lib.oracle_nc.argtypes = [i64, i64]
        lib.oracle_rank.restype = i64
        lib.oracle_rank.argtypes = [i32, i32, p]
        lib.oracle_unrank.restype = None
        lib.oracle_unrank.argtypes = [i32, i32, i64, p]
        lib.oracle_rank_batch.argtypes = [i32, i32, p, i64, p]
        lib.oracle_unrank_batch.argtypes = [i32, i32, p, i64, p]
        lib.oracle_single_jump_map.argtypes = [i32, i32, p]
        lib.oracle_removal_count.restype = ctypes.c_int32
        lib.oracle_removal_count.argtypes = [i32, p]
        lib.oracle_double_jump_map.argtypes = [i32, i32, p, p]
        lib.oracle_apply_push.argtypes = [i32, i32, p, p, p, p]
        lib.oracle_apply_rows.argtypes = [i32, i32, p, p, p, p, i64, p]
        lib.oracle_dense_hamiltonian.argtypes = [i32, i32, p, p, p]
        lib.oracle_column_terms.restype = i64
        lib.oracle_column_terms.argtypes = [i32, i32, p, p, i64]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _cplx(a, shape=None) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.complex128))
    if shape is not None:
        a = a.reshape(shape)
    return a


# --------------------------------------------------------------------------
# Hashing: Eq. nc, Algorithm 1, Algorithm 2
# --------------------------------------------------------------------------
def nc(n: int, m: int) -> int:
    """N_c(n, m) = C(n + m - 1, m - 1) (Eq. nc), N_c(n, 0) = 0 (Eq. TotalCost)."""
    return int(_load().oracle_nc(n, m))


def rank(N: int, M: int, occ) -> int:
    """Index of one occupation vector by Algorithm 1."""
    o = np.ascontiguousarray(np.asarray(occ, dtype=np.int32))
    return int(_load().oracle_rank(N, M, _ptr(o)))


def unrank(N: int, M: int, idx: int) -> np.ndarray:
    """Occupation vector of one index by Algorithm 2."""
    o = np.zeros(M, dtype=np.int32)
    _load().oracle_unrank(N, M, int(idx), _ptr(o))
    return o


def rank_batch(N: int, M: int, occ: np.ndarray) -> np.ndarray:
    o = np.ascontiguousarray(np.asarray(occ, dtype=np.int32).reshape(-1, M))
    out = np.empty(o.shape[0], dtype=np.int64)
    _load().oracle_rank_batch(N, M, _ptr(o), o.shape[0], _ptr(out))
    return out


def unrank_batch(N: int, M: int, idx) -> np.ndarray:
    i = np.ascontiguousarray(np.asarray(idx, dtype=np.int64).reshape(-1))
    out = np.empty((i.shape[0], M), dtype=np.int32)
    _load().oracle_unrank_batch(N, M, _ptr(i), i.shape[0], _ptr(out))
    return out


# --------------------------------------------------------------------------
# Jump maps (Sec. 4)
# --------------------------------------------------------------------------
def single_jump_map(N: int, M: int) -> np.ndarray:
    """J1[gamma, k, l]: index after moving one particle k -> l; -1 if n_k = 0."""
    n = nc(N, M)
    out = np.empty((n, M, M), dtype=np.int32)
    _load().oracle_single_jump_map(N, M, _ptr(out))
    return out


def removal_count(M: int, occ) -> int:
    o = np.ascontiguousarray(np.asarray(occ, dtype=np.int32))
    return int(_load().oracle_removal_count(M, _ptr(o)))


def double_jump_map(N: int, M: int):
    """Variable-length rows of Sec. 4: returns (row_off[Nc+1], data).

    Row gamma holds one stride of M*M entries per allowed removal pair
    (k <= q, lexicographic); entry s*M + l of a stride is the index after
    removing from k and q and adding to s and l.
    """
    n = nc(N, M)
    off = np.empty(n + 1, dtype=np.int64)
    lib = _load()
    lib.oracle_double_jump_map(N, M, _ptr(off), None)
    data = np.empty(int(off[-1]), dtype=np.int32)
    lib.oracle_double_jump_map(N, M, _ptr(off), _ptr(data))
    return off, data


# --------------------------------------------------------------------------
# sigma = H C (Eq. Haction)
# --------------------------------------------------------------------------
def apply_push(N: int, M: int, h, W, C) -> np.ndarray:
    """Full sigma = H C by scattering every column (push form)."""
    n = nc(N, M)
    hh = _cplx(h, (M, M))
    WW = None if W is None else _cplx(W, (M, M, M, M))
    CC = _cplx(C, (n,))
    out = np.empty(n, dtype=np.complex128)
    _load().oracle_apply_push(N, M, _ptr(hh), None if WW is None else _ptr(WW), _ptr(CC), _ptr(out))
    return out


def apply_rows(N: int, M: int, h, W, C, rows) -> np.ndarray:
    """sigma[rows] of sigma = H C, each row as the conjugate of a column of H."""
    n = nc(N, M)
    hh = _cplx(h, (M, M))
    WW = None if W is None else _cplx(W, (M, M, M, M))
    CC = _cplx(C, (n,))
    r = np.ascontiguousarray(np.asarray(rows, dtype=np.int64).reshape(-1))
    out = np.empty(r.shape[0], dtype=np.complex128)
    _load().oracle_apply_rows(N, M, _ptr(hh), None if WW is None else _ptr(WW), _ptr(CC),
                              _ptr(r), r.shape[0], _ptr(out))
    return out


def dense_hamiltonian(N: int, M: int, h, W) -> np.ndarray:
    """Dense H[gamma, beta] for tiny spaces."""
    n = nc(N, M)
    hh = _cplx(h, (M, M))
    WW = None if W is None else _cplx(W, (M, M, M, M))
    out = np.empty((n, n), dtype=np.complex128)
    _load().oracle_dense_hamiltonian(N, M, _ptr(hh), None if WW is None else _ptr(WW), _ptr(out))
    return out


def column_terms(N: int, M: int, h, W, gamma: int) -> int:
    """Operator strings with a nonzero coefficient that do not annihilate
    configuration gamma (Eqs. noninteracting, interacting), counted before
    equal targets are merged."""
    hh = _cplx(h, (M, M))
    WW = None if W is None else _cplx(W, (M, M, M, M))
    return int(_load().oracle_column_terms(N, M, _ptr(hh), None if WW is None else _ptr(WW), int(gamma)))


# --------------------------------------------------------------------------
# Density matrices (Eqs. rho1, rho2)
# --------------------------------------------------------------------------
def rho1(N: int, M: int, C) -> np.ndarray:
    """rho1[k, l] = <C| a^dag_k a_l |C> (Eq. rho1): the expectation of the unit
    one-body operator h = E_kl, applied by the push form."""
    CC = _cplx(C, (nc(N, M),))
    out = np.empty((M, M), dtype=np.complex128)
    for k in range(M):
        for l in range(M):
            h = np.zeros((M, M), dtype=np.complex128)
            h[k, l] = 1.0
            out[k, l] = np.vdot(CC, apply_push(N, M, h, None, CC))
    return out


def rho2(N: int, M: int, C) -> np.ndarray:
    """rho2[k, l, q, s] = <C| a^dag_k a^dag_l a_q a_s |C> (Eq. rho2): the
    expectation of the two-body operator with W[k, l, q, s] = 2 (W multiplies
    1/2 a^dag_k a^dag_l a_q a_s), applied by the push form."""
    CC = _cplx(C, (nc(N, M),))
    zero_h = np.zeros((M, M), dtype=np.complex128)
    out = np.empty((M, M, M, M), dtype=np.complex128)
    for k in range(M):
        for l in range(M):
            for q in range(M):
                for s in range(M):
                    W = np.zeros((M, M, M, M), dtype=np.complex128)
                    W[k, l, q, s] = 2.0
                    out[k, l, q, s] = np.vdot(CC, apply_push(N, M, zero_h, W, CC))
    return out


# --------------------------------------------------------------------------
# Time evolution (the propagator of the SIL integrator named in Sec. 2)
# --------------------------------------------------------------------------
def evolve(N: int, M: int, h, W, C, dt: float) -> np.ndarray:
    """exp(-i H dt) C for a tiny space: H = U diag(E) U^H from the dense
    Hamiltonian (numpy's Hermitian eigen-solver as a step), then
    U diag(exp(-i E dt)) U^H C."""
    H = dense_hamiltonian(N, M, h, W)
    E, U = np.linalg.eigh(H)
    CC = _cplx(C, (nc(N, M),))
    return U @ (np.exp(-1j * E * dt) * (U.conj().T @ CC))


# --------------------------------------------------------------------------
# Sectors of fixed total orbital weight (total momentum for plane waves)
# --------------------------------------------------------------------------
def sector_indices(N: int, M: int, Q: int) -> np.ndarray:
    """Full-space indices, ascending, of the configurations with
    sum_i i n_i = Q.  For the plane-wave orbitals of Sec. 6 (orbital i has
    momentum (i - floor(M/2)) 2 pi / L) this is the sector of total momentum
    (Q - N floor(M/2)) 2 pi / L, which H preserves when h is diagonal and
    W_kqsl = 0 unless k + q = s + l.  The sector's basis is ordered as the
    full space orders it (Algorithm 1), so the rank of a sector configuration
    is its position in this list."""
    occ = unrank_batch(N, M, np.arange(nc(N, M), dtype=np.int64))
    return np.nonzero(occ.astype(np.int64) @ np.arange(M, dtype=np.int64) == Q)[0]


def sector_apply(N: int, M: int, Q: int, h, W, Cs) -> np.ndarray:
    """sigma = H C on a sector: C embedded in the full space (zero outside
    the sector), sigma = H C by the push form, and the sector's rows kept."""
    idx = sector_indices(N, M, Q)
    C = np.zeros(nc(N, M), dtype=np.complex128)
    C[idx] = _cplx(Cs, (idx.shape[0],))
    return apply_push(N, M, h, W, C)[idx]


# --------------------------------------------------------------------------
# Lanczos with complete re-orthogonalisation (Sec. 6)
# --------------------------------------------------------------------------
def lanczos_ground(apply, v0: np.ndarray, max_iter: int, tol: float = 1e-13):
    """Lowest eigenvalue of a Hermitian operator by Lanczos.

    ``apply(v)`` returns H v.  Every new Krylov vector is re-orthogonalised
    against all previous ones (twice, classical Gram-Schmidt), and the
    tridiagonal matrix is diagonalised by LAPACK through scipy.  Stops when the
    Ritz residual estimate |beta_j * y_j| falls below ``tol`` * |theta| or after
    ``max_iter`` steps.  Returns (E0, ground vector, iterations).
    """
    from scipy.linalg import eigh_tridiagonal

    v = np.asarray(v0, dtype=np.complex128).copy()
    v /= np.linalg.norm(v)
    V = [v]
    alpha, beta = [], []
    theta, y = None, None
    for j in range(max_iter):
        w = apply(V[j])
        a = np.vdot(V[j], w).real
        alpha.append(a)
        w = w - a * V[j]
        if j > 0:
            w = w - beta[-1] * V[j - 1]
        for _ in range(2):
            Q = np.array(V)
            w = w - Q.T @ (Q.conj() @ w)
        b = np.linalg.norm(w)
        evals, evecs = eigh_tridiagonal(np.array(alpha), np.array(beta)) if j > 0 else (
            np.array([a]), np.ones((1, 1)))
        theta, y = evals[0], evecs[:, 0]
        if abs(b * y[-1]) <= tol * max(abs(theta), 1.0) or b == 0.0 or j == max_iter - 1:
            break
        beta.append(b)
        V.append(w / b)
    Q = np.array(V[: len(y)])
    vec = Q.T @ y
    return float(theta), vec / np.linalg.norm(vec), len(alpha)


# --------------------------------------------------------------------------
# Bethe ansatz for the Lieb-Liniger ground state (Eqs. LLsystem, LLE0)
# --------------------------------------------------------------------------
def bethe_ground_energy(N: int, g: float, L: float = 1.0, hbar: float = 1.0, m: float = 1.0):
    """Ground-state energy of N bosons on a ring of length L with contact g.

    Solves L k_j = 2 pi I_j - 2 sum_i arctan((k_j - k_i) / c), c = m g / hbar^2,
    with I_j = j - (N + 1)/2 for j = 1..N, by damped Newton iteration, then
    E0 = hbar^2 / (2 m) sum_j k_j^2.  Returns (E0, k).
    """
    c = m * g / hbar ** 2
    I = np.arange(1, N + 1, dtype=np.float64) - (N + 1) / 2.0
    # Strong-coupling estimate as the starting point: k = 2 pi I / (L + 2 N / c).
    k = 2.0 * np.pi * I / (L + 2.0 * N / c)

    def F(k):
        d = k[:, None] - k[None, :]
        return L * k - 2.0 * np.pi * I + 2.0 * np.arctan(d / c).sum(axis=1)

    f = F(k)
    for _ in range(200):
        d = k[:, None] - k[None, :]
        kern = 2.0 * c / (c * c + d * d)
        J = -kern.copy()
        np.fill_diagonal(J, 0.0)
        J[np.diag_indices(N)] = L + kern.sum(axis=1) - kern.diagonal()
        step = np.linalg.solve(J, -f)
        lam = 1.0
        while True:
            kn = k + lam * step
            fn = F(kn)
            if np.linalg.norm(fn) <= (1.0 - 1e-4 * lam) * np.linalg.norm(f) or lam < 1e-6:
                break
            lam *= 0.5
        k, f = kn, fn
        if np.linalg.norm(f) <= 1e-15 * max(1.0, np.abs(2.0 * np.pi * I).max()):
            break
    E0 = hbar ** 2 / (2.0 * m) * float(np.sum(k * k))
    return E0, k
