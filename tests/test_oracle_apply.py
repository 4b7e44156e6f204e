"""Pins for the oracle's Hamiltonian action sigma = H C (Eq. Haction).

Independent references used here:

* a textbook construction of the boson ladder operators as Kronecker products
  of truncated single-mode matrices (a|n> = sqrt(n)|n-1>), restricted to the
  N-particle states in brute-force enumeration order;
* Hermiticity of H for Hermitian, boson-symmetric h and W;
* closed forms: the g = 0 Lieb-Liniger spectrum and the Lieb-Liniger diagonal;
* conservation of total momentum for the Lieb-Liniger ring;
* the matrix-element rules of Appendix B for the one- and two-body density
  matrices, evaluated directly on the brute-force basis.
"""
import itertools

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from paper_2005_13679_gb300 import inputs
from tests.test_oracle_hashing import brute_force_configs


def textbook_hamiltonian(N, M, h, W):
    d = N + 1
    a1 = sp.diags(np.sqrt(np.arange(1, d, dtype=np.float64)), 1, shape=(d, d), format="csr")
    eye = sp.identity(d, format="csr")
    A = []
    for k in range(M):
        op = None
        for j in range(M):
            f = a1 if j == k else eye
            op = f if op is None else sp.kron(op, f, format="csr")
        A.append(op.astype(np.complex128))
    Ad = [x.conj().T.tocsr() for x in A]
    dim = d ** M
    H = sp.csr_matrix((dim, dim), dtype=np.complex128)
    for k in range(M):
        for l in range(M):
            if h[k, l] != 0:
                H = H + h[k, l] * (Ad[k] @ A[l])
    if W is not None:
        for k, q, s, l in itertools.product(range(M), repeat=4):
            if W[k, q, s, l] != 0:
                H = H + 0.5 * W[k, q, s, l] * (Ad[k] @ Ad[q] @ A[s] @ A[l])
    confs = brute_force_configs(N, M)
    flat = [sum(c[j] * d ** (M - 1 - j) for j in range(M)) for c in confs]
    return H[flat][:, flat].toarray()


CASES = [
    (1, 4, "generic"), (2, 3, "generic"), (3, 3, "generic"), (2, 4, "generic"),
    (3, 4, "ll"), (4, 3, "ll"), (3, 5, "ll"), (4, 2, "generic"), (5, 1, "generic"),
]


def make_hw(M, kind, seed=11, g=1.3):
    if kind == "ll":
        return inputs.lieb_liniger_hw(M, g)
    return inputs.random_hermitian_hw(M, seed)


@pytest.mark.parametrize("N,M,kind", CASES)
def test_dense_matches_textbook_operators(N, M, kind):
    h, W = make_hw(M, kind)
    ref = textbook_hamiltonian(N, M, h, W)
    got = oracle.dense_hamiltonian(N, M, h, W)
    assert np.allclose(got, ref, rtol=0, atol=1e-12 * max(1.0, np.abs(ref).max()))


@pytest.mark.parametrize("N,M,kind", CASES)
def test_push_and_rows_agree_with_dense(N, M, kind):
    h, W = make_hw(M, kind)
    n = oracle.nc(N, M)
    C = inputs.random_state(n, 3)
    H = oracle.dense_hamiltonian(N, M, h, W)
    sig = oracle.apply_push(N, M, h, W, C)
    assert np.allclose(sig, H @ C, rtol=0, atol=1e-12)
    rows = oracle.apply_rows(N, M, h, W, C, np.arange(n))
    assert np.allclose(rows, sig, rtol=0, atol=1e-12)


@pytest.mark.parametrize("N,M", [(3, 3), (4, 4), (2, 6), (6, 3)])
def test_hermitian(N, M):
    h, W = inputs.random_hermitian_hw(M, 5)
    H = oracle.dense_hamiltonian(N, M, h, W)
    assert np.allclose(H, H.conj().T, rtol=0, atol=1e-13)
    # <x, H y> = <H x, y> with the push form on random vectors
    n = oracle.nc(N, M)
    x, y = inputs.random_state(n, 1), inputs.random_state(n, 2)
    lhs = np.vdot(x, oracle.apply_push(N, M, h, W, y))
    rhs = np.vdot(oracle.apply_push(N, M, h, W, x), y)
    assert abs(lhs - rhs) < 1e-13


@pytest.mark.parametrize("N,M", [(5, 5), (4, 6), (7, 3)])
def test_ll_noninteracting_closed_form(N, M):
    # g = 0: H is diagonal with entries sum_k p_k^2/2 n_k; ground energy 0.
    h, W = inputs.lieb_liniger_hw(M, 0.0)
    H = oracle.dense_hamiltonian(N, M, h, W)
    confs = np.array(brute_force_configs(N, M))
    eps = 0.5 * inputs.ll_orbital_momenta(M) ** 2
    assert np.allclose(H, np.diag(confs @ eps), rtol=0, atol=1e-12)
    assert abs(np.linalg.eigvalsh(H)[0]) < 1e-12


@pytest.mark.parametrize("N,M,g", [(5, 5, 1.0), (4, 6, 0.37), (6, 3, 5.0)])
def test_ll_diagonal_and_momentum(N, M, g):
    h, W = inputs.lieb_liniger_hw(M, g)
    H = oracle.dense_hamiltonian(N, M, h, W)
    confs = np.array(brute_force_configs(N, M))
    eps = 0.5 * inputs.ll_orbital_momenta(M) ** 2
    diag = confs @ eps + (g / 2.0) * (2 * N * (N - 1) - (confs * (confs - 1)).sum(axis=1))
    assert np.allclose(np.diag(H).real, diag, rtol=0, atol=1e-11)
    # a condensate in the zero-momentum orbital has energy g N (N - 1) / 2L
    z = np.zeros(M, dtype=np.int32); z[M // 2] = N
    gz = oracle.rank(N, M, z)
    assert abs(H[gz, gz] - g * N * (N - 1) / 2.0) < 1e-11
    # total momentum is conserved: H couples only equal-momentum configurations
    P = confs @ (np.arange(M) - M // 2)
    assert np.all(H[P[:, None] != P[None, :]] == 0)


# ---------------------------------------------------------------------------
# Appendix B: matrix elements of the reduced density matrices.  beta_a^b moves
# one particle a -> b; beta_ab^cd removes from a and b and adds to c and d.
# Each rule is evaluated on the brute-force basis and compared with the oracle
# expectation value <C| O |C>, O being the operator string of the rule.
# ---------------------------------------------------------------------------
def _expect(N, M, C, op_h=None, op_W=None):
    h = np.zeros((M, M), dtype=np.complex128) if op_h is None else op_h
    sig = oracle.apply_push(N, M, h, op_W, C)
    return np.vdot(C, sig)


def _unit_h(M, k, l):
    h = np.zeros((M, M), dtype=np.complex128); h[k, l] = 1.0
    return h


def _unit_W(M, k, q, s, l):
    W = np.zeros((M, M, M, M), dtype=np.complex128); W[k, q, s, l] = 2.0   # cancels the 1/2
    return W


def _rule(N, M, C, moves, factor):
    """sum_beta C*_beta C_{beta'} factor(n), beta' = beta edited by ``moves``."""
    confs = brute_force_configs(N, M)
    d = {c: i for i, c in enumerate(confs)}
    tot = 0j
    for b, c in enumerate(confs):
        t = list(c)
        ok = True
        for kind, orb in moves:
            t[orb] += -1 if kind == "rm" else 1
            ok &= t[orb] >= 0
        if not ok:
            continue
        tot += np.conj(C[b]) * C[d[tuple(t)]] * factor(np.array(c, dtype=np.float64))
    return tot


@pytest.mark.parametrize("N,M", [(4, 4), (5, 5)])
def test_appendix_b_rules(N, M):
    n = oracle.nc(N, M)
    C = inputs.random_state(n, 17)
    k, s, q, l = 0, 1, 2, 3
    sq = np.sqrt
    checks = [
        # rho_kk
        (_expect(N, M, C, op_h=_unit_h(M, k, k)), _rule(N, M, C, [], lambda m: m[k])),
        # rho_kl = <a^dag_k a_l>
        (_expect(N, M, C, op_h=_unit_h(M, k, l)),
         _rule(N, M, C, [("rm", k), ("ad", l)], lambda m: sq((m[l] + 1) * m[k]))),
        # rho_ksks
        (_expect(N, M, C, op_W=_unit_W(M, k, s, k, s)), _rule(N, M, C, [], lambda m: m[k] * m[s])),
        # rho_kkkk
        (_expect(N, M, C, op_W=_unit_W(M, k, k, k, k)), _rule(N, M, C, [], lambda m: m[k] ** 2 - m[k])),
        # rho_kkql
        (_expect(N, M, C, op_W=_unit_W(M, k, k, q, l)),
         _rule(N, M, C, [("rm", k), ("rm", k), ("ad", q), ("ad", l)],
               lambda m: sq((m[k] - 1) * m[k] * (m[q] + 1) * (m[l] + 1)))),
        # rho_kkkl
        (_expect(N, M, C, op_W=_unit_W(M, k, k, k, l)),
         _rule(N, M, C, [("rm", k), ("ad", l)], lambda m: (m[k] - 1) * sq(m[k] * (m[l] + 1)))),
        # rho_ksqq
        (_expect(N, M, C, op_W=_unit_W(M, k, s, q, q)),
         _rule(N, M, C, [("rm", k), ("rm", s), ("ad", q), ("ad", q)],
               lambda m: sq(m[k] * m[s] * (m[q] + 1) * (m[q] + 2)))),
        # rho_ksss
        (_expect(N, M, C, op_W=_unit_W(M, k, s, s, s)),
         _rule(N, M, C, [("rm", k), ("ad", s)], lambda m: m[s] * sq(m[k] * (m[s] + 1)))),
        # rho_kssl
        (_expect(N, M, C, op_W=_unit_W(M, k, s, s, l)),
         _rule(N, M, C, [("rm", k), ("ad", l)], lambda m: m[s] * sq(m[k] * (m[l] + 1)))),
        # rho_ksql
        (_expect(N, M, C, op_W=_unit_W(M, k, s, q, l)),
         _rule(N, M, C, [("rm", k), ("rm", s), ("ad", q), ("ad", l)],
               lambda m: sq(m[k] * m[s] * (m[q] + 1) * (m[l] + 1)))),
        # rho_kkqq: the printed rule omits the amplitude; the operator string
        # a^dag_k a^dag_k a_q a_q gives sqrt(n_k (n_k - 1) (n_q + 1) (n_q + 2)).
        (_expect(N, M, C, op_W=_unit_W(M, k, k, q, q)),
         _rule(N, M, C, [("rm", k), ("rm", k), ("ad", q), ("ad", q)],
               lambda m: sq(m[k] * (m[k] - 1) * (m[q] + 1) * (m[q] + 2)))),
    ]
    for got, ref in checks:
        assert abs(got - ref) < 1e-12, (got, ref)
