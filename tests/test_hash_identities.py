"""The counting identities behind the GPU kernels, checked on the CPU against
the oracle (Algorithm 1 and the sector enumeration), independently of the CUDA
code.  The identities are restated here from their derivations.

* Sector hash: with D_m(s, q) the number of configurations of s particles in
  orbitals 0..m-1 of weight q, the position of n among the configurations of
  weight Q (in the full space's order) is
      N_sec - 1 - sum_{m=1}^{M-2} D_{m+2}(S_m - 1, Q_m - m - 1),
  S_m, Q_m the prefix sums of n_i and i n_i; decoding takes, from the top
  orbital down, the largest c with D_{m+1}(S, Q) - D_{m+1}(S - c, Q - m c)
  not above the remaining index.
* Nearest-neighbour hops: moving a particle across the chain bond (m, m + 1)
  changes only S_m, so the target's rank is gamma minus one difference of
  C(S_m + m, m + 1); across the ring bond (M - 1, 0) the differences of all
  m < M - 1 add up.
* Sector targets: for a term removing (k, q) and adding (s, l) with
  k + q = s + l the prefix sums change by a constant between consecutive
  positions of the sorted {k, q, s, l}.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_2005_13679_gb300 import inputs


def D_table(N, M, Q):
    D = np.zeros((M + 2, N + 1, Q + 1), dtype=object)
    for s in range(N + 1):
        D[1, s, 0] = 1
    for m in range(1, M + 1):
        for s in range(N + 1):
            for q in range(Q + 1):
                v = D[m, s, q]
                if s >= 1 and q >= m:
                    v += D[m + 1, s - 1, q - m]
                D[m + 1, s, q] = v
    return D


def Dv(D, m, s, q):
    return 0 if s < 0 or q < 0 or s >= D.shape[1] or q >= D.shape[2] else D[m, s, q]


def sector_rank(n, D, M, ns):
    S, W, acc = n[0], 0, ns - 1
    for m in range(1, M - 1):
        S += n[m]
        W += m * n[m]
        acc -= Dv(D, m + 2, S - 1, W - m - 1)
    return acc


def sector_unrank(r, D, N, M, Q):
    s, q, rem, n = N, Q, r, [0] * M
    for m in range(M - 1, 0, -1):
        top = Dv(D, m + 1, s, q)
        lo, hi = 0, min(s, q // m)
        while lo < hi:
            mid = (lo + hi + 1) // 2
            if top - Dv(D, m + 1, s - mid, q - m * mid) <= rem:
                lo = mid
            else:
                hi = mid - 1
        rem -= top - Dv(D, m + 1, s - lo, q - m * lo)
        n[m], s, q = lo, s - lo, q - m * lo
    n[0] = s
    return n


@pytest.mark.parametrize("N,M,Q", [(5, 5, 10), (6, 4, 0), (6, 4, 18), (7, 6, 14), (4, 7, 9), (9, 1, 0), (6, 2, 3)])
def test_sector_hash_identity(N, M, Q):
    idx = oracle.sector_indices(N, M, Q)
    occ = oracle.unrank_batch(N, M, idx)
    D = D_table(N, M, Q)
    ns = Dv(D, M, N, Q)
    assert ns == len(idx)
    for r, n in enumerate(occ):
        assert sector_rank(list(n), D, M, ns) == r
        assert sector_unrank(r, D, N, M, Q) == list(n)


@pytest.mark.parametrize("N,M", [(5, 4), (4, 6), (6, 3), (3, 2), (2, 7)])
def test_nearest_neighbour_hop_targets(N, M):
    mod = lambda m, x: math.comb(x, m + 1) if x >= 0 else 0
    for g in range(oracle.nc(N, M)):
        n = list(oracle.unrank(N, M, g))
        S = np.cumsum(n)
        fm = fp = 0
        for m in range(M - 1):
            x = S[m] + m
            dm, dp = mod(m, x - 1) - mod(m, x), mod(m, x + 1) - mod(m, x)
            fm, fp = fm + dm, fp + dp
            if n[m] > 0:                                     # particle m -> m + 1
                t = list(n); t[m] -= 1; t[m + 1] += 1
                assert oracle.rank(N, M, t) == g - dm
            if n[m + 1] > 0:                                 # particle m + 1 -> m
                t = list(n); t[m + 1] -= 1; t[m] += 1
                assert oracle.rank(N, M, t) == g - dp
        if M > 2:
            if n[M - 1] > 0:                                 # ring bond, M - 1 -> 0
                t = list(n); t[M - 1] -= 1; t[0] += 1
                assert oracle.rank(N, M, t) == g - fp
            if n[0] > 0:                                     # 0 -> M - 1
                t = list(n); t[0] -= 1; t[M - 1] += 1
                assert oracle.rank(N, M, t) == g - fm


def test_sector_target_segments():
    """For every weight-conserving (k, q) -> (s, l), the per-orbital change of
    the prefix sums is constant on the segments between the sorted positions
    and zero outside them."""
    for M in range(2, 9):
        for k, q, s, l in itertools.product(range(M), repeat=4):
            if not (k <= q and s <= l and k + q == s + l):
                continue
            dn = [0] * M
            for p, d in ((k, -1), (q, -1), (s, 1), (l, 1)):
                dn[p] += d
            dS = np.cumsum(dn)
            dQ = np.cumsum([m * dn[m] for m in range(M)])
            pos = sorted([(k, -1), (q, -1), (s, 1), (l, 1)])
            cs = cq = 0
            expect = [(0, 0)] * M
            for i in range(3):
                cs += pos[i][1]
                cq += pos[i][0] * pos[i][1]
                for m in range(pos[i][0], pos[i + 1][0]):
                    expect[m] = (cs, cq)
            assert [(int(dS[m]), int(dQ[m])) for m in range(M)] == expect


def test_weight_conserving_inputs_conserve():
    """The weight-conserving test operators keep only k + q = s + l."""
    for M in (3, 5, 7):
        h, W = inputs.weight_conserving_hw(M, 2)
        assert np.count_nonzero(h - np.diag(np.diag(h))) == 0
        for k, q, s, l in zip(*np.nonzero(W)):
            assert k + q == s + l
