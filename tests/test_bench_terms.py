"""The configuration-terms count the bench reports, pinned on the CPU.

bench.terms_formula uses the closed form
    N_c + N_c(N-1, M) #{k != l : h_kl != 0} + N_c(N-2, M) #{reduced W entries != 0},
which rests on two counting facts: a configuration with n_k >= 1 is one of
N_c(N-1, M) (remove a particle from k), and one where the removal multiset
{k, q} is possible is one of N_c(N-2, M).  Here the per-configuration
definition (one diagonal term, one term per occupied k and l != k with
h_kl != 0, one term per possible removal multiset and addition multiset with a
nonzero reduced coefficient) is summed over every enumerated configuration.
"""
import numpy as np
import pytest

import oracle
from paper_2005_13679_gb300 import inputs

import bench


class _W:
    def __init__(self, N, M):
        self.N, self.M = N, M


def brute_terms(N, M, h, W):
    pairs = [(k, q) for k in range(M) for q in range(k, M)]
    R = {}
    if W is not None:
        for k in range(M):
            for q in range(M):
                for s in range(M):
                    for l in range(M):
                        key = ((min(k, q), max(k, q)), (min(s, l), max(s, l)))
                        R[key] = R.get(key, 0) + W[k, q, s, l]
    adds = {r: sum(1 for a in pairs if R.get((r, a), 0) != 0) for r in pairs}
    total = 0
    for n in oracle.unrank_batch(N, M, np.arange(oracle.nc(N, M))):
        t = 1
        for k in range(M):
            if n[k] >= 1:
                t += sum(1 for l in range(M) if l != k and h[k, l] != 0)
        if W is not None and N >= 2:
            for (k, q) in pairs:
                ok = n[k] >= 2 if k == q else (n[k] >= 1 and n[q] >= 1)
                if ok:
                    t += adds[(k, q)]
        total += t
    return total


@pytest.mark.parametrize("N,M,kind", [(6, 4, "generic"), (5, 5, "ll"), (7, 3, "bh"), (1, 5, "generic"),
                                      (4, 6, "onebody"), (8, 1, "generic"), (3, 7, "nn")])
def test_terms_formula_against_enumeration(N, M, kind):
    if kind == "generic":
        h, W = inputs.random_hermitian_hw(M, 3)
    elif kind == "ll":
        h, W = inputs.lieb_liniger_hw(M, 0.5)
    elif kind == "bh":
        h, W = inputs.bose_hubbard_hw(M, 1.0, 2.0, 0.1)
    elif kind == "nn":
        h, W = inputs.nearest_neighbour_hw(M, 2, True, True)
    else:
        h, _ = inputs.random_hermitian_hw(M, 3)
        W = None
    assert bench.terms_formula(_W(N, M), h, W) == brute_terms(N, M, h, W)


def test_nearest_neighbour_terms():
    """One diagonal term and two hops per bond: M bonds on a ring of M > 2
    sites, one for M = 2."""
    for N, M in [(5, 2), (4, 3), (6, 8)]:
        w = _W(N, M)
        w.nc = oracle.nc(N, M)
        nb = M if M > 2 else 1
        assert bench.nn_terms(w) == w.nc * (1 + 2 * nb)
