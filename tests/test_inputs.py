"""The seeded input generators: deterministic, Hermitian operators with the
boson symmetries of W, the stated sizes of the named workloads, and
normalised states."""
import math

import numpy as np
import pytest

from paper_2005_13679_gb300 import inputs

GENERATORS = {
    "generic": lambda M: inputs.random_hermitian_hw(M, 5),
    "ll": lambda M: inputs.lieb_liniger_hw(M, 0.8),
    "bh": lambda M: inputs.bose_hubbard_hw(M, 1.0, 2.5, 0.4),
    "nn": lambda M: inputs.nearest_neighbour_hw(M, 5, True, True),
    "wc": lambda M: inputs.weight_conserving_hw(M, 5),
}


@pytest.mark.parametrize("kind", list(GENERATORS))
@pytest.mark.parametrize("M", [1, 2, 3, 6])
def test_operators_are_hermitian_and_boson_symmetric(kind, M):
    h, W = GENERATORS[kind](M)
    h2, W2 = GENERATORS[kind](M)
    assert np.array_equal(h, h2) and np.array_equal(W, W2)          # seeded
    np.testing.assert_allclose(h, h.conj().T, atol=1e-15)
    # the operator sum is unchanged by k <-> q and s <-> l, and Hermitian:
    # W_kqsl = conj(W_lsqk)
    np.testing.assert_allclose(W, W.transpose(1, 0, 3, 2), atol=1e-15)
    np.testing.assert_allclose(W, W.transpose(3, 2, 1, 0).conj(), atol=1e-15)


def test_lieb_liniger_selection_rule_and_kinetic_energy():
    M, g = 5, 0.8
    h, W = inputs.lieb_liniger_hw(M, g)
    p = np.arange(M) - M // 2
    np.testing.assert_allclose(np.diag(h).real, 0.5 * (2 * np.pi * p) ** 2)
    for k, q, s, l in np.ndindex(M, M, M, M):
        expect = g if p[k] + p[q] == p[s] + p[l] else 0.0
        assert W[k, q, s, l] == expect


def test_nearest_neighbour_structure():
    for ring in (True, False):
        h, W = inputs.nearest_neighbour_hw(6, 3, ring, True)
        for k, l in zip(*np.nonzero(h)):
            d = abs(int(k) - int(l))
            assert d <= 1 or (ring and d == 5)
        assert np.count_nonzero(W) == np.count_nonzero(np.einsum("kkkk->k", W))


def test_named_workload_sizes():
    sizes = {"ll_n5_m5": 126, "generic_n100_m6": 96560646, "ll_n30_m10": 211915132,
             "generic_n60_m6": 8259888, "bh_n20_m12": 84672315, "bh_n16_m12": 13037895,
             "generic_n20_m8_rhs16": 888030, "ll_n20_m10": 10015005}
    for name, n in sizes.items():
        w = inputs.WORKLOADS[name]
        assert w.nc == n == math.comb(w.N + w.M - 1, w.M - 1), name
    assert inputs.WORKLOADS["ll_n30_m10_p0"].sector_Q == 30 * (10 // 2)


def test_states_are_normalised_and_seeded():
    a = inputs.random_state(1000, 7)
    assert abs(np.linalg.norm(a) - 1.0) < 1e-12
    assert np.array_equal(a, inputs.random_state(1000, 7))
    assert not np.array_equal(a, inputs.random_state(1000, 8))


def test_uneven_batch_respects_the_cap():
    inst = inputs.uneven_ll_batch()
    assert len(inst) == 64
    for x in inst:
        assert 4 <= x.M <= 12 and 1 <= x.N <= 200 and 0.1 <= x.g <= 10.0
        assert math.comb(x.N + x.M - 1, x.M - 1) <= 10 ** 7
