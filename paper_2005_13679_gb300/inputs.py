"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This module draws random numbers and writes down the one- and two-body
coefficients of the model Hamiltonians.  It holds none of the method's
arithmetic (no hashing, no jump maps, no Hamiltonian action), and it imports
neither the CUDA library nor the oracle, so both sides can be fed the same
inputs.

Conventions (arXiv:2005.13679):

* ``h[k, l]`` multiplies a^dag_k a_l (Eq. noninteracting);
* ``W[k, q, s, l]`` multiplies (1/2) a^dag_k a^dag_q a_s a_l (Eq. interacting,
  index order fixed by this library: creation indices first, then the
  annihilation indices in the order they appear in the operator string);
* complex128 arrays, C-contiguous.

Recipes:

* Lieb-Liniger ring in plane waves (Sec. 6): orbital i carries momentum
  p_i = 2 pi (i - floor(M/2)) / L, so M = 5 gives -2..2 and M = 10 gives -5..4;
  h_kk = p_k^2 / 2 (hbar = m = 1), W_kqsl = g / L when p_k + p_q = p_s + p_l.
* Generic Hermitian model: h = (A + A^dag) / 2 with Re and Im of A drawn
  N(0, 1); W is a draw G with Re and Im N(0, 0.1), averaged over the group
  generated by k<->q, s<->l and W_kqsl -> conj(W_lsqk), so that the operator is
  Hermitian and symmetric under boson exchange.
* Coefficient vectors: Re and Im N(0, 1), normalised to unit 2-norm.
* Uneven batch: N ~ U{10..200}, M ~ U{4..12}, log g ~ U[ln 0.1, ln 10]; when
  N_c(N, M) exceeds the cap, N is lowered to the largest value under it.

All draws use numpy's PCG64 generator with the stated seeds.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def space_size(N: int, M: int) -> int:
    """Number of ways to put N bosons in M orbitals (used only to size inputs)."""
    return math.comb(N + M - 1, M - 1)


def ll_orbital_momenta(M: int, L: float = 1.0) -> np.ndarray:
    """Plane-wave momenta 2 pi (i - floor(M/2)) / L, i = 0..M-1."""
    return 2.0 * np.pi * (np.arange(M) - M // 2) / L


def lieb_liniger_hw(M: int, g: float, L: float = 1.0):
    """One- and two-body coefficients of the Lieb-Liniger ring in plane waves."""
    p = ll_orbital_momenta(M, L)
    h = np.zeros((M, M), dtype=np.complex128)
    h[np.arange(M), np.arange(M)] = 0.5 * p * p
    idx = np.arange(M) - M // 2
    tot_in = idx[:, None] + idx[None, :]
    cons = tot_in[:, :, None, None] == tot_in[None, None, :, :]
    W = np.where(cons, g / L, 0.0).astype(np.complex128)
    return h, W


def bose_hubbard_hw(M: int, J: float = 1.0, U: float = 1.0, mu: float = 0.0, periodic: bool = True):
    """Bose-Hubbard chain of M sites: hopping -J between neighbouring sites
    (a ring when periodic), on-site energy -mu, and on-site repulsion U as the
    two-body coefficient W[k, k, k, k] = U (multiplying 1/2 a^dag_k a^dag_k a_k a_k)."""
    h = np.zeros((M, M), dtype=np.complex128)
    for k in range(M):
        h[k, k] = -mu
        for l in ((k + 1) % M if periodic else k + 1,):
            if l < M and l != k:
                h[k, l] += -J
                h[l, k] += -J
    W = np.zeros((M, M, M, M), dtype=np.complex128)
    W[np.arange(M), np.arange(M), np.arange(M), np.arange(M)] = U
    return h, W


def nearest_neighbour_hw(M: int, seed: int, ring: bool = True, complex_hops: bool = True):
    """Random operator of the Bose-Hubbard class: site energies h[k, k] and
    on-site repulsions W[k, k, k, k] drawn uniformly, hops h[k, k + 1] (and
    h[M - 1, 0] on a ring) of random size and, when complex_hops, random
    phase; h[l, k] = conj(h[k, l])."""
    rng = np.random.Generator(np.random.PCG64(seed))
    h = np.zeros((M, M), dtype=np.complex128)
    h[np.arange(M), np.arange(M)] = rng.uniform(-1.0, 1.0, M)
    nb = M if (ring and M > 2) else M - 1
    for b in range(nb):
        k, l = b, (b + 1) % M
        t = -rng.uniform(0.5, 1.5)
        if complex_hops:
            t *= np.exp(1j * rng.uniform(-np.pi, np.pi))
        h[k, l] += t
        h[l, k] += np.conj(t)
    W = np.zeros((M, M, M, M), dtype=np.complex128)
    W[np.arange(M), np.arange(M), np.arange(M), np.arange(M)] = rng.uniform(0.0, 8.0, M)
    return h, W


def weight_conserving_hw(M: int, seed: int):
    """Random operator that preserves the total orbital weight sum_i i n_i:
    real diagonal h, and the random symmetrised W of ``random_hermitian_hw``
    kept only where k + q = s + l (the Lieb-Liniger selection rule, with
    complex coefficients)."""
    h0, W0 = random_hermitian_hw(M, seed)
    h = np.diag(np.real(np.diag(h0))).astype(np.complex128)
    i = np.arange(M)
    tot = i[:, None] + i[None, :]
    W = np.where(tot[:, :, None, None] == tot[None, None, :, :], W0, 0.0)
    return np.ascontiguousarray(h), np.ascontiguousarray(W)


def random_hermitian_hw(M: int, seed: int, sigma_h: float = 1.0, sigma_w: float = 0.1):
    """Random Hermitian h and boson-symmetric Hermitian W (see module notes)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    A = rng.standard_normal((M, M)) + 1j * rng.standard_normal((M, M))
    A *= sigma_h
    h = 0.5 * (A + A.conj().T)
    G = rng.standard_normal((M, M, M, M)) + 1j * rng.standard_normal((M, M, M, M))
    G *= sigma_w
    S = 0.5 * (G + G.transpose(1, 0, 2, 3))
    S = 0.5 * (S + S.transpose(0, 1, 3, 2))
    W = 0.5 * (S + S.transpose(3, 2, 1, 0).conj())
    return np.ascontiguousarray(h), np.ascontiguousarray(W)


def random_state(nc: int, seed: int) -> np.ndarray:
    """Normalised complex128 vector of length nc."""
    rng = np.random.Generator(np.random.PCG64(seed))
    v = np.empty(nc, dtype=np.complex128)
    f = v.view(np.float64)
    f[:] = rng.standard_normal(2 * nc)
    v /= np.linalg.norm(v)
    return v


def random_block(nc: int, seeds) -> np.ndarray:
    """[nc, nrhs] block, column j from ``random_state(nc, seeds[j])``."""
    seeds = list(seeds)
    out = np.empty((nc, len(seeds)), dtype=np.complex128)
    for j, s in enumerate(seeds):
        out[:, j] = random_state(nc, s)
    return out


@dataclass
class Instance:
    N: int
    M: int
    g: float
    L: float = 1.0


def uneven_ll_batch(count: int = 64, seed: int = 5, cap: int = 10 ** 7,
                    n_range=(10, 200), m_range=(4, 12), g_range=(0.1, 10.0)):
    """Lieb-Liniger instances of uneven size (see module notes)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(count):
        N = int(rng.integers(n_range[0], n_range[1] + 1))
        M = int(rng.integers(m_range[0], m_range[1] + 1))
        g = float(math.exp(rng.uniform(math.log(g_range[0]), math.log(g_range[1]))))
        while N > 1 and space_size(N, M) > cap:
            N -= 1
        out.append(Instance(N=N, M=M, g=g))
    return out


@dataclass
class Workload:
    """A named synthetic workload (sizes of the experiments of the paper's Secs. 4-6)."""
    name: str
    N: int
    M: int
    kind: str                 # "ll", "generic" or "bh"
    seed: int
    g: float = 1.0
    L: float = 1.0
    nrhs: int = 1
    rhs_seeds: list = field(default_factory=list)
    lanczos_seed: int = 0
    sector_Q: int | None = None   # total orbital weight sum_i i n_i of a sector workload

    @property
    def nc(self) -> int:
        return space_size(self.N, self.M)

    def hamiltonian(self):
        if self.kind == "ll":
            return lieb_liniger_hw(self.M, self.g, self.L)
        if self.kind == "bh":
            return bose_hubbard_hw(self.M, 1.0, self.g)
        return random_hermitian_hw(self.M, self.seed)

    def state(self) -> np.ndarray:
        if self.nrhs > 1:
            return random_block(self.nc, self.rhs_seeds)
        return random_state(self.nc, self.seed)


WORKLOADS = {
    # Lieb-Liniger ring, 5 bosons in 5 plane waves (momenta -2..2), g = 1.
    "ll_n5_m5": Workload("ll_n5_m5", N=5, M=5, kind="ll", g=1.0, seed=1, lanczos_seed=101),
    # Generic Hermitian h/W, 100 bosons in 6 orbitals: 96,560,646 configurations.
    "generic_n100_m6": Workload("generic_n100_m6", N=100, M=6, kind="generic", seed=2),
    # Lieb-Liniger ring, 30 bosons in 10 plane waves, g = 0.5: 211,915,132 configurations.
    "ll_n30_m10": Workload("ll_n30_m10", N=30, M=10, kind="ll", g=0.5, seed=3, lanczos_seed=103),
    # Profiling size of the generic N, M = 6 workload: 17,259,390 configurations
    # (complex128 C of 276 MB, larger than L2), same kernel as N = 100.
    "generic_n70_m6": Workload("generic_n70_m6", N=70, M=6, kind="generic", seed=2),
    # Profiling size for the two-phase kernels of the generic M = 6 workload:
    # 8,259,888 configurations (complex128 C of 132 MB, larger than L2) and an
    # (N-2)-space intermediate of 21 x 7,028,847 FP32-pair rows (2.4 GB).
    "generic_n60_m6": Workload("generic_n60_m6", N=60, M=6, kind="generic", seed=2),
    # Profiling size of the Lieb-Liniger M = 10 workload: 20,160,075
    # configurations (complex128 C of 323 MB, larger than L2).
    "ll_n22_m10": Workload("ll_n22_m10", N=22, M=10, kind="ll", g=0.5, seed=3),
    # Profiling size of the Lieb-Liniger M = 10 two-phase kernels: 10,015,005
    # configurations (complex128 C of 160 MB, larger than L2) and an
    # (N-2)-space intermediate of 55 x 4,686,825 FP32-pair rows (4.1 GB).
    "ll_n20_m10": Workload("ll_n20_m10", N=20, M=10, kind="ll", g=0.5, seed=3),
    # Lieb-Liniger ring N = 30, M = 10, g = 0.5 restricted to total momentum 0
    # (orbital weights sum_i i n_i = 150): 2,462,733 of the 211,915,132 configurations.
    "ll_n30_m10_p0": Workload("ll_n30_m10_p0", N=30, M=10, kind="ll", g=0.5, seed=3, lanczos_seed=103,
                              sector_Q=150),
    # Bose-Hubbard ring, 20 bosons on 12 sites, J = 1, U = 4: 84,672,315 configurations.
    "bh_n20_m12": Workload("bh_n20_m12", N=20, M=12, kind="bh", g=4.0, seed=6),
    # Profiling size of the Bose-Hubbard ring: 16 bosons on 12 sites,
    # 13,037,895 configurations (complex128 C of 209 MB, larger than L2).
    "bh_n16_m12": Workload("bh_n16_m12", N=16, M=12, kind="bh", g=4.0, seed=6),
    # Generic Hermitian h/W, 20 bosons in 8 orbitals, a block of 16 vectors.
    "generic_n20_m8_rhs16": Workload("generic_n20_m8_rhs16", N=20, M=8, kind="generic", seed=4,
                                     nrhs=16, rhs_seeds=list(range(4000, 4016))),
}
