"""Seeded one- and two-body integrals standing in for a molecule's active space.

The paper's Hamiltonian (Eq. 2) is defined by a constant, one-body integrals
h_ij and two-body integrals h_ijkl of a molecule. The molecules themselves are
not available, so integrals are drawn at random with the structure a real
active space has: h real symmetric with an ascending diagonal, and two-body
integrals (pq|rs) = sum_k L^k_pq L^k_rs built from K real symmetric factors,
which gives the 8-fold permutational symmetry and positive semidefiniteness of
real electron-repulsion integrals.

Draw order (fixed, so every seed reproduces): h off-diagonal upper triangle in
row-major order, then for k = 0..K-1 the upper triangle (diagonal included) of
L^k in row-major order. "N(0, s)" means standard deviation s.
"""
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Problem:
    """A spin-free active-space problem.

    n_spatial: spatial orbitals; the qubit count is 2 * n_spatial.
    n_elec: electrons; the reference state fills the lowest n_elec spin orbitals.
    h: (n_s, n_s) one-body integrals; eri: (n_s,)*4 two-body integrals in
    chemists' order (pq|rs); c0: constant energy shift.
    """
    n_spatial: int
    n_elec: int
    h: np.ndarray
    eri: np.ndarray
    c0: float = 0.0
    label: str = ""

    @property
    def n_qubits(self) -> int:
        return 2 * self.n_spatial


def draw_one_body(rng, n_s, sigma=0.5, diag_lo=-1.0, diag_hi=-0.3):
    """Real symmetric h: off-diagonal N(0, sigma), diagonal linspace(diag_lo, diag_hi)."""
    h = np.zeros((n_s, n_s))
    iu = np.triu_indices(n_s, 1)
    h[iu] = rng.normal(0.0, sigma, size=len(iu[0]))
    h = h + h.T
    h[np.diag_indices(n_s)] = np.linspace(diag_lo, diag_hi, n_s)
    return h


def draw_factors(rng, n_s, K, sigma=0.3):
    """K real symmetric factors L^k with upper-triangle entries N(0, sigma)."""
    L = np.zeros((K, n_s, n_s))
    iu = np.triu_indices(n_s, 0)
    for k in range(K):
        m = np.zeros((n_s, n_s))
        m[iu] = rng.normal(0.0, sigma, size=len(iu[0]))
        L[k] = m + np.triu(m, 1).T
    return L


def eri_from_factors(L):
    """(pq|rs) = sum_k L^k_pq L^k_rs (the input definition of the workloads)."""
    return np.einsum("kpq,krs->pqrs", L, L)


def random_problem(rng, n_s, n_elec, K, label=""):
    h = draw_one_body(rng, n_s)
    L = draw_factors(rng, n_s, K)
    return Problem(n_s, n_elec, h, eri_from_factors(L), 0.0, label)


@dataclass
class ScanProblem:
    """A bond-stretch-like scan: h(r) = h0 + exp(-r) h1, L^k(r) = L0^k + exp(-r) L1^k."""
    n_spatial: int
    n_elec: int
    h0: np.ndarray
    h1: np.ndarray
    L0: np.ndarray
    L1: np.ndarray
    rs: np.ndarray = field(default_factory=lambda: np.zeros(0))

    def at(self, r) -> Problem:
        w = np.exp(-r)
        h = self.h0 + w * self.h1
        L = self.L0 + w * self.L1
        return Problem(self.n_spatial, self.n_elec, h, eri_from_factors(L), 0.0, f"r={r:.6f}")

    def problems(self):
        return [self.at(r) for r in self.rs]


def draw_scan(rng, n_s, n_elec, K, rs):
    """Draw h0, L0 then h1, L1 (each as in draw_one_body / draw_factors)."""
    h0 = draw_one_body(rng, n_s)
    L0 = draw_factors(rng, n_s, K)
    h1 = draw_one_body(rng, n_s)
    L1 = draw_factors(rng, n_s, K)
    return ScanProblem(n_s, n_elec, h0, h1, L0, L1, np.asarray(rs, dtype=float))
