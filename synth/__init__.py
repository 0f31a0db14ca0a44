"""Seeded synthetic inputs shared by the oracle, the tests and the bench.

This package draws random numbers and enumerates index sets; it holds none of
the method's arithmetic (no Jordan-Wigner mapping, no gate, no energy). Every
workload stands in for the paper's molecules (STO-3G integrals of F2 / CH3F are
not available), using the active-space sizes of the paper's experiments.
"""
from .integrals import (Problem, draw_one_body, draw_factors, eri_from_factors,
                        random_problem, ScanProblem, draw_scan)
from .pools import uccsd_pool, hf_bitstring, spin_counts, upccgsd_pool, puccd_pool, hcb_pair_pool, hcb_pairs_of
from .pauli import random_pauli_terms
from .configs import (config0, config1, config2, config3, config4,
                      config2_instance, puccd_scan, puccd_large, Workload)

__all__ = [
    "Problem", "draw_one_body", "draw_factors", "eri_from_factors", "random_problem",
    "ScanProblem", "draw_scan", "uccsd_pool", "hf_bitstring", "spin_counts",
    "upccgsd_pool", "puccd_pool", "hcb_pair_pool", "hcb_pairs_of",
    "random_pauli_terms", "config0", "config1", "config2", "config3", "config4",
    "puccd_scan", "puccd_large",
    "config2_instance", "Workload",
]
