"""Plain FP64 CPU oracle for the VQE energy and gradient (test infrastructure).

This package is test infrastructure, not part of the product. Only the tests,
the smoke check and the bench's CPU-baseline leg may import it. It shares no
code with the CUDA library: it builds the Hamiltonian of Eq. 2 from integrals
by literal creation/annihilation operators, has its own Jordan-Wigner mapping,
applies excitation rotations U = exp(theta (T - T^dagger)) (Sec. 2.1.2) through
the same ladder operators, and evaluates E(theta) of Eq. 1 as <psi|H|psi>.
It also holds ADAPT-VQE's pool screening and adaptive loop (Sec. 2.1.1) and
pUCCD's hard-core boson form (Sec. 2.1.2), and the frozen-core folding of
Eq. 3 (Sec. 2.1.3).
Everything is numpy/scipy in float64 / complex128, dense or plain sparse, with
no blocking or fusion.

Parity status: every function here is pinned by a test under tests/ against a
closed form, a textbook special case, a library routine or a hand derivation;
the MLP oracle (when present) is pinned by finite differences.
"""
from .fermion import popcount, ladder, apply_string, fermion_matrix_op
from .hamiltonian import hamiltonian_matrix, sector_basis, full_basis
from .jw import jordan_wigner
from .pauli import pauli_dense, pauli_apply, pauli_sum_apply, pauli_sum_dense, pauli_sum_row
from .ansatz import (excitation_ops, apply_gate, apply_generator, prepare_state,
                     hf_state)
from .vqe import (energy, energy_pauli, gradient_direct, gradient_shift,
                  gradient_fd, exact_ground_energy, run_bfgs, EnergyModel)
from .adapt import pool_gradients, hf_pool_gradients, adapt_vqe
from .frozen import fold_frozen
from .hcb import (pair_basis, fermion_state, hcb_hamiltonian_matrix, HcbModel, hcb_gate,
                  hcb_generator, hcb_state, hcb_energy_grad)

__all__ = [
    "popcount", "ladder", "apply_string", "fermion_matrix_op", "hamiltonian_matrix",
    "sector_basis", "full_basis", "jordan_wigner", "pauli_dense", "pauli_apply",
    "pauli_sum_apply", "pauli_sum_dense", "pauli_sum_row", "excitation_ops", "apply_gate",
    "apply_generator", "prepare_state", "hf_state", "energy", "energy_pauli",
    "gradient_direct", "gradient_shift", "gradient_fd", "exact_ground_energy",
    "run_bfgs", "EnergyModel", "pool_gradients", "hf_pool_gradients", "adapt_vqe",
    "pair_basis", "fermion_state", "hcb_hamiltonian_matrix", "HcbModel", "hcb_gate", "hcb_generator",
    "hcb_state", "hcb_energy_grad", "fold_frozen",
]
