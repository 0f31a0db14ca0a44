"""Excitation pools and reference bitstrings (index enumeration only).

Qubit q is spin orbital q: spatial orbital q // 2, spin alpha when q is even and
beta when q is odd (interleaved order). Bit q of a basis index is qubit q.
The Hartree-Fock reference of Eq. 1 occupies the lowest n_elec spin orbitals,
so an odd electron count puts the extra electron in alpha.

The UCCSD pool of the paper (Sec. 2.1.2) holds single and double excitations
out of the reference. Each excitation is a 4-tuple: (i, a, -1, -1) for a single
i -> a and (i, j, a, b) with i < j occupied and a < b virtual for a double.
Only spin-conserving excitations enter: a single keeps its spin, a double keeps
the multiset of spins. Canonical order: singles by (i, a), then doubles by
(i, j, a, b).
"""
import numpy as np


def hf_bitstring(n_elec: int) -> int:
    return (1 << n_elec) - 1


def spin_counts(n_elec: int):
    """(N_alpha, N_beta) of the reference with the lowest n_elec spin orbitals filled."""
    return (n_elec + 1) // 2, n_elec // 2


def uccsd_pool(n_qubits: int, n_elec: int):
    occ = list(range(n_elec))
    virt = list(range(n_elec, n_qubits))
    singles = [(i, a, -1, -1) for i in occ for a in virt if i % 2 == a % 2]
    doubles = []
    for ii, i in enumerate(occ):
        for j in occ[ii + 1:]:
            for aa, a in enumerate(virt):
                for b in virt[aa + 1:]:
                    if sorted((i % 2, j % 2)) == sorted((a % 2, b % 2)):
                        doubles.append((i, j, a, b))
    return np.array(singles + doubles, dtype=np.int32).reshape(-1, 4)
