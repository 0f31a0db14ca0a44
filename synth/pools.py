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

The other chemistry ansatze of Sec. 2.1.2 use the same tuples:
  k-UpCCGSD: every spin-conserving single p -> q between spatial orbitals
    p < q (generalised: not only out of the reference), and every pair double
    (p alpha, p beta) -> (q alpha, q beta), p < q; the whole list repeated k
    times, each copy with its own angles.
  pUCCD: pair doubles out of the reference only (occupied spatial orbital i,
    virtual a), in the fermionic form on 2 n_s qubits; hcb_pair_pool gives
    the same excitations as (i, a) pairs for the hard-core boson form on n_s
    qubits (qubit p = spatial orbital p doubly occupied).
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


def upccgsd_pool(n_qubits: int, k: int = 1):
    n_s = n_qubits // 2
    singles, doubles = [], []
    for p in range(n_s):
        for q in range(p + 1, n_s):
            singles.append((2 * p, 2 * q, -1, -1))
            singles.append((2 * p + 1, 2 * q + 1, -1, -1))
            doubles.append((2 * p, 2 * p + 1, 2 * q, 2 * q + 1))
    one = np.array(singles + doubles, dtype=np.int32).reshape(-1, 4)
    return np.concatenate([one] * k) if k > 0 else one[:0]


def puccd_pool(n_qubits: int, n_elec: int):
    """Pair doubles out of a closed-shell reference (n_elec even)."""
    if n_elec % 2:
        raise ValueError("pUCCD needs an even electron count")
    n_s, n_occ = n_qubits // 2, n_elec // 2
    return np.array([(2 * i, 2 * i + 1, 2 * a, 2 * a + 1) for i in range(n_occ) for a in range(n_occ, n_s)],
                    dtype=np.int32).reshape(-1, 4)


def hcb_pair_pool(n_s: int, n_pairs: int):
    """pUCCD pair excitations i -> a (i < n_pairs <= a) as (i, a) on n_s boson qubits."""
    return np.array([(i, a) for i in range(n_pairs) for a in range(n_pairs, n_s)], dtype=np.int32).reshape(-1, 2)


def hcb_pairs_of(puccd_excitations):
    """(i, a) boson pairs of fermionic pair doubles (2i, 2i+1, 2a, 2a+1)."""
    e = np.asarray(puccd_excitations, dtype=np.int32).reshape(-1, 4)
    return np.ascontiguousarray(e[:, [0, 2]] // 2)
