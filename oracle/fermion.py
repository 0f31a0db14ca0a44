"""Fermionic ladder operators on occupation-number basis states.

Basis state |k>: bit p of k is the occupation of spin orbital p. Following the
second-quantised form of Eq. 2, a_p removes and a_p^dagger adds an electron in
orbital p, each with the sign (-1)^(number of occupied orbitals with index < p).
That ordering convention is the one the Jordan-Wigner mapping (Sec. 2.1.1)
reproduces with Z strings on the lower qubits.
"""
import numpy as np

_M1 = np.uint64(0x5555555555555555)
_M2 = np.uint64(0x3333333333333333)
_M4 = np.uint64(0x0F0F0F0F0F0F0F0F)
_H01 = np.uint64(0x0101010101010101)


def popcount(a):
    """Number of set bits of each uint64 entry (int64 result)."""
    a = np.asarray(a, dtype=np.uint64)
    if hasattr(np, "bitwise_count"):
        return np.bitwise_count(a).astype(np.int64)
    a = a - ((a >> np.uint64(1)) & _M1)
    a = (a & _M2) + ((a >> np.uint64(2)) & _M2)
    a = (a + (a >> np.uint64(4))) & _M4
    return ((a * _H01) >> np.uint64(56)).astype(np.int64)


def ladder(ks, p, dagger):
    """Apply a_p (dagger False) or a_p^dagger (dagger True) to each basis state.

    Returns (new_ks, sign, valid); entries with valid False are annihilated.
    """
    ks = np.asarray(ks, dtype=np.uint64)
    bit = np.uint64(1) << np.uint64(p)
    occupied = (ks & bit) != 0
    valid = ~occupied if dagger else occupied
    below = bit - np.uint64(1)
    sign = 1 - 2 * (popcount(ks & below) & 1)
    return ks ^ bit, sign, valid


def apply_string(ks, ops):
    """Apply an operator product to basis states.

    ops lists (orbital, dagger) factors left to right as written; the rightmost
    factor acts first. Returns (new_ks, sign, valid).
    """
    cur = np.asarray(ks, dtype=np.uint64).copy()
    sign = np.ones(cur.shape, dtype=np.int64)
    valid = np.ones(cur.shape, dtype=bool)
    for p, dag in reversed(ops):
        cur, s, v = ladder(cur, p, dag)
        sign = sign * s
        valid &= v
    return cur, sign, valid


def fermion_matrix_op(ops, n_qubits):
    """Dense 2^n x 2^n matrix of an operator product (small n only)."""
    dim = 1 << n_qubits
    ks = np.arange(dim, dtype=np.uint64)
    new, sign, valid = apply_string(ks, ops)
    m = np.zeros((dim, dim))
    m[new[valid].astype(np.int64), ks[valid].astype(np.int64)] = sign[valid]
    return m
