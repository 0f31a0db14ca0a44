"""Pauli strings: dense Kronecker matrices and explicit action on a state vector.

A string is given by masks (x, z): qubit q carries I, X, Z or Y for
(x_q, z_q) = (0,0), (1,0), (0,1), (1,1). Bit q of a basis index is qubit q, so
the dense matrix is the Kronecker product with the highest qubit leftmost.
The explicit action on a basis state is
    P(x, z) |k> = i^{|x & z|} (-1)^{|k & z|} |k XOR x>,
which the tests pin against the Kronecker product.
"""
import numpy as np

from .fermion import popcount

_I = np.eye(2, dtype=complex)
_X = np.array([[0, 1], [1, 0]], dtype=complex)
_Y = np.array([[0, -1j], [1j, 0]], dtype=complex)
_Z = np.array([[1, 0], [0, -1]], dtype=complex)


def _single(xq, zq):
    return {(0, 0): _I, (1, 0): _X, (0, 1): _Z, (1, 1): _Y}[(xq, zq)]


def pauli_dense(x, z, n_qubits):
    x, z = int(x), int(z)
    m = np.ones((1, 1), dtype=complex)
    for q in range(n_qubits - 1, -1, -1):
        m = np.kron(m, _single((x >> q) & 1, (z >> q) & 1))
    return m


def pauli_sum_dense(xs, zs, cs, n_qubits):
    dim = 1 << n_qubits
    out = np.zeros((dim, dim), dtype=complex)
    for x, z, c in zip(xs, zs, cs):
        out += c * pauli_dense(x, z, n_qubits)
    return out


def pauli_apply(x, z, psi):
    """P(x, z) psi for a full state vector psi of length 2^n."""
    dim = len(psi)
    ks = np.arange(dim, dtype=np.uint64)
    x = np.uint64(int(x))
    z = np.uint64(int(z))
    phase = (1j) ** int(popcount(np.array([x & z]))[0])
    sign = 1 - 2 * (popcount(ks & z) & 1)
    out = np.zeros(dim, dtype=complex)
    out[(ks ^ x).astype(np.int64)] = phase * sign * psi
    return out


def pauli_sum_apply(xs, zs, cs, psi):
    out = np.zeros(len(psi), dtype=complex)
    for x, z, c in zip(xs, zs, cs):
        out += c * pauli_apply(x, z, psi)
    return out


def pauli_sum_row(xs, zs, cs, k, amp):
    """(H psi)[k] for H = sum_t c_t P(x_t, z_t), where amp(indices) returns psi
    at an array of basis indices. From the action above, the amplitude at k
    comes from source j = k XOR x_t:
        (H psi)[k] = sum_t c_t i^{|x_t & z_t|} (-1)^{|j_t & z_t|} psi[j_t].
    For one output row of a state too large to hold on the host."""
    xs = np.asarray(xs, dtype=np.uint64)
    zs = np.asarray(zs, dtype=np.uint64)
    cs = np.asarray(cs)
    src = np.uint64(int(k)) ^ xs
    phase = np.array([1, 1j, -1, -1j])[popcount(xs & zs) % 4]
    sign = 1 - 2 * (popcount(src & zs) & 1)
    return complex(np.sum(cs * phase * sign * amp(src)))
