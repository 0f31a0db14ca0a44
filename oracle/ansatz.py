"""UCCSD-type excitation rotations U_k = exp(theta_k (T_k - T_k^dagger)) (Sec. 2.1.2).

Readings (the paper writes U = e^{T - T^dagger} and leaves the rest open):
* the full angle: U_k = exp(theta_k (T_k - T_k^dagger)) with no factor 1/2;
* single i -> a: T = a+_a a_i; double (i, j) -> (a, b), i < j, a < b:
  T = a+_a a+_b a_j a_i;
* one rotation per excitation, applied in list order: psi = U_M ... U_1 |HF>
  (one Trotter step of Sec. 2.1.2's UCCSD), |HF> the bitstring of Eq. 1's
  reference state.

For a basis state |k> with T|k> = s|k'> (s = +-1), the generator
A = T - T^dagger maps |k> -> s|k'> and |k'> -> -s|k>, and kills every state
outside such pairs, so exp(theta A) is the rotation
    psi'[k]  = cos(theta) psi[k] - s sin(theta) psi[k'],
    psi'[k'] = s sin(theta) psi[k] + cos(theta) psi[k'].
The tests pin this against scipy.linalg.expm of the dense generator.
"""
import numpy as np

from .fermion import apply_string


def excitation_ops(exc):
    """(T ops, T^dagger ops) for an excitation tuple (i, a, -1, -1) or (i, j, a, b)."""
    e = [int(v) for v in exc]
    if e[2] < 0:
        i, a = e[0], e[1]
        if i == a:
            raise ValueError("single excitation with i == a")
        return [(a, True), (i, False)], [(i, True), (a, False)]
    i, j, a, b = e
    if len({i, j, a, b}) != 4:
        raise ValueError("double excitation indices must be distinct")
    return ([(a, True), (b, True), (j, False), (i, False)],
            [(i, True), (j, True), (b, False), (a, False)])


def hf_state(n_qubits, hf_bits):
    psi = np.zeros(1 << n_qubits, dtype=complex)
    psi[int(hf_bits)] = 1.0
    return psi


def _pairs(n_qubits, exc):
    t_ops, _ = excitation_ops(exc)
    ks = np.arange(1 << n_qubits, dtype=np.uint64)
    new, sign, valid = apply_string(ks, t_ops)
    return ks[valid].astype(np.int64), new[valid].astype(np.int64), sign[valid].astype(float)


def apply_gate(psi, exc, theta):
    """exp(theta (T - T^dagger)) psi on a full state vector."""
    n = int(np.log2(len(psi)))
    k, kp, s = _pairs(n, exc)
    c, sn = np.cos(theta), np.sin(theta)
    out = psi.copy()
    out[k] = c * psi[k] - s * sn * psi[kp]
    out[kp] = s * sn * psi[k] + c * psi[kp]
    return out


def apply_generator(psi, exc):
    """(T - T^dagger) psi, applying the ladder operators of T and T^dagger literally."""
    n = int(np.log2(len(psi)))
    t_ops, td_ops = excitation_ops(exc)
    ks = np.arange(1 << n, dtype=np.uint64)
    out = np.zeros(len(psi), dtype=complex)
    new, sign, valid = apply_string(ks, t_ops)
    np.add.at(out, new[valid].astype(np.int64), sign[valid] * psi[valid])
    new, sign, valid = apply_string(ks, td_ops)
    np.add.at(out, new[valid].astype(np.int64), -sign[valid] * psi[valid])
    return out


def prepare_state(n_qubits, hf_bits, excitations, thetas):
    """psi(theta) = U_M ... U_1 |HF> (Eq. 1's U(theta)|0>)."""
    psi = hf_state(n_qubits, hf_bits)
    for exc, th in zip(excitations, thetas):
        psi = apply_gate(psi, exc, float(th))
    return psi
