"""pUCCD in the hard-core boson form (Sec. 2.1.2, pUCCD).

pUCCD moves electron pairs: T = a+_{a alpha} a+_{a beta} a_{i beta} a_{i alpha}.
Starting from a closed-shell reference, every state it reaches is a
combination of seniority-zero determinants (each spatial orbital empty or
doubly occupied), so its energy only needs the block P0 H P0 of Eq. 2 on those
determinants, and a determinant is fixed by which orbitals hold a pair: one
qubit per spatial orbital (the hard-core boson form, half the qubits).

Here the block comes from the fermionic operators themselves: every term of
Eq. 2 is applied by literal ladder operators to each seniority-zero
determinant and only results that are again seniority-zero are kept. Boson
basis state u (bit p = orbital p doubly occupied) is the determinant with
qubits 2p and 2p+1 set for every p in u. The pair rotation is
exp(theta (b+_a b_i - b+_i b_a)): on a pair (u, u') with u holding i and not a,
u' = u - i + a, it is psi'[u] = cos psi[u] - sin psi[u'], psi'[u'] = sin psi[u]
+ cos psi[u'] (the fermionic pair excitation maps the one determinant onto the
other with sign +1, which the tests pin against the fermionic route).

Test infrastructure: plain numpy, no code shared with the CUDA library.
"""
import itertools

import numpy as np
import scipy.sparse as sp

from .fermion import apply_string


def pair_basis(n_s, n_pairs):
    """Sorted boson bitstrings of n_pairs doubly occupied orbitals out of n_s."""
    out = [sum(1 << p for p in occ) for occ in itertools.combinations(range(n_s), n_pairs)]
    return np.array(sorted(out), dtype=np.uint64)


def fermion_state(u):
    """Determinant (bitstring on 2 n_s qubits) of boson bitstring u."""
    u = int(u)
    k, p = 0, 0
    while u >> p:
        if (u >> p) & 1:
            k |= 3 << (2 * p)
        p += 1
    return k


def hcb_hamiltonian_matrix(problem, n_pairs):
    """P0 H P0 of Eq. 2 in the boson basis pair_basis(n_s, n_pairs) (csr)."""
    n_s = problem.n_spatial
    bos = pair_basis(n_s, n_pairs)
    det = np.array([fermion_state(u) for u in bos], dtype=np.uint64)
    order = np.argsort(det)
    det_sorted = det[order]
    dim = len(bos)
    rows, cols, vals = [], [], []

    def add(coef, ops):
        new, sign, valid = apply_string(det, ops)
        if not valid.any():
            return
        src = np.nonzero(valid)[0]
        dst_states = new[valid]
        pos = np.minimum(np.searchsorted(det_sorted, dst_states), dim - 1)
        keep = det_sorted[pos] == dst_states   # projection onto seniority zero
        if not keep.any():
            return
        rows.append(order[pos[keep]])
        cols.append(src[keep])
        vals.append(coef * sign[valid][keep].astype(float))

    if problem.c0 != 0.0:
        rows.append(np.arange(dim))
        cols.append(np.arange(dim))
        vals.append(np.full(dim, float(problem.c0)))
    h, eri = problem.h, problem.eri
    for p in range(n_s):
        for q in range(n_s):
            if h[p, q] != 0.0:
                for sg in (0, 1):
                    add(h[p, q], [(2 * p + sg, True), (2 * q + sg, False)])
    for p, q, r, s in itertools.product(range(n_s), repeat=4):
        g = eri[p, q, r, s]
        if g == 0.0:
            continue
        for sg in (0, 1):
            for tau in (0, 1):
                add(0.5 * g, [(2 * p + sg, True), (2 * r + tau, True), (2 * s + tau, False), (2 * q + sg, False)])
    if not rows:
        return sp.csr_matrix((dim, dim)), bos
    m = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(dim, dim))
    return m.tocsr(), bos


class HcbModel:
    """P0 H P0 acting on full 2^{n_s} boson state vectors (zero outside the sector)."""

    def __init__(self, problem, n_pairs):
        self.n_qubits = problem.n_spatial
        self.matrix, self.basis = hcb_hamiltonian_matrix(problem, n_pairs)
        self._idx = self.basis.astype(np.int64)

    def apply(self, psi):
        out = np.zeros(1 << self.n_qubits, dtype=complex)
        out[self._idx] = self.matrix @ psi[self._idx]
        return out


def _pairs(n, i, a):
    ks = np.arange(1 << n, dtype=np.int64)
    lower = ks[(((ks >> i) & 1) == 1) & (((ks >> a) & 1) == 0)]
    return lower, lower ^ ((1 << i) | (1 << a))


def hcb_gate(psi, i, a, theta):
    n = int(np.log2(len(psi)))
    k, kp = _pairs(n, i, a)
    c, s = np.cos(theta), np.sin(theta)
    out = psi.copy()
    out[k] = c * psi[k] - s * psi[kp]
    out[kp] = s * psi[k] + c * psi[kp]
    return out


def hcb_generator(psi, i, a):
    """(b+_a b_i - b+_i b_a) psi."""
    n = int(np.log2(len(psi)))
    k, kp = _pairs(n, i, a)
    out = np.zeros(len(psi), dtype=complex)
    out[kp] += psi[k]
    out[k] -= psi[kp]
    return out


def hcb_state(n_s, hf_bits, pairs, thetas):
    psi = np.zeros(1 << n_s, dtype=complex)
    psi[int(hf_bits)] = 1.0
    for (i, a), t in zip(pairs, thetas):
        psi = hcb_gate(psi, int(i), int(a), float(t))
    return psi


def hcb_energy_grad(model, hf_bits, pairs, thetas):
    """E(theta) and g_k = 2 Re <H psi| U_M .. U_{k+1} A_k U_k .. U_1 |HF> (O(M^2) gates)."""
    pairs = np.asarray(pairs, dtype=np.int64).reshape(-1, 2)
    thetas = np.asarray(thetas, dtype=float)
    states = [hcb_state(model.n_qubits, hf_bits, [], [])]
    for (i, a), t in zip(pairs, thetas):
        states.append(hcb_gate(states[-1], int(i), int(a), float(t)))
    psi = states[-1]
    hpsi = model.apply(psi)
    g = np.zeros(len(pairs))
    for k, (i, a) in enumerate(pairs):
        v = hcb_generator(states[k + 1], int(i), int(a))
        for m in range(k + 1, len(pairs)):
            v = hcb_gate(v, int(pairs[m][0]), int(pairs[m][1]), float(thetas[m]))
        g[k] = 2.0 * np.vdot(hpsi, v).real
    return float(np.vdot(psi, hpsi).real), g
