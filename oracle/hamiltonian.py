"""The molecular Hamiltonian of Eq. 2 as a sparse matrix in a basis of bitstrings.

Reading of Eq. 2 (the paper writes the two-body sum without a factor and
without an index order): with spatial integrals h_pq and chemists'-order
two-body integrals (pq|rs),

    H = c0 + sum_{p,q,sigma} h_pq a+_{p,sigma} a_{q,sigma}
           + 1/2 sum_{p,q,r,s,sigma,tau} (pq|rs) a+_{p,sigma} a+_{r,tau} a_{s,tau} a_{q,sigma}

with sigma, tau running over both spins. Spin orbital (p, sigma) is qubit
2p + sigma (sigma = 0 alpha, 1 beta). Every matrix element comes from applying
the ladder operators literally to each basis state.
"""
import itertools

import numpy as np
import scipy.sparse as sp

from .fermion import apply_string


def full_basis(n_qubits):
    return np.arange(1 << n_qubits, dtype=np.uint64)


def sector_basis(n_qubits, n_alpha, n_beta):
    """Sorted bitstrings with n_alpha electrons on even qubits and n_beta on odd."""
    n_s = n_qubits // 2
    alphas = []
    for occ in itertools.combinations(range(n_s), n_alpha):
        alphas.append(sum(1 << (2 * p) for p in occ))
    betas = []
    for occ in itertools.combinations(range(n_s), n_beta):
        betas.append(sum(1 << (2 * p + 1) for p in occ))
    a = np.array(alphas, dtype=np.uint64)
    b = np.array(betas, dtype=np.uint64)
    ks = (a[:, None] | b[None, :]).ravel()
    return np.sort(ks)


def _add_term(rows, cols, vals, basis, coef, ops):
    new, sign, valid = apply_string(basis, ops)
    if not valid.any():
        return
    src = np.nonzero(valid)[0]
    dst_states = new[valid]
    dst = np.searchsorted(basis, dst_states)
    dst = np.minimum(dst, len(basis) - 1)
    if not np.array_equal(basis[dst], dst_states):
        raise ValueError("basis is not closed under the Hamiltonian")
    rows.append(dst)
    cols.append(src)
    vals.append(coef * sign[valid].astype(float))


def hamiltonian_matrix(problem, basis):
    """Sparse (csr) matrix <basis_i|H|basis_j> of Eq. 2 for a synth.Problem."""
    n_s = problem.n_spatial
    basis = np.asarray(basis, dtype=np.uint64)
    dim = len(basis)
    rows, cols, vals = [], [], []
    if problem.c0 != 0.0:
        idx = np.arange(dim)
        rows.append(idx)
        cols.append(idx)
        vals.append(np.full(dim, float(problem.c0)))
    h = problem.h
    for p in range(n_s):
        for q in range(n_s):
            if h[p, q] == 0.0:
                continue
            for sg in (0, 1):
                _add_term(rows, cols, vals, basis, h[p, q],
                          [(2 * p + sg, True), (2 * q + sg, False)])
    eri = problem.eri
    for p in range(n_s):
        for q in range(n_s):
            for r in range(n_s):
                for s in range(n_s):
                    g = eri[p, q, r, s]
                    if g == 0.0:
                        continue
                    for sg in (0, 1):
                        for tau in (0, 1):
                            _add_term(rows, cols, vals, basis, 0.5 * g,
                                      [(2 * p + sg, True), (2 * r + tau, True),
                                       (2 * s + tau, False), (2 * q + sg, False)])
    if not rows:
        return sp.csr_matrix((dim, dim))
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    v = np.concatenate(vals)
    return sp.coo_matrix((v, (r, c)), shape=(dim, dim)).tocsr()
