"""Random Pauli-sum inputs for kernel-level tests that do not come from chemistry.

A term is (x_mask, z_mask, coef): the string carries X on the qubits of x only,
Z on those of z only and Y where both bits are set. Coefficients are real.
Several terms are made to share an x mask so that X-mask groups hold more than
one term, and masks with an odd number of Y's are included (complex phases).
"""
import numpy as np


def random_pauli_terms(rng, n_qubits, n_terms, n_xmasks=None, max_weight=None, scale=1.0):
    full = (1 << n_qubits) - 1
    if n_xmasks is None:
        n_xmasks = max(1, n_terms // 4)
    xs_pool = [0]
    while len(xs_pool) < n_xmasks:
        if max_weight is None:
            x = int(rng.integers(0, full + 1))
        else:
            w = int(rng.integers(1, max_weight + 1))
            x = 0
            for q in rng.choice(n_qubits, size=min(w, n_qubits), replace=False):
                x |= 1 << int(q)
        xs_pool.append(x)
    xs = np.empty(n_terms, dtype=np.uint64)
    zs = np.empty(n_terms, dtype=np.uint64)
    for t in range(n_terms):
        xs[t] = xs_pool[int(rng.integers(0, len(xs_pool)))]
        zs[t] = int(rng.integers(0, full + 1))
    cs = rng.normal(0.0, scale, size=n_terms)
    return xs, zs, cs
