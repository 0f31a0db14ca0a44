"""The oracle's own Jordan-Wigner mapping of Eq. 2 to a Pauli sum (Sec. 2.1.1).

Operators are kept symbolically as sums of products X^x Z^z (X on the qubits
of mask x, then Z on those of mask z). Under Jordan-Wigner, spin orbital p is
qubit p and

    a_p  = Z_{<p} (X_p + i Y_p)/2 = (X^{p} Z^{<p} - X^{p} Z^{<p,p}) / 2,
    a+_p = Z_{<p} (X_p - i Y_p)/2 = (X^{p} Z^{<p} + X^{p} Z^{<p,p}) / 2,

using Y = i X Z. Two products multiply as
(X^a Z^b)(X^c Z^d) = (-1)^{|b & c|} X^{a^c} Z^{b^d}. The result is expressed in
Pauli strings P(x, z) = i^{|x & z|} X^x Z^z (Y where both bits are set), so a
coefficient c on X^x Z^z becomes c (-i)^{|x & z|} on P(x, z).
"""
import numpy as np


def _pc(v: int) -> int:
    return bin(v).count("1")


def _mul(a, b):
    out = {}
    for (x1, z1), c1 in a.items():
        for (x2, z2), c2 in b.items():
            c = c1 * c2
            if _pc(z1 & x2) & 1:
                c = -c
            key = (x1 ^ x2, z1 ^ z2)
            out[key] = out.get(key, 0.0) + c
    return out


def _ladder(p, dagger):
    bit = 1 << p
    below = bit - 1
    return {(bit, below): 0.5, (bit, below | bit): (0.5 if dagger else -0.5)}


def _product(ops):
    acc = {(0, 0): 1.0 + 0.0j}
    for p, dag in ops:
        acc = _mul(acc, _ladder(p, dag))
    return acc


def _accumulate(total, coef, ops):
    for key, c in _product(ops).items():
        total[key] = total.get(key, 0.0) + coef * c


def jordan_wigner(problem, drop_tol=1e-14, imag_tol=1e-10):
    """Pauli sum of Eq. 2 for a synth.Problem: (x_masks, z_masks, real coefs).

    Terms with equal masks are merged; terms with |coef| < drop_tol are dropped.
    Raises if a merged coefficient has an imaginary part above imag_tol.
    """
    n_s = problem.n_spatial
    total = {}
    if problem.c0 != 0.0:
        total[(0, 0)] = complex(problem.c0)
    h = problem.h
    for p in range(n_s):
        for q in range(n_s):
            if h[p, q] == 0.0:
                continue
            for sg in (0, 1):
                _accumulate(total, h[p, q], [(2 * p + sg, True), (2 * q + sg, False)])
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
                            _accumulate(total, 0.5 * g,
                                        [(2 * p + sg, True), (2 * r + tau, True),
                                         (2 * s + tau, False), (2 * q + sg, False)])
    xs, zs, cs = [], [], []
    for (x, z), c in sorted(total.items()):
        cp = c * ((-1j) ** _pc(x & z))
        if abs(cp.imag) > imag_tol:
            raise ValueError(f"non-real Pauli coefficient {cp} for x={x:#x} z={z:#x}")
        if abs(cp.real) < drop_tol:
            continue
        xs.append(x)
        zs.append(z)
        cs.append(cp.real)
    return (np.array(xs, dtype=np.uint64), np.array(zs, dtype=np.uint64),
            np.array(cs, dtype=np.float64))
