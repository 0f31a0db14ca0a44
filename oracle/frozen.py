"""Frozen-core folding of Eq. 3 (Sec. 2.1.3, orbital reduction).

Frozen spatial orbitals F are doubly occupied in every determinant; the
Hamiltonian on the active orbitals A keeps the active integrals and absorbs
the frozen ones into a constant and an effective one-body term. Eq. 3 prints
the one-body fold over frozen spin orbitals k as four integrals
(h_kijk - h_kikj + h_ikkj - h_ikjk); summed over both spins of each frozen
spatial orbital c and written with chemists' integrals (pq|rs) this is
    h'_pq = h_pq + sum_{c in F} [2 (pq|cc) - (pc|cq)].
Eq. 3's constant shows only sum_{i in F} h_ii over frozen spin orbitals; the
energy of the frozen pairs among themselves belongs to it as well, so the
reading taken here is the full core energy
    c0' = c0 + sum_{c in F} 2 h_cc + sum_{c, d in F} [2 (cc|dd) - (cd|dc)].
The tests pin this against the defining property: for every determinant with
F doubly occupied, the full Hamiltonian's matrix elements equal the folded
one's on the active part.

Test infrastructure: plain numpy, no code shared with the CUDA library.
"""
import numpy as np


def fold_frozen(problem, frozen, active):
    """synth.Problem on the active orbitals (in the given order) with the
    frozen orbitals folded in; its electron count drops by 2 per frozen orbital."""
    from synth import Problem

    F = [int(c) for c in frozen]
    A = [int(p) for p in active]
    if set(F) & set(A):
        raise ValueError("an orbital is both frozen and active")
    h, v = problem.h, problem.eri
    c0 = problem.c0
    for c in F:
        c0 += 2.0 * h[c, c]
        for d in F:
            c0 += 2.0 * v[c, c, d, d] - v[c, d, d, c]
    ha = np.zeros((len(A), len(A)))
    for x, p in enumerate(A):
        for y, q in enumerate(A):
            ha[x, y] = h[p, q] + sum(2.0 * v[p, q, c, c] - v[p, c, c, q] for c in F)
    va = v[np.ix_(A, A, A, A)].copy()
    return Problem(len(A), problem.n_elec - 2 * len(F), ha, va, c0, problem.label + " (frozen core)")
