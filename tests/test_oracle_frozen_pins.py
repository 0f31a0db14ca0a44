"""Pins of the oracle's frozen-core folding (Eq. 3, Sec. 2.1.3) against its
defining property: on determinants whose frozen orbitals are doubly occupied,
the full Hamiltonian of Eq. 2 and the folded one on the active orbitals have
the same matrix elements (brute force over the whole block)."""
import numpy as np
import pytest

import oracle
import synth


def _embed(d, active, frozen):
    """Full determinant of active determinant d (bit 2x+s = spin s of active[x])."""
    k = 0
    for c in frozen:
        k |= 3 << (2 * c)
    for x, p in enumerate(active):
        for s in (0, 1):
            if (d >> (2 * x + s)) & 1:
                k |= 1 << (2 * p + s)
    return k


@pytest.mark.parametrize("seed,n_s,n_elec,frozen", [(111, 4, 4, [0]), (112, 5, 6, [0, 1]),
                                                    (113, 5, 5, [0, 2]), (114, 6, 6, [1])])
def test_folded_block_equals_full_block(seed, n_s, n_elec, frozen):
    prob = synth.random_problem(np.random.default_rng(seed), n_s, n_elec, 3)
    prob.c0 = 0.125
    active = [p for p in range(n_s) if p not in frozen]
    red = oracle.fold_frozen(prob, frozen, active)
    na, nb = synth.spin_counts(n_elec)
    nf = len(frozen)
    small = oracle.sector_basis(2 * len(active), na - nf, nb - nf)
    Hs = oracle.hamiltonian_matrix(red, small).toarray()
    full = np.array(sorted(_embed(int(d), active, frozen) for d in small), dtype=np.uint64)
    order = np.argsort([_embed(int(d), active, frozen) for d in small])
    big = oracle.sector_basis(2 * n_s, na, nb)
    Hb = oracle.hamiltonian_matrix(prob, big).toarray()
    pos = np.searchsorted(big, full)
    block = Hb[np.ix_(pos, pos)]
    # rows/cols of block are in sorted full order; map the small basis to it
    inv = np.empty_like(order)
    inv[order] = np.arange(len(order))
    assert np.abs(block[np.ix_(inv, inv)] - Hs).max() < 1e-12
    assert np.abs(Hs).max() > 0.1


def test_folded_exact_energy_bounds_full_ci():
    prob = synth.random_problem(np.random.default_rng(115), 5, 6, 3)
    red = oracle.fold_frozen(prob, [0], [1, 2, 3, 4])
    assert oracle.exact_ground_energy(red) >= oracle.exact_ground_energy(prob) - 1e-12


def test_no_frozen_orbitals_is_identity():
    prob = synth.random_problem(np.random.default_rng(116), 4, 4, 3)
    red = oracle.fold_frozen(prob, [], [0, 1, 2, 3])
    assert np.array_equal(red.h, prob.h) and np.array_equal(red.eri, prob.eri) and red.c0 == prob.c0
