"""Pins of the oracle's hard-core boson form of pUCCD (Sec. 2.1.2, pUCCD).

The boson route (seniority-zero block of Eq. 2, pair rotations without a
parity sign, n_s qubits) must give the energies and gradients of the fermionic
route (pair doubles applied as four ladder operators on 2 n_s qubits with the
full Hamiltonian); the block itself must match the two-orbital closed form and
the Slater-Condon diagonal."""
import itertools

import numpy as np
import pytest

import oracle
import synth


def _problem(seed, n_s, n_elec, K=3):
    return synth.random_problem(np.random.default_rng(seed), n_s, n_elec, K)


@pytest.mark.parametrize("seed,n_s,n_pairs", [(81, 3, 1), (82, 4, 2), (83, 5, 2)])
def test_boson_route_equals_fermionic_route(seed, n_s, n_pairs):
    prob = _problem(seed, n_s, 2 * n_pairs)
    th = np.random.default_rng(seed + 100).normal(0, 0.4, size=n_pairs * (n_s - n_pairs))
    ferm = oracle.EnergyModel.from_problem(prob)
    e_f, g_f = oracle.gradient_direct(ferm, synth.hf_bitstring(2 * n_pairs),
                                      synth.puccd_pool(2 * n_s, 2 * n_pairs), th)
    hcb = oracle.HcbModel(prob, n_pairs)
    e_b, g_b = oracle.hcb_energy_grad(hcb, (1 << n_pairs) - 1, synth.hcb_pair_pool(n_s, n_pairs), th)
    assert abs(e_f - e_b) < 1e-12
    assert np.abs(g_f - g_b).max() < 1e-12
    assert np.abs(g_b).max() > 1e-3


def test_two_orbitals_one_pair_closed_form():
    """Basis (pair on orbital 0, pair on orbital 1): diagonal 2 h_pp + (pp|pp)
    (+ c0), off-diagonal (01|01)."""
    prob = _problem(84, 2, 2)
    prob.c0 = 0.375
    m, bos = oracle.hcb_hamiltonian_matrix(prob, 1)
    h, v = prob.h, prob.eri
    want = np.array([[2 * h[0, 0] + v[0, 0, 0, 0], v[0, 1, 0, 1]],
                     [v[0, 1, 0, 1], 2 * h[1, 1] + v[1, 1, 1, 1]]]) + 0.375 * np.eye(2)
    assert list(bos) == [1, 2]
    assert np.abs(m.toarray() - want).max() < 1e-14


def test_diagonal_is_slater_condon_of_pair_determinants():
    prob = _problem(85, 5, 4)
    m, bos = oracle.hcb_hamiltonian_matrix(prob, 2)
    h, v = prob.h, prob.eri
    for r, u in enumerate(bos):
        occ = [p for p in range(5) if (int(u) >> p) & 1]
        e = sum(2 * h[p, p] + v[p, p, p, p] for p in occ)
        e += sum(2 * v[p, p, q, q] - v[p, q, q, p] for p, q in itertools.permutations(occ, 2))
        assert abs(m[r, r] - e) < 1e-13


def test_block_is_symmetric_and_above_full_ci():
    prob = _problem(86, 5, 4)
    m, _ = oracle.hcb_hamiltonian_matrix(prob, 2)
    a = m.toarray()
    assert np.abs(a - a.T).max() < 1e-14
    assert np.linalg.eigvalsh(a)[0] >= oracle.exact_ground_energy(prob) - 1e-12
