"""Pins of the oracle's ADAPT-VQE screening (Sec. 2.1.1, ADAPT-VQE) against facts
fixed outside it: the exact four-point shift rule of the extended ansatz, the
Slater-Condon closed form at the reference state, the identity between the pool
gradient of the last gate's own operator and that gate's angle derivative, and
the full-CI energy that the adaptive loop must reach on the 4-qubit problem."""
import numpy as np
import pytest

import oracle
import synth


def _problem(seed, n_s, n_elec, K=3):
    return synth.random_problem(np.random.default_rng(seed), n_s, n_elec, K)


def test_pool_gradient_is_shift_rule_of_appended_operator():
    """g_j = dE/dt at t = 0 of the ansatz with pool operator j appended, taken by
    the exact four-point shift rule (energies only)."""
    prob = _problem(51, 4, 4)
    model = oracle.EnergyModel.from_problem(prob)
    pool = synth.uccsd_pool(8, 4)
    rng = np.random.default_rng(52)
    exc = pool[rng.permutation(len(pool))[:5]]
    th = rng.normal(0, 0.3, size=5)
    e, g = oracle.pool_gradients(model, 15, exc, th, pool)
    assert abs(e - oracle.energy(model, 15, exc, th)) < 1e-14
    for j in range(len(pool)):
        ext = np.concatenate([exc, pool[j:j + 1]])
        gs = oracle.gradient_shift(model, 15, ext, np.append(th, 0.0), indices=[5])
        assert abs(g[j] - gs[0]) < 1e-12, j
    assert np.abs(g).max() > 1e-3


@pytest.mark.parametrize("seed,n_s,n_elec", [(61, 3, 2), (62, 4, 4), (63, 5, 3), (64, 4, 5)])
def test_reference_state_gradients_match_slater_condon(seed, n_s, n_elec):
    """At psi = |HF> (empty ansatz) g_j = 2 <HF|H T_j|HF>: Fock elements for
    singles, antisymmetrised integrals for doubles (odd N included)."""
    prob = _problem(seed, n_s, n_elec)
    model = oracle.EnergyModel.from_problem(prob)
    hf = synth.hf_bitstring(n_elec)
    pool = synth.uccsd_pool(2 * n_s, n_elec)
    _, g = oracle.pool_gradients(model, hf, pool[:0], [], pool)
    g_sc = oracle.hf_pool_gradients(prob, hf, pool)
    assert np.abs(g - g_sc).max() < 1e-12
    assert np.abs(g_sc).max() > 1e-2


def test_pool_gradient_of_last_gate_equals_its_angle_derivative():
    """A_M commutes with U_M = exp(theta_M A_M), so appending A_M again at angle 0
    moves E as theta_M does: the pool gradient equals dE/dtheta_M."""
    prob = _problem(71, 4, 4)
    model = oracle.EnergyModel.from_problem(prob)
    pool = synth.uccsd_pool(8, 4)
    rng = np.random.default_rng(72)
    idx = rng.permutation(len(pool))[:6]
    th = rng.normal(0, 0.4, size=6)
    _, g = oracle.pool_gradients(model, 15, pool[idx], th, pool)
    _, gd = oracle.gradient_direct(model, 15, pool[idx], th)
    assert abs(g[idx[-1]] - gd[-1]) < 1e-12


def test_adapt_reaches_full_ci_on_four_qubits():
    """config 0's sector is 4-dimensional and real; ADAPT from the full UCCSD pool
    reaches the full-CI energy, every round lowers E, and E stays above E0."""
    w = synth.config0()
    prob = w.problems[0]
    model = oracle.EnergyModel.from_problem(prob)
    e0 = oracle.exact_ground_energy(prob)
    e, chosen, theta, hist = oracle.adapt_vqe(model, 3, w.excitations[0], grad_tol=1e-6, max_ops=6)
    assert abs(e - e0) < 1e-8
    es = [h[0] for h in hist]
    assert all(b <= a + 1e-12 for a, b in zip(es, es[1:]))
    assert min(es) >= e0 - 1e-12
    assert hist[-1][1] < 1e-6
