"""Pins of the CPU oracle against facts fixed outside it.

Each test checks the oracle against a closed form, a textbook identity, a
library routine, a hand derivation (tests/golden) or brute force, so that a
dropped term, a wrong sign or index, or a transposed operand in the oracle
fails at least one of them.
"""
import itertools
import os

import numpy as np
import pytest
import scipy.linalg as sla

import oracle
import synth
from oracle.fermion import fermion_matrix_op

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_problem(seed, n_s, n_elec, K=3):
    return synth.random_problem(np.random.default_rng(seed), n_s, n_elec, K)


# ---------------------------------------------------------------- ladder algebra
def test_canonical_anticommutation():
    """{a_p, a_q^dagger} = delta_pq, {a_p, a_q} = 0 (second quantisation of Eq. 2)."""
    n = 4
    dim = 1 << n
    a = [fermion_matrix_op([(p, False)], n) for p in range(n)]
    ad = [fermion_matrix_op([(p, True)], n) for p in range(n)]
    for p in range(n):
        assert np.array_equal(ad[p], a[p].T)
        for q in range(n):
            acomm = a[p] @ ad[q] + ad[q] @ a[p]
            assert np.array_equal(acomm, np.eye(dim) * (p == q))
            assert not np.any(a[p] @ a[q] + a[q] @ a[p])


def test_number_operator_counts_electrons():
    n = 4
    N = sum(fermion_matrix_op([(p, True), (p, False)], n) for p in range(n))
    ks = np.arange(1 << n)
    assert np.array_equal(np.diag(N), [bin(k).count("1") for k in ks])
    assert np.count_nonzero(N - np.diag(np.diag(N))) == 0


# ---------------------------------------------------------------- Hamiltonian
def test_two_body_operator_identity():
    """For (pq|rs) = L_pq L_rs the two-body part of Eq. 2 equals
    1/2 (O^2 - sum_ps (L^2)_ps E_ps), O = sum_pq L_pq E_pq, E_pq = sum_s a+_ps a_qs
    (anticommutation identity), pinning operator order and the factor 1/2."""
    rng = np.random.default_rng(11)
    n_s = 3
    L = synth.draw_factors(rng, n_s, 1)[0]
    zero_h = np.zeros((n_s, n_s))
    two = synth.Problem(n_s, 2, zero_h, np.einsum("pq,rs->pqrs", L, L))
    basis = oracle.full_basis(2 * n_s)
    H2 = oracle.hamiltonian_matrix(two, basis).toarray()
    O = oracle.hamiltonian_matrix(synth.Problem(n_s, 2, L, np.zeros((n_s,) * 4)), basis).toarray()
    OL2 = oracle.hamiltonian_matrix(synth.Problem(n_s, 2, L @ L, np.zeros((n_s,) * 4)),
                                    basis).toarray()
    assert np.abs(H2 - 0.5 * (O @ O - OL2)).max() < 1e-13


@pytest.mark.parametrize("seed,n_s,n_elec", [(0, 2, 2), (1, 3, 2), (2, 3, 3), (3, 4, 4)])
def test_slater_condon_hf_energy(seed, n_s, n_elec):
    """E(theta=0) is the Hartree-Fock energy (Sec. 3.2 uses this), whose closed form
    is sum_P h_pp + 1/2 sum_{P,Q} [(pp|qq) - delta_{sP sQ} (pq|qp)] over occupied
    spin orbitals P = (p, sP)."""
    prob = _rand_problem(seed, n_s, n_elec)
    occ = list(range(n_elec))
    e_sc = sum(prob.h[P // 2, P // 2] for P in occ)
    for P in occ:
        for Q in occ:
            p, q = P // 2, Q // 2
            e_sc += 0.5 * prob.eri[p, p, q, q]
            if P % 2 == Q % 2:
                e_sc -= 0.5 * prob.eri[p, q, q, p]
    model = oracle.EnergyModel.from_problem(prob)
    hf = synth.hf_bitstring(n_elec)
    exc = synth.uccsd_pool(2 * n_s, n_elec)
    assert abs(oracle.energy(model, hf, exc, np.zeros(len(exc))) - e_sc) < 1e-12
    xs, zs, cs = oracle.jordan_wigner(prob)
    diag = sum(c * (-1) ** bin(hf & int(z)).count("1") for x, z, c in zip(xs, zs, cs) if x == 0)
    assert abs(diag - e_sc) < 1e-12


def test_one_body_ground_energy():
    """With no two-body term the sector ground energy is the sum of the lowest
    N_alpha and N_beta eigenvalues of h (non-interacting fermions)."""
    rng = np.random.default_rng(5)
    for n_s, n_elec in [(3, 2), (4, 3), (5, 4)]:
        h = synth.draw_one_body(rng, n_s)
        prob = synth.Problem(n_s, n_elec, h, np.zeros((n_s,) * 4))
        eps = np.linalg.eigvalsh(h)
        na, nb = synth.spin_counts(n_elec)
        assert abs(oracle.exact_ground_energy(prob) - (eps[:na].sum() + eps[:nb].sum())) < 1e-12


@pytest.mark.parametrize("seed,n_s,n_elec", [(0, 2, 2), (1, 3, 3), (2, 4, 4)])
def test_jordan_wigner_matches_fermionic_matrix(seed, n_s, n_elec):
    """Route 1 (ladder operators) equals route 2 (Kronecker products of the JW
    Pauli sum) element by element; the JW coefficients are real."""
    prob = _rand_problem(seed, n_s, n_elec)
    n = 2 * n_s
    H1 = oracle.hamiltonian_matrix(prob, oracle.full_basis(n)).toarray()
    assert np.abs(H1 - H1.T).max() < 1e-14
    xs, zs, cs = oracle.jordan_wigner(prob)
    H2 = oracle.pauli_sum_dense(xs, zs, cs, n)
    assert np.abs(H1 - H2).max() < 1e-13
    assert len(set(zip(xs.tolist(), zs.tolist()))) == len(xs)


def test_jw_term_and_group_counts_config0():
    """Config 0's Pauli sum stays within the upper bounds 1 + n + C(n,2) + ... and
    G = 1 + 2 C(n_s,2) + Q for n = 4."""
    w = synth.config0()
    xs, zs, cs = oracle.jordan_wigner(w.problems[0])
    assert 15 <= len(xs) <= 31
    assert len(set(xs.tolist())) <= 4


# ---------------------------------------------------------------- Pauli action
def test_pauli_action_matches_kronecker():
    rng = np.random.default_rng(7)
    n = 5
    for _ in range(20):
        x, z = int(rng.integers(0, 32)), int(rng.integers(0, 32))
        psi = rng.normal(size=32) + 1j * rng.normal(size=32)
        assert np.abs(oracle.pauli_apply(x, z, psi) - oracle.pauli_dense(x, z, n) @ psi).max() < 1e-14


def test_pauli_sum_row_matches_kronecker_rows():
    """One output row of H psi (for states too large for the host) equals the
    row of the Kronecker-product matrix times psi, including Y phases."""
    rng = np.random.default_rng(11)
    n = 6
    xs = rng.integers(0, 64, size=40).astype(np.uint64)
    zs = rng.integers(0, 64, size=40).astype(np.uint64)
    cs = rng.normal(size=40)
    psi = rng.normal(size=64) + 1j * rng.normal(size=64)
    full = oracle.pauli_sum_dense(xs, zs, cs, n) @ psi
    for k in range(64):
        row = oracle.pauli_sum_row(xs, zs, cs, k, lambda idx: psi[idx.astype(np.int64)])
        assert abs(row - full[k]) < 1e-13


def test_single_qubit_paulis_are_textbook():
    X = oracle.pauli_dense(1, 0, 1)
    Z = oracle.pauli_dense(0, 1, 1)
    Y = oracle.pauli_dense(1, 1, 1)
    assert np.array_equal(X, [[0, 1], [1, 0]])
    assert np.array_equal(Z, [[1, 0], [0, -1]])
    assert np.array_equal(Y, [[0, -1j], [1j, 0]])
    # qubit 0 is the least significant bit of the basis index
    assert np.array_equal(oracle.pauli_dense(1, 0, 2) @ np.eye(4)[:, 0], np.eye(4)[:, 1])


def test_z_only_energy_is_weighted_diagonal():
    rng = np.random.default_rng(8)
    n = 6
    zs = rng.integers(0, 64, size=10).astype(np.uint64)
    xs = np.zeros(10, dtype=np.uint64)
    cs = rng.normal(size=10)
    psi = rng.normal(size=64) + 1j * rng.normal(size=64)
    diag = np.array([sum(c * (-1) ** bin(k & int(z)).count("1") for z, c in zip(zs, cs))
                     for k in range(64)])
    e, im = oracle.EnergyModel.from_pauli(n, xs, zs, cs).expectation(psi)
    assert abs(e - np.sum(np.abs(psi) ** 2 * diag)) < 1e-12 and abs(im) < 1e-12


# ---------------------------------------------------------------- gates
def _generator_dense(exc, n):
    t_ops, td_ops = oracle.excitation_ops(exc)
    return fermion_matrix_op(t_ops, n) - fermion_matrix_op(td_ops, n)


@pytest.mark.parametrize("exc", [(0, 2, -1, -1), (1, 5, -1, -1), (0, 1, 2, 3), (0, 3, 4, 5),
                                 (1, 2, 3, 4), (0, 2, 4, 5), (4, 1, -1, -1), (3, 5, 0, 2), (2, 3, 0, 1)])
def test_gate_matches_expm(exc):
    """The pair rotation equals scipy.linalg.expm(theta (T - T^dagger)) on random states,
    including generalised excitations that move electrons to lower orbitals (k-UpCCGSD)."""
    n = 6
    rng = np.random.default_rng(9)
    A = _generator_dense(exc, n)
    assert np.abs(A + A.T).max() == 0  # anti-Hermitian, real
    psi = rng.normal(size=64) + 1j * rng.normal(size=64)
    for th in (0.37, -1.2):
        ref = sla.expm(th * A) @ psi
        assert np.abs(oracle.apply_gate(psi, exc, th) - ref).max() < 1e-13
    assert np.abs(oracle.apply_generator(psi, exc) - A @ psi).max() < 1e-14


def test_golden_p1_gate_actions():
    rows = []
    with open(os.path.join(GOLDEN, "p1_excitations_4q.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append(line.split())
    th = 0.3
    by_exc = {}
    for r in rows:
        exc = tuple(int(v) for v in r[:4])
        by_exc.setdefault(exc, []).append((int(r[4]), r[5], int(r[6])))
    for exc, amps in by_exc.items():
        psi = oracle.prepare_state(4, 0b0011, [exc], [th])
        expect = np.zeros(16)
        for k, fn, sgn in amps:
            expect[k] = sgn * (np.cos(th) if fn == "cos" else np.sin(th))
        assert np.abs(psi - expect).max() < 1e-15, exc


def test_double_only_two_level_closed_form():
    """With the double excitation alone, E = cos^2 H_aa + sin^2 H_bb + sin 2t H_ab."""
    w = synth.config0()
    prob = w.problems[0]
    model = oracle.EnergyModel.from_problem(prob)
    H = model.matrix.toarray()
    haa, hbb, hab = H[3, 3], H[12, 12], H[3, 12]
    for th in np.linspace(-1.5, 1.5, 7):
        e = oracle.energy(model, 3, [(0, 1, 2, 3)], [th])
        ref = np.cos(th) ** 2 * haa + np.sin(th) ** 2 * hbb + np.sin(2 * th) * hab
        assert abs(e - ref) < 1e-13


def test_generators_conserve_number_and_sz():
    n = 6
    Nop = sum(fermion_matrix_op([(p, True), (p, False)], n) for p in range(n))
    Sz = sum((1 if p % 2 == 0 else -1) * fermion_matrix_op([(p, True), (p, False)], n)
             for p in range(n))
    for exc in synth.uccsd_pool(n, 3):
        A = _generator_dense(exc, n)
        assert not np.any(A @ Nop - Nop @ A)
        assert not np.any(A @ Sz - Sz @ A)


def test_norm_sector_support_and_reversal():
    """Norm stays 1 after hundreds of gates; amplitudes outside the reference's
    (N, S_z) sector stay exactly 0.0; undoing the gates returns |HF>."""
    rng = np.random.default_rng(10)
    n, n_elec = 10, 5
    pool = synth.uccsd_pool(n, n_elec)
    excs = pool[rng.integers(0, len(pool), size=512)]
    ths = rng.normal(0, 0.5, size=512)
    hf = synth.hf_bitstring(n_elec)
    psi = oracle.prepare_state(n, hf, excs, ths)
    assert abs(np.linalg.norm(psi) - 1.0) < 1e-12
    na, nb = synth.spin_counts(n_elec)
    inside = np.zeros(1 << n, dtype=bool)
    inside[oracle.sector_basis(n, na, nb).astype(np.int64)] = True
    assert np.all(psi[~inside] == 0.0)
    back = psi
    for exc, th in zip(excs[::-1], ths[::-1]):
        back = oracle.apply_gate(back, exc, -th)
    assert np.abs(back - oracle.hf_state(n, hf)).max() < 1e-12


def test_sector_basis_and_pool_counts():
    from math import comb
    for n, N in [(4, 2), (12, 6), (14, 7), (16, 8), (18, 9), (20, 10)]:
        na, nb = synth.spin_counts(N)
        assert len(oracle.sector_basis(n, na, nb)) == comb(n // 2, na) * comb(n // 2, nb)
    assert len(synth.uccsd_pool(4, 2)) == 3
    assert len(synth.uccsd_pool(12, 6)) == 117
    assert len(synth.uccsd_pool(16, 8)) == 360
    assert len(synth.uccsd_pool(30, 10)) == 3500
    assert len(synth.uccsd_pool(14, 7)) == 204


# ---------------------------------------------------------------- energy and gradient
def test_variational_bound():
    """E(theta) >= E0 for every theta (Sec. 2.1.1's variational principle)."""
    prob = _rand_problem(21, 4, 4)
    model = oracle.EnergyModel.from_problem(prob)
    e0 = oracle.exact_ground_energy(prob)
    exc = synth.uccsd_pool(8, 4)
    rng = np.random.default_rng(22)
    for _ in range(10):
        e = oracle.energy(model, 15, exc, rng.normal(0, 1.0, size=len(exc)))
        assert e >= e0 - 1e-12


def test_gradients_three_ways():
    """Direct gradient = four-point shift rule (exact) = central differences (approx.)."""
    prob = _rand_problem(31, 4, 4)
    exc = synth.uccsd_pool(8, 4)
    rng = np.random.default_rng(32)
    th = rng.normal(0, 0.3, size=len(exc))
    model = oracle.EnergyModel.from_problem(prob)
    e, g = oracle.gradient_direct(model, 15, exc, th)
    gs = oracle.gradient_shift(model, 15, exc, th)
    gf = oracle.gradient_fd(model, 15, exc, th)
    assert np.abs(g - gs).max() < 1e-12
    assert np.abs(g - gf).max() < 1e-7
    assert abs(e - oracle.energy(model, 15, exc, th)) < 1e-14


def test_route1_route2_energy_and_gradient_agree():
    prob = _rand_problem(41, 4, 4)
    xs, zs, cs = oracle.jordan_wigner(prob)
    exc = synth.uccsd_pool(8, 4)
    th = np.random.default_rng(42).normal(0, 0.2, size=len(exc))
    e1, g1 = oracle.gradient_direct(oracle.EnergyModel.from_problem(prob), 15, exc, th)
    e2, g2 = oracle.gradient_direct(oracle.EnergyModel.from_pauli(8, xs, zs, cs), 15, exc, th)
    assert abs(e1 - e2) < 1e-12 and np.abs(g1 - g2).max() < 1e-12


def test_sector_route_equals_full_route():
    prob = _rand_problem(43, 5, 4)
    exc = synth.uccsd_pool(10, 4)
    th = np.random.default_rng(44).normal(0, 0.2, size=len(exc))
    mf = oracle.EnergyModel.from_problem(prob, full=True)
    ms = oracle.EnergyModel.from_problem(prob, full=False)
    assert abs(oracle.energy(mf, 15, exc, th) - oracle.energy(ms, 15, exc, th)) < 1e-12


def test_config0_bfgs_reaches_exact_energy():
    """The 3-parameter UCCSD spans config 0's 4-dimensional real sector, so BFGS
    from the HF start reaches the full-CI energy to 1e-8 Ha."""
    w = synth.config0()
    prob = w.problems[0]
    model = oracle.EnergyModel.from_problem(prob)
    e0 = oracle.exact_ground_energy(prob)
    best = None
    for start in (np.zeros(3), w.thetas[0], np.array([0.5, -0.5, 1.0])):
        res, _ = oracle.run_bfgs(model, 3, w.excitations[0], start)
        best = res.fun if best is None else min(best, res.fun)
    assert abs(best - e0) < 1e-8
