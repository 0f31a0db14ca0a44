"""Parity at the workloads' full sizes, on sampled outputs and exact identities.

30 qubits (9.0M sector amplitudes, 512 angles): the energy at theta = 0 is the
Hartree-Fock energy, whose closed form comes from the integrals; at a random
theta, sampled gradient components equal the four-point shift rule evaluated
with the library's own energies (exact for rotations generated by T - T^dagger,
whose spectrum is {0, +-i}), and the gradient from the kept forward outputs
equals the one from un-applying the gates to rounding; one H psi pass on a random sector vector equals
the oracle's explicit Pauli action at sampled rows; psi(theta) after 512 gates
has unit norm and no weight outside the sector. 256 uneven instances (14-20 qubits): the batched
launch agrees with single-instance calls on sampled instances, and with the
oracle on the smallest ones. The real-amplitude string-driven H psi of the
energy and gradient calls, in each of its three forms (warp form at 20 qubits,
staged block form at 24, wide block form at 30), equals the oracle's explicit
Pauli action at sampled rows.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
import paper_2311_01242_gb300 as vq

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    vq.load()


def _slater_condon(p):
    occ = range(p.n_elec)
    e = sum(p.h[P // 2, P // 2] for P in occ)
    for P in occ:
        for Q in occ:
            e += 0.5 * p.eri[P // 2, P // 2, Q // 2, Q // 2]
            if P % 2 == Q % 2:
                e -= 0.5 * p.eri[P // 2, Q // 2, Q // 2, P // 2]
    return e


def test_30_qubits_hf_energy_and_shift_rule_gradient():
    w = synth.config3()
    p, exc, th = w.problems[0], w.excitations[0], w.thetas[0]
    H = vq.Hamiltonian.from_problem(p, w.drop_tol)
    A = vq.Ansatz(30, synth.hf_bitstring(10), exc)
    ws = vq.alloc_workspace(vq.workspace_bytes(H, A, vq.VQE_WS_GRAD))
    e0 = float(vq.energy(H, A, np.zeros(len(exc)), workspace=ws))
    # the Pauli terms dropped below 1e-8 bound the difference (none for these integrals)
    _, _, c_all = vq.jordan_wigner(p.n_spatial, p.h, p.eri, 0.0, 0.0)
    dropped = float(np.abs(c_all[np.abs(c_all) < w.drop_tol]).sum())
    assert abs(e0 - _slater_condon(p)) <= 1e-10 + dropped
    e, g = vq.energy_grad(H, A, th, workspace=ws)
    g = g.cpu().numpy()
    # the reverse sweep un-applying each gate to psi instead of reading the kept
    # forward outputs: the same energy bits, the gradient to rounding
    old = vq.set_flags(vq.VQE_FLAG_NO_PHI_STORE)
    try:
        e1, g1 = vq.energy_grad(H, A, th, workspace=ws)
    finally:
        vq.set_flags(old)
    g1 = g1.cpu().numpy()
    assert float(e1) == float(e)
    assert np.abs(g1 - g).max() <= 1e-11
    # persistent sweeps instead of one launch per gate: the same bits as the un-applying path
    old = vq.set_flags(vq.VQE_FLAG_PERSISTENT_SWEEPS)
    try:
        e2, g2 = vq.energy_grad(H, A, th, workspace=ws)
    finally:
        vq.set_flags(old)
    assert float(e2) == float(e) and np.array_equal(g2.cpu().numpy(), g1)
    w_ = (np.sqrt(2.0) - 1.0) / 2.0
    for k in (0, 255, 511):
        def e_at(shift):
            t = th.copy()
            t[k] += shift
            return float(vq.energy(H, A, t, workspace=ws))
        gs = (e_at(np.pi / 4) - e_at(-np.pi / 4)) - w_ * (e_at(np.pi / 2) - e_at(-np.pi / 2))
        assert abs(gs - g[k]) <= 1e-9, (k, gs, g[k])


def test_config2_full_batch_matches_single_calls_and_oracle():
    insts = [synth.config2_instance(j) for j in range(256)]
    hams = [vq.Hamiltonian.from_problem(p) for p, _, _ in insts]
    ans = [vq.Ansatz(p.n_qubits, synth.hf_bitstring(p.n_elec), e) for p, e, _ in insts]
    B = vq.Batch(hams, ans)
    theta = torch.zeros(256, B.max_params, dtype=torch.float64)
    for i, (_, _, t) in enumerate(insts):
        theta[i, :len(t)] = torch.as_tensor(t)
    e, g = B.energy_grad(theta.cuda())
    e, g = e.cpu().numpy(), g.cpu().numpy()
    rng = np.random.default_rng(0)
    for i in rng.choice(256, size=6, replace=False):
        m = len(insts[i][2])
        e1, g1 = vq.energy_grad(hams[i], ans[i], theta[i, :m])
        assert float(e1) == e[i]                     # the persistent launch: the same bits
        assert np.array_equal(g1.cpu().numpy(), g[i, :m])
    small = [i for i, (p, _, _) in enumerate(insts) if p.n_qubits == 14][:2]
    for i in small:
        p, exc, t = insts[i]
        idx = [0, len(exc) - 1]
        e_o, g_o = oracle.gradient_direct(oracle.EnergyModel.from_problem(p, full=False),
                                          synth.hf_bitstring(p.n_elec), exc, t, idx)
        assert abs(e[i] - e_o) <= 1e-10
        assert np.abs(g[i, idx] - g_o).max() <= 1e-9


def _lookup(sec, vals):
    def amp(idx):
        pos = np.minimum(np.searchsorted(sec, idx), len(sec) - 1)
        return np.where(sec[pos] == idx, vals[pos], 0.0)
    return amp


def test_30_qubits_hpsi_rows_norm_and_sector_support():
    w = synth.config3()
    p, exc, th = w.problems[0], w.excitations[0], w.thetas[0]
    xs, zs, cs = oracle.jordan_wigner(p, w.drop_tol)      # the oracle's own Pauli list
    H = vq.Hamiltonian(30, xs, zs, cs)
    A = vq.Ansatz(30, synth.hf_bitstring(10), exc)
    sec = oracle.sector_basis(30, 5, 5)
    assert len(sec) == 9018009
    sec_t = torch.as_tensor(sec.astype(np.int64)).cuda()
    rng = np.random.default_rng(30)
    vals = rng.normal(size=len(sec)) + 1j * rng.normal(size=len(sec))
    vals /= np.linalg.norm(vals)
    psi = torch.zeros(1 << 30, dtype=torch.complex128, device="cuda")
    psi[sec_t] = torch.as_tensor(vals).cuda()
    lam, e = vq.apply_hamiltonian(H, A, psi)
    amp = _lookup(sec, vals)
    rows = np.concatenate([[0, len(sec) - 1, int(np.searchsorted(sec, synth.hf_bitstring(10)))],
                           rng.choice(len(sec), 45, replace=False)])
    for r in rows:
        k = int(sec[r])
        want = oracle.pauli_sum_row(xs, zs, cs, k, amp)
        got = complex(lam[k].item())
        assert abs(got - want) <= 1e-12, (k, got, want)
    # the energy reduction agrees with its own lambda output
    assert abs(float(e) - float(torch.vdot(psi, lam).real)) <= 1e-12
    del psi, lam
    # psi(theta) after all 512 gates: unit norm, support inside the sector
    st = vq.state(A, H, th)
    assert abs(float(torch.linalg.vector_norm(st)) - 1.0) <= 1e-12
    assert int(torch.count_nonzero(st)) <= len(sec)
    assert abs(float(torch.linalg.vector_norm(st[sec_t])) - 1.0) <= 1e-12
    # the real-amplitude energy equals the complex H psi pass on that state
    e_real = float(vq.energy(H, A, th))
    _, e_cplx = vq.apply_hamiltonian(H, A, st)
    assert abs(e_real - float(e_cplx)) <= 1e-10


def _real_rows(p, n, n_elec, drop, seed, n_rows=45):
    """lambda = H psi through the real-amplitude kernels (vqe_apply_hamiltonian_sector)
    on a random real sector vector, against oracle.pauli_sum_row on the oracle's
    own Pauli list at sampled rows (first, last, HF and random ones)."""
    xs, zs, cs = oracle.jordan_wigner(p, drop)
    H = vq.Hamiltonian(n, xs, zs, cs)
    A = vq.Ansatz(n, synth.hf_bitstring(n_elec), [[0, 2, -1, -1]])
    na, nb = (n_elec + 1) // 2, n_elec // 2
    sec = oracle.sector_basis(n, na, nb)
    rng = np.random.default_rng(seed)
    vals = rng.normal(size=len(sec))
    vals /= np.linalg.norm(vals)
    psi = torch.as_tensor(vals).cuda()
    lam, e = vq.apply_hamiltonian_sector(H, A, psi)
    lam = lam.cpu().numpy()
    amp = _lookup(sec, vals)
    rows = np.concatenate([[0, len(sec) - 1, int(np.searchsorted(sec, synth.hf_bitstring(n_elec)))],
                           rng.choice(len(sec), n_rows, replace=False)])
    for r in rows:
        want = oracle.pauli_sum_row(xs, zs, cs, int(sec[r]), amp)
        assert abs(want.imag) <= 1e-12  # a real Hamiltonian: real rows for a real state
        assert abs(lam[r] - want.real) <= 1e-12, (n, r, lam[r], want)
    assert abs(float(e) - float(np.dot(vals, lam))) <= 1e-12


def test_real_string_hpsi_rows_warp_form_20_qubits():
    ns, _ = synth.configs.config2_sizes()
    p, _, _ = synth.config2_instance(int(np.nonzero(ns == 20)[0][0]))
    _real_rows(p, 20, 10, 1e-14, 20)


def test_real_string_hpsi_rows_staged_block_form_24_qubits():
    p = synth.integrals.random_problem(np.random.default_rng(24), 12, 10, 6, label="q24")
    _real_rows(p, 24, 10, 1e-14, 24)


def test_real_string_hpsi_rows_wide_block_form_30_qubits():
    w = synth.config3()
    _real_rows(w.problems[0], 30, 10, w.drop_tol, 31)
