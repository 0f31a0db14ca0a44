"""The other chemistry ansatze of Sec. 2.1.2 through the C ABI against the oracle.

k-UpCCGSD (generalised singles and pair doubles, repeated k times) and pUCCD
in its fermionic form run on the UCCSD kernels; pUCCD's hard-core boson form
runs on n_s qubits (vqe_hcb_hamiltonian, vqe_create_ansatz_hcb) in the
pair-number sector. Bar as for UCCSD: |dE| <= 1e-10 Ha, |dg| <= 1e-9.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
import paper_2311_01242_gb300 as vq

pytestmark = pytest.mark.gpu

E_TOL = 1e-10
G_TOL = 1e-9
PATHS = [0, vq.VQE_FLAG_FORCE_STREAMING, vq.VQE_FLAG_FORCE_COMPLEX, vq.VQE_FLAG_NO_CLUSTER]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    vq.build()
    vq.load()
    yield
    vq.set_flags(0)


def _eg(H, A, th, flags=0):
    old = vq.set_flags(flags)
    try:
        e, g = vq.energy_grad(H, A, th)
        torch.cuda.synchronize()
        return float(e), g.cpu().numpy()
    finally:
        vq.set_flags(old)


@pytest.mark.parametrize("seed,n_s,n_elec,k", [(401, 4, 4, 2), (402, 4, 3, 1), (403, 6, 6, 1)])
def test_k_upccgsd_matches_oracle(seed, n_s, n_elec, k):
    p = synth.random_problem(np.random.default_rng(seed), n_s, n_elec, 3)
    exc = synth.upccgsd_pool(2 * n_s, k)
    th = np.random.default_rng(seed + 1).normal(0, 0.2, size=len(exc))
    hf = synth.hf_bitstring(n_elec)
    e_o, g_o = oracle.gradient_direct(oracle.EnergyModel.from_problem(p), hf, exc, th)
    H = vq.Hamiltonian.from_problem(p)
    A = vq.Ansatz(2 * n_s, hf, exc)
    for flags in PATHS:
        e, g = _eg(H, A, th, flags)
        assert abs(e - e_o) <= E_TOL, flags
        assert np.abs(g - g_o).max() <= G_TOL, flags


def test_puccd_fermionic_matches_oracle():
    p = synth.random_problem(np.random.default_rng(404), 6, 6, 3)
    exc = synth.puccd_pool(12, 6)
    th = np.random.default_rng(405).normal(0, 0.3, size=len(exc))
    e_o, g_o = oracle.gradient_direct(oracle.EnergyModel.from_problem(p), 63, exc, th)
    H = vq.Hamiltonian.from_problem(p)
    A = vq.Ansatz(12, 63, exc)
    for flags in PATHS:
        e, g = _eg(H, A, th, flags)
        assert abs(e - e_o) <= E_TOL and np.abs(g - g_o).max() <= G_TOL, flags


@pytest.mark.parametrize("geom", [0, 37])
def test_hcb_puccd_ch3f_size_matches_oracle(geom):
    """11 orbitals, 4 pairs (330 boson states), 28 angles: the boson form on
    11 qubits against the oracle's seniority-zero block."""
    w = synth.puccd_scan()
    p, th = w.problems[geom], w.thetas[geom] * 8.0
    pairs = synth.hcb_pairs_of(w.excitations[geom])
    e_o, g_o = oracle.hcb_energy_grad(oracle.HcbModel(p, 4), 15, pairs, th)
    H = vq.Hamiltonian.from_problem_hcb(p)
    A = vq.Ansatz(11, 15, pairs, hcb=True)
    assert A.info()["sector_dim"] == 330
    for flags in PATHS:
        e, g = _eg(H, A, th, flags)
        assert abs(e - e_o) <= E_TOL, flags
        assert np.abs(g - g_o).max() <= G_TOL, flags


def test_hcb_equals_fermionic_puccd_on_gpu():
    """8 orbitals, 4 pairs: the boson form on 8 qubits (70 states) and the
    fermionic form on 16 qubits (4,900 states) give the same E and gradient,
    and both match the oracle."""
    p = synth.random_problem(np.random.default_rng(406), 8, 8, 4)
    exc = synth.puccd_pool(16, 8)
    th = np.random.default_rng(407).normal(0, 0.3, size=len(exc))
    e_f, g_f = _eg(vq.Hamiltonian.from_problem(p), vq.Ansatz(16, 255, exc), th)
    e_b, g_b = _eg(vq.Hamiltonian.from_problem_hcb(p), vq.Ansatz(8, 15, synth.hcb_pairs_of(exc), hcb=True), th)
    e_o, g_o = oracle.hcb_energy_grad(oracle.HcbModel(p, 4), 15, synth.hcb_pairs_of(exc), th)
    assert abs(e_f - e_b) <= E_TOL and np.abs(g_f - g_b).max() <= G_TOL
    assert abs(e_b - e_o) <= E_TOL and np.abs(g_b - g_o).max() <= G_TOL


def test_hcb_scan_batch_matches_single_calls_and_oracle():
    """The 64-geometry pUCCD scan in one batched launch."""
    w = synth.puccd_scan()
    pairs = synth.hcb_pairs_of(w.excitations[0])
    hams = [vq.Hamiltonian.from_problem_hcb(p) for p in w.problems]
    A = vq.Ansatz(11, 15, pairs, hcb=True)
    B = vq.Batch(hams, [A] * 64)
    theta = torch.as_tensor(np.stack(w.thetas)).cuda().contiguous()
    e, g = B.energy_grad(theta)
    e, g = e.cpu().numpy(), g.cpu().numpy()
    for i in (0, 21, 63):
        e1, g1 = _eg(hams[i], A, w.thetas[i])
        assert abs(e[i] - e1) <= E_TOL and np.abs(g[i, :28] - g1).max() <= G_TOL
    for i in (5, 50):
        e_o, g_o = oracle.hcb_energy_grad(oracle.HcbModel(w.problems[i], 4), 15, pairs, w.thetas[i])
        assert abs(e[i] - e_o) <= E_TOL and np.abs(g[i, :28] - g_o).max() <= G_TOL


def test_hcb_24_orbitals_full_size():
    """24 orbitals, 12 pairs (2,704,156 boson states), 144 angles: the energy at
    theta = 0 is the Slater-Condon energy of the closed-shell reference, and
    sampled gradient components equal the four-point shift rule of the
    library's own energies (exact: the pair generators have spectrum {0, +-i})."""
    w = synth.puccd_large()
    p, th = w.problems[0], w.thetas[0]
    pairs = synth.hcb_pairs_of(w.excitations[0])
    H = vq.Hamiltonian.from_problem_hcb(p)
    A = vq.Ansatz(24, (1 << 12) - 1, pairs, hcb=True)
    assert A.info()["sector_dim"] == 2704156
    ws = vq.alloc_workspace(vq.workspace_bytes(H, A, vq.VQE_WS_GRAD))
    occ = range(12)
    e_sc = sum(2 * p.h[i, i] + p.eri[i, i, i, i] for i in occ)
    e_sc += sum(2 * p.eri[i, i, j, j] - p.eri[i, j, j, i] for i in occ for j in occ if i != j)
    assert abs(float(vq.energy(H, A, np.zeros(len(th)), workspace=ws)) - e_sc) <= 1e-10
    e, g = vq.energy_grad(H, A, th, workspace=ws)
    g = g.cpu().numpy()
    w_ = (np.sqrt(2.0) - 1.0) / 2.0
    for k in (0, 71, 143):
        def e_at(shift):
            t = th.copy()
            t[k] += shift
            return float(vq.energy(H, A, t, workspace=ws))
        gs = (e_at(np.pi / 4) - e_at(-np.pi / 4)) - w_ * (e_at(np.pi / 2) - e_at(-np.pi / 2))
        assert abs(gs - g[k]) <= 1e-9, (k, gs, g[k])


def test_hcb_pool_screening_matches_oracle():
    """ADAPT screening in the boson form: every pair excitation of the 11-orbital
    pool against 2 Re <H psi| (b+_a b_i - b+_i b_a) |psi> from the oracle."""
    w = synth.puccd_scan(1)
    p = w.problems[0]
    pool = synth.hcb_pair_pool(11, 4)
    cur = pool[[3, 17, 25]]
    th = np.array([0.3, -0.2, 0.15])
    model = oracle.HcbModel(p, 4)
    psi = oracle.hcb_state(11, 15, cur, th)
    hpsi = model.apply(psi)
    g_o = np.array([2.0 * np.vdot(hpsi, oracle.hcb_generator(psi, int(i), int(a))).real for i, a in pool])
    H = vq.Hamiltonian.from_problem_hcb(p)
    A = vq.Ansatz(11, 15, cur, hcb=True)
    P = vq.Ansatz(11, 15, pool, hcb=True)
    for flags in (0, vq.VQE_FLAG_FORCE_COMPLEX):
        old = vq.set_flags(flags)
        try:
            e, g = vq.pool_gradients(H, A, P, th)
        finally:
            vq.set_flags(old)
        assert abs(float(e) - np.vdot(psi, hpsi).real) <= E_TOL
        assert np.abs(g.cpu().numpy() - g_o).max() <= G_TOL


def test_downward_generalised_excitations_match_oracle():
    """Generalised excitations that move electrons to lower orbitals, and
    repeats, in one ansatz (the gates after the first layer start from states
    where those orbitals are occupied)."""
    p = synth.random_problem(np.random.default_rng(408), 4, 4, 3)
    exc = np.array([(0, 4, -1, -1), (1, 7, -1, -1), (0, 1, 4, 5), (4, 0, -1, -1), (7, 3, -1, -1),
                    (4, 5, 2, 3), (2, 6, 0, 1), (0, 4, -1, -1)], dtype=np.int32)
    th = np.random.default_rng(409).normal(0, 0.5, size=len(exc))
    e_o, g_o = oracle.gradient_direct(oracle.EnergyModel.from_problem(p), 15, exc, th)
    H = vq.Hamiltonian.from_problem(p)
    A = vq.Ansatz(8, 15, exc)
    for flags in PATHS:
        e, g = _eg(H, A, th, flags)
        assert abs(e - e_o) <= E_TOL and np.abs(g - g_o).max() <= G_TOL, flags
