"""Parity of the CUDA path (through the C ABI) against the CPU oracle.

Bar: |dE| <= 1e-10 Ha and |dg_k| <= 1e-9 for every compared component, on the
same seeded inputs. The oracle evaluates Eq. 2 from the integrals by literal
ladder operators (not the library's Jordan-Wigner list) unless a test feeds a
random Pauli sum, where it applies the Pauli strings explicitly.
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


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    vq.build()
    vq.load()
    yield
    vq.set_flags(0)


def gpu_eg(problem, exc, theta, drop_tol=1e-14, flags=0):
    old = vq.set_flags(flags)
    try:
        H = vq.Hamiltonian.from_problem(problem, drop_tol)
        A = vq.Ansatz(problem.n_qubits, synth.hf_bitstring(problem.n_elec), exc)
        e, g = vq.energy_grad(H, A, torch.as_tensor(theta, dtype=torch.float64).cuda())
        torch.cuda.synchronize()
        return float(e), g.cpu().numpy()
    finally:
        vq.set_flags(old)


def oracle_eg(problem, exc, theta, indices=None, full=None):
    model = oracle.EnergyModel.from_problem(problem, full=full)
    return oracle.gradient_direct(model, synth.hf_bitstring(problem.n_elec), exc, theta, indices)


# ------------------------------------------------------------------ small chemistry
def test_config0_energy_gradient():
    w = synth.config0()
    p, exc, th = w.problems[0], w.excitations[0], w.thetas[0]
    e_o, g_o = oracle_eg(p, exc, th)
    for flags in (0, vq.VQE_FLAG_FORCE_STREAMING, vq.VQE_FLAG_FORCE_COMPLEX,
                  vq.VQE_FLAG_FORCE_COMPLEX | vq.VQE_FLAG_FORCE_STREAMING):
        e, g = gpu_eg(p, exc, th, flags=flags)
        assert abs(e - e_o) <= E_TOL, flags
        assert np.abs(g - g_o).max() <= G_TOL, flags


def test_config0_bfgs_on_gpu_reaches_exact_energy():
    import scipy.optimize as so
    w = synth.config0()
    p, exc = w.problems[0], w.excitations[0]
    H = vq.Hamiltonian.from_problem(p)
    A = vq.Ansatz(4, 3, exc)
    ws = vq.alloc_workspace(vq.workspace_bytes(H, A))

    def fun(t):
        e, g = vq.energy_grad(H, A, torch.as_tensor(t).cuda(), workspace=ws)
        return float(e), g.cpu().numpy()

    e0 = oracle.exact_ground_energy(p)
    best = min(so.minimize(fun, x0, jac=True, method="BFGS", options={"gtol": 1e-10}).fun
               for x0 in (np.zeros(3), w.thetas[0], np.array([0.5, -0.5, 1.0])))
    assert abs(best - e0) < 1e-8


@pytest.mark.parametrize("seed,n_s,n_elec", [(101, 3, 2), (102, 4, 3), (103, 4, 4), (104, 5, 4),
                                             (105, 6, 6)])
def test_random_problems_resident_and_streaming(seed, n_s, n_elec):
    rng = np.random.default_rng(seed)
    p = synth.random_problem(rng, n_s, n_elec, 3)
    exc = synth.uccsd_pool(2 * n_s, n_elec)
    exc = exc[rng.permutation(len(exc))]
    th = rng.normal(0, 0.3, size=len(exc))
    e_o, g_o = oracle_eg(p, exc, th)
    for flags in (0, vq.VQE_FLAG_FORCE_STREAMING):
        e, g = gpu_eg(p, exc, th, flags=flags)
        assert abs(e - e_o) <= E_TOL
        assert np.abs(g - g_o).max() <= G_TOL


def test_real_and_complex_paths_agree_bitwise_on_energy():
    rng = np.random.default_rng(7)
    p = synth.random_problem(rng, 5, 5, 4)
    exc = synth.uccsd_pool(10, 5)
    th = rng.normal(0, 0.2, size=len(exc))
    for stream_flag in (0, vq.VQE_FLAG_FORCE_STREAMING):
        e_r, g_r = gpu_eg(p, exc, th, flags=stream_flag)
        e_c, g_c = gpu_eg(p, exc, th, flags=stream_flag | vq.VQE_FLAG_FORCE_COMPLEX)
        assert abs(e_r - e_c) <= 1e-13
        assert np.abs(g_r - g_c).max() <= 1e-13


# ------------------------------------------------------------------ the 12-qubit scan, batched
def test_config1_batch_energies_and_sampled_gradients():
    w = synth.config1()
    exc = w.excitations[0]
    hams = [vq.Hamiltonian.from_problem(p) for p in w.problems]
    A = vq.Ansatz(12, synth.hf_bitstring(6), exc)
    B = vq.Batch(hams, [A] * len(hams))
    theta = torch.as_tensor(np.stack(w.thetas)).cuda().contiguous()
    e, g = B.energy_grad(theta)
    torch.cuda.synchronize()
    e, g = e.cpu().numpy(), g.cpu().numpy()
    hf = synth.hf_bitstring(6)
    for i in range(0, 64, 9):
        model = oracle.EnergyModel.from_problem(w.problems[i])
        if i in (0, 63):
            e_o, g_o = oracle.gradient_direct(model, hf, exc, w.thetas[i])
            assert np.abs(g[i] - g_o).max() <= G_TOL
        else:
            e_o = oracle.energy(model, hf, exc, w.thetas[i])
        assert abs(e[i] - e_o) <= E_TOL, i
    # batched result equals the single-instance result
    for i in (0, 31, 63):
        e1, g1 = vq.energy_grad(hams[i], A, theta[i])
        assert abs(float(e1) - e[i]) <= 1e-14
        assert np.abs(g1.cpu().numpy() - g[i]).max() <= 1e-14


def test_batch_host_entry_matches_device_entry():
    w = synth.config1(8)
    hams = [vq.Hamiltonian.from_problem(p) for p in w.problems]
    A = vq.Ansatz(12, synth.hf_bitstring(6), w.excitations[0])
    B = vq.Batch(hams, [A] * len(hams))
    th = np.ascontiguousarray(np.stack(w.thetas))
    e_d, g_d = B.energy_grad(torch.as_tensor(th).cuda())
    ws = vq.alloc_workspace(B.host_workspace_bytes(True))
    e_h = np.zeros(8)
    g_h = np.zeros((8, B.max_params))
    B.energy_grad_host(th, e_h, g_h, ws)
    assert np.array_equal(e_h, e_d.cpu().numpy())
    assert np.array_equal(g_h, g_d.cpu().numpy()[:, :B.max_params])


# ------------------------------------------------------------------ uneven batch sizes
def test_config2_instances_mixed_sizes():
    picks = {}
    ns, _ = synth.configs.config2_sizes()
    for j in range(256):
        n = int(ns[j])
        if n not in picks:
            picks[n] = j
    assert set(picks) == {14, 16, 18, 20}
    insts = [synth.config2_instance(picks[n]) for n in (14, 16)]
    hams, ans, ths = [], [], []
    for p, exc, th in insts:
        hams.append(vq.Hamiltonian.from_problem(p))
        ans.append(vq.Ansatz(p.n_qubits, synth.hf_bitstring(p.n_elec), exc))
        ths.append(th)
    B = vq.Batch(hams, ans)
    ld = B.max_params
    theta = np.zeros((len(insts), ld))
    for i, th in enumerate(ths):
        theta[i, :len(th)] = th
    e, g = B.energy_grad(torch.as_tensor(theta).cuda())
    e, g = e.cpu().numpy(), g.cpu().numpy()
    rng = np.random.default_rng(0)
    for i, (p, exc, th) in enumerate(insts):
        idx = sorted(rng.choice(len(exc), size=6, replace=False).tolist())
        e_o, g_o = oracle_eg(p, exc, th, indices=idx, full=False)
        assert abs(e[i] - e_o) <= E_TOL
        assert np.abs(g[i][idx] - g_o).max() <= G_TOL


@pytest.mark.parametrize("n", [18, 20])
def test_config2_large_instances_energy_and_sampled_gradient(n):
    ns, _ = synth.configs.config2_sizes()
    j = int(np.nonzero(ns == n)[0][0])
    p, exc, th = synth.config2_instance(j)
    e, g = gpu_eg(p, exc, th)
    M = len(exc)
    idx = [M - 40, M - 2, M - 1] if n == 18 else [M - 2, M - 1]
    e_o, g_o = oracle_eg(p, exc, th, indices=idx, full=False)
    assert abs(e - e_o) <= E_TOL
    assert np.abs(g[idx] - g_o).max() <= G_TOL


# ------------------------------------------------------------------ row-level checks
@pytest.mark.parametrize("n_s,n_elec", [(2, 2), (4, 3), (6, 6), (7, 7)])
def test_state_matches_oracle_and_sector(n_s, n_elec):
    rng = np.random.default_rng(n_s * 10 + n_elec)
    n = 2 * n_s
    exc = synth.uccsd_pool(n, n_elec)
    exc = exc[rng.integers(0, len(exc), size=min(300, 3 * len(exc)))]
    th = rng.normal(0, 0.5, size=len(exc))
    hf = synth.hf_bitstring(n_elec)
    p = synth.random_problem(rng, n_s, n_elec, 2)
    H = vq.Hamiltonian.from_problem(p)
    A = vq.Ansatz(n, hf, exc)
    psi = vq.state(A, H, th).cpu().numpy()
    ref = oracle.prepare_state(n, hf, exc, th)
    assert np.abs(psi - ref).max() <= 1e-12
    assert abs(np.linalg.norm(psi) - 1.0) <= 1e-12
    na, nb = synth.spin_counts(n_elec)
    inside = np.zeros(1 << n, dtype=bool)
    inside[oracle.sector_basis(n, na, nb).astype(np.int64)] = True
    assert np.all(psi[~inside] == 0.0)


def _sector_state(rng, n, n_elec, complex_amp=True):
    na, nb = synth.spin_counts(n_elec)
    basis = oracle.sector_basis(n, na, nb).astype(np.int64)
    psi = np.zeros(1 << n, dtype=complex)
    v = rng.normal(size=len(basis)) + (1j * rng.normal(size=len(basis)) if complex_amp else 0)
    psi[basis] = v / np.linalg.norm(v)
    return psi, basis


@pytest.mark.parametrize("n,T,maxw", [(8, 60, None), (10, 200, 4), (12, 400, 6)])
def test_apply_hamiltonian_random_pauli_sum(n, T, maxw):
    """lambda = H psi on the sector for arbitrary Pauli sums (Y phases, wide X masks)."""
    rng = np.random.default_rng(n + T)
    xs, zs, cs = synth.random_pauli_terms(rng, n, T, max_weight=maxw)
    n_elec = n // 2
    psi, basis = _sector_state(rng, n, n_elec)
    exc = synth.uccsd_pool(n, n_elec)[:3]
    H = vq.Hamiltonian(n, xs, zs, cs)
    A = vq.Ansatz(n, synth.hf_bitstring(n_elec), exc)
    lam, e = vq.apply_hamiltonian(H, A, torch.as_tensor(psi).cuda())
    lam = lam.cpu().numpy()
    ref = oracle.pauli_sum_apply(xs, zs, cs, psi)
    assert np.abs(lam[basis] - ref[basis]).max() <= 1e-12
    outside = np.ones(1 << n, dtype=bool)
    outside[basis] = False
    assert np.all(lam[outside] == 0)
    assert abs(float(e) - np.vdot(psi, ref).real) <= E_TOL


@pytest.mark.parametrize("n,T", [(8, 80), (10, 150)])
def test_energy_gradient_random_pauli_sum(n, T):
    rng = np.random.default_rng(3 * n + T)
    xs, zs, cs = synth.random_pauli_terms(rng, n, T, max_weight=5)
    n_elec = n // 2
    exc = synth.uccsd_pool(n, n_elec)
    th = rng.normal(0, 0.4, size=len(exc))
    hf = synth.hf_bitstring(n_elec)
    model = oracle.EnergyModel.from_pauli(n, xs, zs, cs)
    e_o, g_o = oracle.gradient_direct(model, hf, exc, th)
    H = vq.Hamiltonian(n, xs, zs, cs)
    A = vq.Ansatz(n, hf, exc)
    for flags in (0, vq.VQE_FLAG_FORCE_STREAMING, vq.VQE_FLAG_FORCE_COMPLEX):
        old = vq.set_flags(flags)
        try:
            e, g = vq.energy_grad(H, A, th)
        finally:
            vq.set_flags(old)
        assert abs(float(e) - e_o) <= E_TOL
        assert np.abs(g.cpu().numpy() - g_o).max() <= G_TOL


# ------------------------------------------------------------------ edge cases
def test_no_excitations_gives_hf_energy():
    p = synth.random_problem(np.random.default_rng(5), 4, 4, 3)
    H = vq.Hamiltonian.from_problem(p)
    A = vq.Ansatz(8, 15, np.zeros((0, 4), dtype=np.int32))
    e = float(vq.energy(H, A, np.zeros(0)))
    e_o = oracle.energy(oracle.EnergyModel.from_problem(p), 15, [], [])
    assert abs(e - e_o) <= E_TOL


def test_identity_only_hamiltonian_and_dropped_terms():
    n = 6
    A = vq.Ansatz(n, 7, synth.uccsd_pool(n, 3))
    th = np.random.default_rng(1).normal(size=A.n_params)
    H = vq.Hamiltonian(n, [0], [0], [2.5])
    e, g = vq.energy_grad(H, A, th)
    assert abs(float(e) - 2.5) <= 1e-12 and np.abs(g.cpu().numpy()).max() <= 1e-12
    H0 = vq.Hamiltonian(n, [3, 3], [0, 0], [1e-20, -1e-20], drop_tol=1e-16)
    e0, g0 = vq.energy_grad(H0, A, th)
    assert float(e0) == 0.0 and np.all(g0.cpu().numpy() == 0.0)


PATHS = [0, vq.VQE_FLAG_FORCE_STREAMING, vq.VQE_FLAG_FORCE_STREAMING | vq.VQE_FLAG_NO_STRINGS,
         vq.VQE_FLAG_FORCE_COMPLEX]


@pytest.mark.parametrize("flags", PATHS, ids=["resident", "streaming-strings", "streaming-rows", "complex"])
def test_degenerate_inputs_on_every_path(flags):
    """No excitations, one-state sectors (no electrons, all orbitals filled),
    an identity-only and an all-dropped Hamiltonian, and a batch mixing them
    with a full pool, on each kernel path; against the oracle and exact values."""
    rng = np.random.default_rng(31)
    p = synth.random_problem(rng, 4, 4, 3)  # 8 qubits, 2 + 2 electrons
    model = oracle.EnergyModel.from_problem(p, full=True)
    exc = synth.uccsd_pool(8, 4)
    th = rng.normal(0.0, 0.3, size=len(exc))
    old = vq.set_flags(flags)
    try:
        H = vq.Hamiltonian.from_problem(p)
        A0 = vq.Ansatz(8, 15, np.zeros((0, 4), dtype=np.int32))
        e0, g0 = vq.energy_grad(H, A0, np.zeros(0))
        assert abs(float(e0) - oracle.energy(model, 15, [], [])) <= E_TOL and g0.numel() == 0
        for hf in (0, 255):  # sectors of a single state
            A1 = vq.Ansatz(8, hf, np.zeros((0, 4), dtype=np.int32))
            assert abs(float(vq.energy(H, A1, np.zeros(0))) - oracle.energy(model, hf, [], [])) <= E_TOL
        A = vq.Ansatz(8, 15, exc)
        Hi = vq.Hamiltonian(8, [0], [0], [2.5])
        e, g = vq.energy_grad(Hi, A, th)
        assert abs(float(e) - 2.5) <= 1e-12 and float(g.abs().max()) <= 1e-12
        Hz = vq.Hamiltonian(8, [3, 3], [0, 0], [1e-20, -1e-20], drop_tol=1e-16)
        e, g = vq.energy_grad(Hz, A, th)
        assert float(e) == 0.0 and float(g.abs().max()) == 0.0
        e, g = vq.energy_grad(H, A, th)
        idx = [0, len(exc) // 2, len(exc) - 1]
        e_o, g_o = oracle.gradient_direct(model, 15, exc, th, idx)
        assert abs(float(e) - e_o) <= E_TOL and np.abs(g.cpu().numpy()[idx] - g_o).max() <= G_TOL
        B = vq.Batch([H, H, Hi, Hz], [A0, A, A, A])
        theta = torch.zeros(4, B.max_params, dtype=torch.float64)
        for i in (1, 2, 3):
            theta[i] = torch.as_tensor(th)
        eb, gb = B.energy_grad(theta.cuda())
        assert abs(float(eb[0]) - float(e0)) <= 1e-12 and abs(float(eb[1]) - float(e)) <= 1e-12
        assert float((gb[1] - g).abs().max()) <= 1e-12
        assert abs(float(eb[2]) - 2.5) <= 1e-12 and float(eb[3]) == 0.0
    finally:
        vq.set_flags(old)


def test_non_spin_conserving_excitations_use_number_sector():
    rng = np.random.default_rng(9)
    p = synth.random_problem(rng, 3, 2, 2)
    exc = np.array([[0, 3, -1, -1], [1, 2, -1, -1], [0, 1, 4, 5], [0, 4, -1, -1]], dtype=np.int32)
    th = rng.normal(size=4)
    model = oracle.EnergyModel.from_problem(p, full=True)
    e_o, g_o = oracle.gradient_direct(model, 3, exc, th)
    for flags in (0, vq.VQE_FLAG_FORCE_STREAMING):
        e, g = gpu_eg(p, exc, th, flags=flags)
        assert abs(e - e_o) <= E_TOL and np.abs(g - g_o).max() <= G_TOL


def test_unsorted_double_indices_follow_operator_order():
    """{i, j, a, b} is T = a+_a a+_b a_j a_i as given, also when i > j or a > b."""
    rng = np.random.default_rng(12)
    p = synth.random_problem(rng, 3, 2, 2)
    exc = np.array([[1, 0, 2, 3], [0, 1, 5, 4], [1, 0, 3, 2]], dtype=np.int32)
    th = rng.normal(size=3)
    e_o, g_o = oracle.gradient_direct(oracle.EnergyModel.from_problem(p), 3, exc, th)
    e, g = gpu_eg(p, exc, th)
    assert abs(e - e_o) <= E_TOL and np.abs(g - g_o).max() <= G_TOL


def test_invalid_arguments_raise():
    with pytest.raises(vq.VQEError):
        vq.Hamiltonian(4, [1 << 4], [0], [1.0])
    with pytest.raises(vq.VQEError):
        vq.Ansatz(4, 3, [[0, 0, -1, -1]])
    H = vq.Hamiltonian(4, [0], [1], [1.0])
    A = vq.Ansatz(6, 3, [[0, 2, -1, -1]])
    with pytest.raises(vq.VQEError):
        vq.energy(H, A, np.zeros(1))
    A4 = vq.Ansatz(4, 3, [[0, 2, -1, -1]])
    with pytest.raises(vq.VQEError):
        vq.set_flags(vq.VQE_FLAG_FORCE_STREAMING)
        try:
            vq.api._check(vq.load().vqe_energy(H.handle, A4.handle, None, None, None, 0, None))
        finally:
            vq.set_flags(0)


def test_autograd_function():
    w = synth.config0()
    p, exc, th = w.problems[0], w.excitations[0], w.thetas[0]
    H = vq.Hamiltonian.from_problem(p)
    A = vq.Ansatz(4, 3, exc)
    t = torch.as_tensor(th).cuda().requires_grad_(True)
    e = vq.vqe_energy(t, H, A)
    (3.0 * e).backward()
    e_o, g_o = oracle_eg(p, exc, th)
    assert abs(float(e.detach()) - e_o) <= E_TOL
    assert np.abs(t.grad.cpu().numpy() - 3.0 * g_o).max() <= 3 * G_TOL


def test_cluster_of_two_matches_single_cta():
    """Splitting H psi over a cluster of two CTAs changes only the order in which
    the two energy halves are added; gradients are bitwise equal."""
    w = synth.config1(16)
    hams = [vq.Hamiltonian.from_problem(p) for p in w.problems]
    A = vq.Ansatz(12, synth.hf_bitstring(6), w.excitations[0])
    B = vq.Batch(hams, [A] * len(hams))
    theta = torch.as_tensor(np.stack(w.thetas)).cuda().contiguous()
    e2, g2 = [t.clone() for t in B.energy_grad(theta)]
    old = vq.set_flags(vq.VQE_FLAG_NO_CLUSTER)
    try:
        e1, g1 = [t.clone() for t in B.energy_grad(theta)]
        es1, gs1 = vq.energy_grad(hams[3], A, theta[3])
    finally:
        vq.set_flags(old)
    es2, gs2 = vq.energy_grad(hams[3], A, theta[3])
    assert float((e1 - e2).abs().max()) <= 1e-13
    assert torch.equal(g1, g2)
    assert abs(float(es1) - float(es2)) <= 1e-13 and torch.equal(gs1, gs2)


def test_fixed_point_sweeps_match_fp64_sweeps():
    """The resident kernel's integer (Q1.62) sweeps and its FP64 sweeps compute
    the same energies and gradients up to rounding: |dE| <= 1e-12, |dg| <= 1e-11,
    in both the single-CTA and the cluster form; both stay within the oracle bar."""
    w = synth.config1(8)
    hams = [vq.Hamiltonian.from_problem(p) for p in w.problems]
    A = vq.Ansatz(12, synth.hf_bitstring(6), w.excitations[0])
    B = vq.Batch(hams, [A] * len(hams))
    theta = torch.as_tensor(np.stack(w.thetas)).cuda().contiguous()
    for extra in (0, vq.VQE_FLAG_NO_CLUSTER):
        old = vq.set_flags(extra)
        try:
            e_fix, g_fix = [t.clone() for t in B.energy_grad(theta)]
        finally:
            vq.set_flags(old)
        old = vq.set_flags(extra | vq.VQE_FLAG_FP64_SWEEPS)
        try:
            e_f64, g_f64 = [t.clone() for t in B.energy_grad(theta)]
        finally:
            vq.set_flags(old)
        assert float((e_fix - e_f64).abs().max()) <= 1e-12
        assert float((g_fix - g_f64).abs().max()) <= 1e-11
    p = w.problems[5]
    idx = [0, 58, A.n_params - 1]
    e_o, g_o = oracle.gradient_direct(oracle.EnergyModel.from_problem(p, full=False), synth.hf_bitstring(6),
                                      w.excitations[0], w.thetas[5], idx)
    assert abs(float(e_fix[5]) - e_o) <= 1e-10
    assert np.abs(g_fix[5, idx].cpu().numpy() - g_o).max() <= 1e-9


def _instance_24q(seed):
    """24 qubits, 10 electrons (792 beta strings: the string-driven H psi),
    64 excitations of a seeded shuffle of the spin-conserving pool."""
    rng = np.random.default_rng([24, seed])
    p = synth.integrals.random_problem(rng, 12, 10, 6, label=f"24q[{seed}]")
    pool = synth.uccsd_pool(24, 10)
    exc = pool[rng.permutation(len(pool))[:64]]
    return p, exc, rng.normal(0.0, 0.05, size=64)


def test_string_driven_hpsi_matches_group_scan():
    """The alpha/beta string-driven H psi and the scan over all groups sum the
    same terms in different orders: energies within 1e-12, gradients within
    1e-11, single calls and a batch of two alike; H psi itself (complex, via
    vqe_apply_hamiltonian) within 1e-12 per entry."""
    insts = [_instance_24q(s) for s in (0, 1)]
    hams = [vq.Hamiltonian.from_problem(p) for p, _, _ in insts]
    ans = [vq.Ansatz(24, synth.hf_bitstring(10), e) for _, e, _ in insts]
    B = vq.Batch(hams, ans)
    theta = torch.as_tensor(np.stack([t for _, _, t in insts])).cuda().contiguous()
    e_s, g_s = [t.clone() for t in B.energy_grad(theta)]
    singles = [vq.energy_grad(h, a, theta[i]) for i, (h, a) in enumerate(zip(hams, ans))]
    psi = vq.state(ans[1], hams[1], theta[1])
    lam_s, _ = vq.apply_hamiltonian(hams[1], ans[1], psi)
    old = vq.set_flags(vq.VQE_FLAG_NO_STRINGS)
    try:
        e_r, g_r = [t.clone() for t in B.energy_grad(theta)]
        singles_r = [vq.energy_grad(h, a, theta[i]) for i, (h, a) in enumerate(zip(hams, ans))]
        lam_r, _ = vq.apply_hamiltonian(hams[1], ans[1], psi)
    finally:
        vq.set_flags(old)
    assert float((e_s - e_r).abs().max()) <= 1e-12
    assert float((g_s - g_r).abs().max()) <= 1e-11
    for i in range(2):
        assert abs(float(singles[i][0]) - float(singles_r[i][0])) <= 1e-12
        assert float((singles[i][1] - singles_r[i][1]).abs().max()) <= 1e-11
        assert abs(float(singles[i][0]) - float(e_s[i])) <= 1e-12
    assert float((lam_s - lam_r).abs().max()) <= 1e-12
    # and the HF energy (theta = 0) equals the Slater-Condon closed form
    p = insts[0][0]
    occ = range(10)
    e_hf = sum(p.h[P // 2, P // 2] for P in occ)
    for P in occ:
        for Q in occ:
            e_hf += 0.5 * p.eri[P // 2, P // 2, Q // 2, Q // 2]
            if P % 2 == Q % 2:
                e_hf -= 0.5 * p.eri[P // 2, Q // 2, Q // 2, P // 2]
    assert abs(float(vq.energy(hams[0], ans[0], np.zeros(64))) - e_hf) <= 1e-10


# ------------------------------------------------------------------ central finite differences
@pytest.mark.parametrize("cfg", ["config0", "config1"])
def test_adjoint_gradient_matches_central_differences(cfg):
    """Every gradient component against central differences of the library's
    own energies, h = 1e-5: truncation (h^2 E'''/6) and rounding (eps |E| / h)
    both stay below 1e-8 here, far under the 1e-7 bar."""
    if cfg == "config0":
        w = synth.config0()
        cases = [(w.problems[0], w.excitations[0], w.thetas[0])]
    else:
        w = synth.config1()
        cases = [(w.problems[i], w.excitations[i], w.thetas[i]) for i in (0, 63)]
    h = 1e-5
    for p, exc, th in cases:
        H = vq.Hamiltonian.from_problem(p)
        A = vq.Ansatz(p.n_qubits, synth.hf_bitstring(p.n_elec), exc)
        _, g = vq.energy_grad(H, A, th)
        g = g.cpu().numpy()
        fd = np.empty(len(th))
        for k in range(len(th)):
            tp, tm = th.copy(), th.copy()
            tp[k] += h
            tm[k] -= h
            fd[k] = (float(vq.energy(H, A, tp)) - float(vq.energy(H, A, tm))) / (2 * h)
        assert np.abs(fd - g).max() <= 1e-7, (cfg, float(np.abs(fd - g).max()))


@pytest.mark.parametrize("n", [14, 20])
def test_persistent_sweeps_equal_per_gate_launches(n):
    """The streaming gate sweeps run as one launch per gate; with
    VQE_FLAG_PERSISTENT_SWEEPS as one persistent launch per sweep. Both give the
    same bits: the same rotation per pair and the same gradient partial sums."""
    ns, _ = synth.configs.config2_sizes()
    p, exc, th = synth.config2_instance(int(np.nonzero(ns == n)[0][0]))
    H = vq.Hamiltonian.from_problem(p)
    A = vq.Ansatz(n, synth.hf_bitstring(p.n_elec), exc)
    out = []
    for flags in (vq.VQE_FLAG_FORCE_STREAMING, vq.VQE_FLAG_FORCE_STREAMING | vq.VQE_FLAG_PERSISTENT_SWEEPS):
        old = vq.set_flags(flags)
        try:
            e, g = vq.energy_grad(H, A, th)
            st = vq.state(A, H, th)
            out.append((float(e), g.clone(), st))
        finally:
            vq.set_flags(old)
    assert out[0][0] == out[1][0]
    assert torch.equal(out[0][1], out[1][1])
    assert torch.equal(out[0][2], out[1][2])
