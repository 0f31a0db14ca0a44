"""ADAPT-VQE screening (Sec. 2.1.1, ADAPT-VQE) through the C ABI against the oracle.

vqe_pool_gradients returns E(theta) and g_j = 2 Re <H psi| T_j - T_j^dagger |psi>
for every operator of a pool. Bar: |dE| <= 1e-10 Ha, |dg_j| <= 1e-9, as for the
adjoint gradient. Cases: the 12-qubit scan problem with the full 117-operator
pool (every kernel-path switch), 14-20 qubit instances, the empty starting
ansatz against the Slater-Condon closed form (20 and 30 qubits), the identity
with the adjoint gradient of the extended ansatz, determinism and graph
replay, rejected arguments, and the adaptive loop against the oracle's.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
import paper_2311_01242_gb300 as vq
from paper_2311_01242_gb300 import adapt as vadapt

pytestmark = pytest.mark.gpu

E_TOL = 1e-10
G_TOL = 1e-9

FLAGS = [0, vq.VQE_FLAG_NO_STRINGS, vq.VQE_FLAG_FORCE_COMPLEX]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    vq.build()
    vq.load()
    yield
    vq.set_flags(0)


def gpu_screen(p, exc, th, pool, drop_tol=1e-14, flags=0):
    old = vq.set_flags(flags)
    try:
        hf = synth.hf_bitstring(p.n_elec)
        H = vq.Hamiltonian.from_problem(p, drop_tol)
        A = vq.Ansatz(p.n_qubits, hf, exc)
        P = vq.Ansatz(p.n_qubits, hf, pool)
        e, g = vq.pool_gradients(H, A, P, th)
        torch.cuda.synchronize()
        return float(e), g.cpu().numpy()
    finally:
        vq.set_flags(old)


def test_12_qubit_full_pool_matches_oracle():
    w = synth.config1(2)
    p = w.problems[1]
    pool = synth.uccsd_pool(12, 6)
    rng = np.random.default_rng(301)
    exc = pool[rng.permutation(len(pool))[:40]]
    th = rng.normal(0, 0.1, size=40)
    model = oracle.EnergyModel.from_problem(p)
    e_o, g_o = oracle.pool_gradients(model, 63, exc, th, pool)
    for flags in FLAGS:
        e, g = gpu_screen(p, exc, th, pool, flags=flags)
        assert abs(e - e_o) <= E_TOL, flags
        assert np.abs(g - g_o).max() <= G_TOL, flags


@pytest.mark.parametrize("n", [14, 16])
def test_uneven_instances_match_oracle(n):
    """14- and 16-qubit instances of the uneven batch (oracle in sector form),
    48 operators of the full UCCSD pool."""
    ns, _ = synth.configs.config2_sizes()
    j = int(np.nonzero(ns == n)[0][0])
    p, exc, th = synth.config2_instance(j)
    pool = synth.uccsd_pool(n, p.n_elec)
    model = oracle.EnergyModel.from_problem(p, full=False)
    hf = synth.hf_bitstring(p.n_elec)
    sel = np.random.default_rng(302 + j).choice(len(pool), size=min(len(pool), 48), replace=False)
    e_o, g_o = oracle.pool_gradients(model, hf, exc, th, pool[sel])
    e, g = gpu_screen(p, exc, th, pool[sel])
    assert abs(e - e_o) <= E_TOL
    assert np.abs(g - g_o).max() <= G_TOL


@pytest.mark.parametrize("flags", FLAGS)
def test_empty_ansatz_matches_slater_condon_20_qubits(flags):
    ns, _ = synth.configs.config2_sizes()
    j = int(np.nonzero(ns == 20)[0][0])
    p, _, _ = synth.config2_instance(j)
    pool = synth.uccsd_pool(20, p.n_elec)
    hf = synth.hf_bitstring(p.n_elec)
    e, g = gpu_screen(p, pool[:0], np.zeros(0), pool, flags=flags)
    g_sc = oracle.hf_pool_gradients(p, hf, pool)
    assert np.abs(g - g_sc).max() <= G_TOL
    assert np.abs(g_sc).max() > 1e-2


def test_empty_ansatz_matches_slater_condon_30_qubits():
    """30 qubits (9.0M sector amplitudes): 256 operators sampled from the
    3,500-operator pool against the closed form at the reference state."""
    w = synth.config3()
    p = w.problems[0]
    pool = synth.uccsd_pool(30, 10)
    sel = np.sort(np.random.default_rng(303).choice(len(pool), size=256, replace=False))
    e, g = gpu_screen(p, pool[:0], np.zeros(0), pool[sel], drop_tol=w.drop_tol)
    _, _, c_all = vq.jordan_wigner(p.n_spatial, p.h, p.eri, 0.0, 0.0)
    dropped = float(np.abs(c_all[np.abs(c_all) < w.drop_tol]).sum())
    g_sc = oracle.hf_pool_gradients(p, synth.hf_bitstring(10), pool[sel])
    assert np.abs(g - g_sc).max() <= G_TOL + 2 * dropped


def test_pool_gradient_equals_adjoint_gradient_of_extended_ansatz():
    """Appending operator j at angle 0 and taking the adjoint gradient of that
    last angle (a different kernel path) gives g_j; 18 qubits, random theta."""
    ns, _ = synth.configs.config2_sizes()
    j = int(np.nonzero(ns == 18)[0][0])
    p, exc, th = synth.config2_instance(j)
    pool = synth.uccsd_pool(p.n_qubits, p.n_elec)
    hf = synth.hf_bitstring(p.n_elec)
    H = vq.Hamiltonian.from_problem(p)
    A = vq.Ansatz(p.n_qubits, hf, exc)
    P = vq.Ansatz(p.n_qubits, hf, pool)
    e, g = vq.pool_gradients(H, A, P, th)
    g = g.cpu().numpy()
    for k in np.random.default_rng(304).choice(len(pool), size=6, replace=False):
        ext = vq.Ansatz(p.n_qubits, hf, np.concatenate([exc, pool[k:k + 1]]))
        e2, g2 = vq.energy_grad(H, ext, np.append(th, 0.0))
        assert abs(float(e2) - float(e)) <= E_TOL
        assert abs(float(g2[-1]) - g[k]) <= G_TOL, k


def test_deterministic_and_graph_capturable():
    w = synth.config1(1)
    p = w.problems[0]
    pool = synth.uccsd_pool(12, 6)
    H = vq.Hamiltonian.from_problem(p)
    A = vq.Ansatz(12, 63, pool[:30])
    P = vq.Ansatz(12, 63, pool)
    th = torch.as_tensor(w.thetas[0][:30]).cuda()
    ws = vq.alloc_workspace(vq.pool_workspace_bytes(H, A, P))
    e1, g1 = [t.clone() for t in vq.pool_gradients(H, A, P, th, workspace=ws)]
    e2, g2 = vq.pool_gradients(H, A, P, th, workspace=ws)
    assert torch.equal(e1, e2) and torch.equal(g1, g2)
    e_out = torch.zeros(1, dtype=torch.float64, device="cuda")
    g_out = torch.zeros(len(pool), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        with torch.cuda.graph(graph, stream=side):
            vq.pool_gradients(H, A, P, th, workspace=ws, out=(e_out, g_out))
    torch.cuda.current_stream().wait_stream(side)
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(e_out[0], e1) and torch.equal(g_out, g1)


def test_rejects_other_sector_and_short_workspace():
    w = synth.config1(1)
    p = w.problems[0]
    H = vq.Hamiltonian.from_problem(p)
    A = vq.Ansatz(12, 63, synth.uccsd_pool(12, 6)[:5])
    wrong = vq.Ansatz(12, 31, synth.uccsd_pool(12, 5)[:5])  # 5 electrons
    with pytest.raises(vq.VQEError):
        vq.pool_gradients(H, A, wrong, np.zeros(5))
    P = vq.Ansatz(12, 63, synth.uccsd_pool(12, 6))
    ws = vq.alloc_workspace(vq.pool_workspace_bytes(H, A, P) - 256)
    with pytest.raises(vq.VQEError):
        vq.pool_gradients(H, A, P, np.zeros(5), workspace=ws)
    empty = vq.Ansatz(12, 63, np.zeros((0, 4), dtype=np.int32))
    e, g = vq.pool_gradients(H, A, empty, np.zeros(5))
    assert g.numel() == 0 and np.isfinite(float(e))


def test_adapt_loop_matches_oracle_loop():
    """The GPU-driven loop reaches the oracle loop's energies round by round.
    config 0 (closed shell) has exact alpha/beta mirror ties in |g|, so there
    only energies and gradient norms are compared (a mirror choice leaves them
    unchanged) and the end point is full CI; the 8-qubit 3-electron problem has
    no such symmetry, so the chosen operators must match as well."""
    w = synth.config0()
    p = w.problems[0]
    model = oracle.EnergyModel.from_problem(p)
    e_o, ch_o, _, hist_o = oracle.adapt_vqe(model, 3, w.excitations[0], grad_tol=1e-6, max_ops=6)
    r = vadapt.adapt_vqe(vq.Hamiltonian.from_problem(p), 4, 3, w.excitations[0], grad_tol=1e-6, max_ops=6)
    assert len(r.history) == len(hist_o)
    for (eg, ng, _), (eo, no, _) in zip(r.history, hist_o):
        assert abs(eg - eo) <= 1e-8 and abs(ng - no) <= 1e-6
    assert abs(r.energy - oracle.exact_ground_energy(p)) <= 1e-8

    p8 = synth.random_problem(np.random.default_rng(305), 4, 3, 3)
    pool8 = synth.uccsd_pool(8, 3)
    model8 = oracle.EnergyModel.from_problem(p8)
    e_o, ch_o, _, hist_o = oracle.adapt_vqe(model8, 7, pool8, grad_tol=1e-4, max_ops=4)
    r = vadapt.adapt_vqe(vq.Hamiltonian.from_problem(p8), 8, 7, pool8, grad_tol=1e-4, max_ops=4)
    assert r.chosen == ch_o
    for (eg, ng, jg), (eo, no, jo) in zip(r.history, hist_o):
        assert abs(eg - eo) <= 1e-8 and abs(ng - no) <= 1e-6 and jg == jo
