"""New coefficients for the same Pauli structure (vqe_set_coefs) and the
batched calls by instance list (vqe_energy_batched, vqe_energy_grad_batched).

A scan's geometries share their Pauli strings (Sec. 2.1.1 applied to h(r),
eri(r)), so a Hamiltonian built at one geometry and refolded with another's
coefficients must give that geometry's energies and gradients bit for bit,
through single calls, batches and captured graphs alike."""
import numpy as np
import pytest
import torch

import oracle
import synth
import paper_2311_01242_gb300 as vq
from paper_2311_01242_gb300 import batch as vb

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def scan():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    vq.load()
    w = synth.config1(4)
    terms = [vq.jordan_wigner(p.n_spatial, p.h, p.eri, p.c0) for p in w.problems]
    return w, terms


def test_set_coefs_equals_fresh_hamiltonian(scan):
    w, terms = scan
    n = w.problems[0].n_qubits
    A = vq.Ansatz(n, synth.hf_bitstring(w.problems[0].n_elec), w.excitations[0])
    th = w.thetas[0]
    H0 = vq.Hamiltonian(n, *terms[0])
    for j in (1, 2, 3):
        Hj = vq.Hamiltonian(n, *terms[j])
        H0.set_coefs_from(*terms[j])
        for flags in (0, vq.VQE_FLAG_NO_CLUSTER, vq.VQE_FLAG_FORCE_STREAMING):
            old = vq.set_flags(flags)
            try:
                e0, g0 = vq.energy_grad(H0, A, th)
                ej, gj = vq.energy_grad(Hj, A, th)
            finally:
                vq.set_flags(old)
            assert torch.equal(e0, ej), (j, flags)
            assert torch.equal(g0, gj), (j, flags)
    # and against the oracle at the last geometry
    p = w.problems[3]
    idx = [0, A.n_params // 2, A.n_params - 1]
    e_o, g_o = oracle.gradient_direct(oracle.EnergyModel.from_problem(p, full=False),
                                      synth.hf_bitstring(p.n_elec), w.excitations[0], th, idx)
    e, g = vq.energy_grad(H0, A, th)
    assert abs(float(e) - e_o) <= 1e-10
    assert np.abs(g.cpu().numpy()[idx] - g_o).max() <= 1e-9


def test_set_coefs_rejects_other_strings(scan):
    w, terms = scan
    n = w.problems[0].n_qubits
    H0 = vq.Hamiltonian(n, *terms[0])
    xs, zs, cs = terms[1]
    with pytest.raises(ValueError):
        H0.set_coefs_from(xs[1:], zs[1:], cs[1:])
    with pytest.raises(ValueError):
        H0.set_coefs(torch.zeros(len(xs) + 1, dtype=torch.float64, device="cuda"))


def test_set_coefs_reaches_batches_and_graphs(scan):
    w, terms = scan
    n = w.problems[0].n_qubits
    A = vq.Ansatz(n, synth.hf_bitstring(w.problems[0].n_elec), w.excitations[0])
    H0 = vq.Hamiltonian(n, *terms[0])
    refs = [vq.Hamiltonian(n, *terms[j]) for j in range(4)]
    B = vq.Batch([H0], [A])
    theta = torch.as_tensor(w.thetas[0]).reshape(1, -1).cuda().contiguous()
    gb = vb.GraphBatch(B)
    g1 = vq.GraphEnergyGrad(H0, A)
    for j in (2, 0, 3):
        c = torch.as_tensor(terms[j][2]).cuda()
        H0.set_coefs(c)
        e_ref, g_ref = vq.energy_grad(refs[j], A, w.thetas[0])
        e_b, g_b = B.energy_grad(theta)
        assert torch.equal(e_b[0], e_ref) and torch.equal(g_b[0, :A.n_params], g_ref)
        e_g, g_g = gb(theta)
        assert torch.equal(e_g[0], e_ref) and torch.equal(g_g[0, :A.n_params], g_ref)
        e_1, g_1 = g1(w.thetas[0])
        assert torch.equal(e_1[0], e_ref) and torch.equal(g_1, g_ref)


def test_batched_by_instance_list_matches_batch_handle(scan):
    w, terms = scan
    # two resident 12-qubit geometries and two streamed 14-qubit instances
    ns, _ = synth.configs.config2_sizes()
    insts = [(w.problems[i], w.excitations[i], w.thetas[i]) for i in range(2)]
    insts += [synth.config2_instance(int(np.nonzero(ns == 14)[0][k])) for k in range(2)]
    hams = [vq.Hamiltonian.from_problem(p) for p, _, _ in insts]
    ans = [vq.Ansatz(p.n_qubits, synth.hf_bitstring(p.n_elec), e) for p, e, _ in insts]
    thetas = [torch.as_tensor(t).cuda() for _, _, t in insts]
    e, gs = vq.energy_grad_batched(hams, ans, thetas)
    B = vq.Batch(hams, ans)
    th = torch.zeros(len(insts), B.max_params, dtype=torch.float64)
    for i, (_, _, t) in enumerate(insts):
        th[i, :len(t)] = torch.as_tensor(t)
    e_ref, g_ref = B.energy_grad(th.cuda())
    assert torch.equal(e, e_ref)
    for i, a in enumerate(ans):
        assert torch.equal(gs[i], g_ref[i, :a.n_params])
    e2, none = vq.energy_grad_batched(hams, ans, thetas, with_grad=False)
    assert none is None and torch.equal(e2, e_ref)
    # second call reuses the cached plan; results unchanged
    e3, gs3 = vq.energy_grad_batched(hams, ans, thetas)
    assert torch.equal(e3, e_ref) and all(torch.equal(a, b) for a, b in zip(gs3, gs))


def test_batched_plan_survives_handle_turnover(scan):
    w, _ = scan
    p, exc, t = w.problems[0], w.excitations[0], w.thetas[0]
    A = vq.Ansatz(p.n_qubits, synth.hf_bitstring(p.n_elec), exc)
    th = [torch.as_tensor(t).cuda()]
    e_ref, _ = vq.energy_grad(vq.Hamiltonian.from_problem(p), A, t)
    for _ in range(20):  # more instance lists than the plan cache holds
        H = vq.Hamiltonian.from_problem(p)
        e, gs = vq.energy_grad_batched([H], [A], th)
        assert torch.equal(e[0], e_ref)
        del H
