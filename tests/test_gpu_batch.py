"""Batched evaluation of uneven instances: gate-major streaming, CUDA-graph
replay and autotuned launch shapes, checked against single-instance calls and
the oracle."""
import numpy as np
import pytest
import torch

import oracle
import synth
import paper_2311_01242_gb300 as vq
from paper_2311_01242_gb300 import batch as vb

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mixed():
    """Two 12-qubit scan geometries (shared-memory resident) and config-2
    instances of 14 and 16 qubits (streamed), in one batch."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    vq.load()
    ns, _ = synth.configs.config2_sizes()
    picks = [int(np.nonzero(ns == n)[0][k]) for n in (14, 16) for k in range(3)]
    insts = [synth.config2_instance(j) for j in picks]
    w1 = synth.config1(2)
    insts += [(w1.problems[i], w1.excitations[i], w1.thetas[i]) for i in range(2)]
    hams = [vq.Hamiltonian.from_problem(p) for p, _, _ in insts]
    ans = [vq.Ansatz(p.n_qubits, synth.hf_bitstring(p.n_elec), e) for p, e, _ in insts]
    B = vq.Batch(hams, ans)
    theta = torch.zeros(len(insts), B.max_params, dtype=torch.float64)
    for i, (_, _, th) in enumerate(insts):
        theta[i, :len(th)] = torch.as_tensor(th)
    return insts, hams, ans, B, theta.cuda()


def test_batch_matches_single_instance_calls(mixed):
    insts, hams, ans, B, theta = mixed
    e, g = B.energy_grad(theta)
    e, g = e.cpu().numpy(), g.cpu().numpy()
    for i, (p, exc, th) in enumerate(insts):
        e1, g1 = vq.energy_grad(hams[i], ans[i], theta[i, :len(th)])
        assert abs(float(e1) - e[i]) <= 1e-12
        assert np.abs(g1.cpu().numpy() - g[i, :len(th)]).max() <= 1e-12


def test_batch_matches_oracle_on_streamed_instances(mixed):
    insts, hams, ans, B, theta = mixed
    e, g = B.energy_grad(theta)
    e, g = e.cpu().numpy(), g.cpu().numpy()
    for i in (0, 3):
        p, exc, th = insts[i]
        idx = [0, len(exc) - 1]
        model = oracle.EnergyModel.from_problem(p, full=False)
        e_o, g_o = oracle.gradient_direct(model, synth.hf_bitstring(p.n_elec), exc, th, idx)
        assert abs(e[i] - e_o) <= 1e-10
        assert np.abs(g[i, idx] - g_o).max() <= 1e-9


def _same(e, g, e_ref, g_ref, ms):
    """Bitwise equal energies and gradients (each row up to its instance's M)."""
    if not torch.equal(e, e_ref):
        return False
    return all(torch.equal(g[i, :m], g_ref[i, :m]) for i, m in enumerate(ms))


def test_graph_replay_and_tuning_do_not_change_results(mixed, tmp_path):
    insts, hams, ans, B, theta = mixed
    ms = [a.n_params for a in ans]
    e_ref, g_ref = [t.clone() for t in B.energy_grad(theta)]
    gb = vb.GraphBatch(B)
    e, g = gb(theta)
    assert _same(e, g, e_ref, g_ref, ms)
    theta2 = theta + 0.01
    e2, g2 = gb(theta2)
    e2_ref, g2_ref = B.energy_grad(theta2.contiguous())
    assert _same(e2, g2, e2_ref, g2_ref, ms)
    cache = str(tmp_path / "tune.json")
    choice, timings = vb.autotune(B, theta, ctas_per_sm=(1, 2), gate_chunk=(256, 1024), sweep_threads=(64, 128),
                                  reps=2, cache_path=cache)
    assert len(timings) == 8
    assert choice in [(c, g, w) for c in (1, 2) for g in (256, 1024) for w in (64, 128)]
    e3, g3 = B.energy_grad(theta)
    assert _same(e3, g3, e_ref, g_ref, ms)
    choice2, _ = vb.autotune(B, theta, cache_path=cache)  # served from the cache
    assert choice2 == choice


def test_host_entry_replays_graph_with_new_inputs(mixed):
    """vqe_batch_energy_grad_host with pinned buffers replays a captured graph
    from the second call on; new angles written into the same buffers, a flag
    change and a tuning change must all show up in the results (mixed batch:
    resident and streamed instances)."""
    insts, hams, ans, B, theta = mixed
    n, M = len(insts), B.max_params
    th_h = torch.empty(n, M, dtype=torch.float64).pin_memory()
    e_h = torch.empty(n, dtype=torch.float64).pin_memory()
    g_h = torch.empty(n, M, dtype=torch.float64).pin_memory()
    ws = vq.alloc_workspace(B.host_workspace_bytes(True))
    rng = np.random.default_rng(501)
    for step in range(4):
        th = theta.cpu() * (1.0 + 0.5 * step) + torch.as_tensor(rng.normal(0, 0.01, size=(n, M))) * (theta.cpu() != 0)
        th_h.copy_(th)
        B.energy_grad_host(th_h.numpy(), e_h.numpy(), g_h.numpy(), ws)
        e_d, g_d = B.energy_grad(th.cuda().contiguous())
        assert torch.equal(e_h, e_d.cpu()), step
        for i, a in enumerate(ans):  # columns past an instance's parameters are not written
            assert torch.equal(g_h[i, :a.n_params], g_d.cpu()[i, :a.n_params]), (step, i)
    old = vq.set_flags(vq.VQE_FLAG_FP64_SWEEPS)
    try:
        B.energy_grad_host(th_h.numpy(), e_h.numpy(), g_h.numpy(), ws)
        e_d, g_d = B.energy_grad(th_h.cuda())
        assert torch.equal(e_h, e_d.cpu())
        for i, a in enumerate(ans):
            assert torch.equal(g_h[i, :a.n_params], g_d.cpu()[i, :a.n_params]), i
    finally:
        vq.set_flags(old)
    B.energy_grad_host(th_h.numpy(), e_h.numpy(), g_h.numpy(), ws)
    B.set_tuning(1, 512, 96)
    try:
        e2 = e_h.clone()
        B.energy_grad_host(th_h.numpy(), e_h.numpy(), g_h.numpy(), ws)
        B.energy_grad_host(th_h.numpy(), e_h.numpy(), g_h.numpy(), ws)
        assert torch.equal(e_h, e2)
    finally:
        B.set_tuning(0, 1024, 128)


def test_prepared_host_call_matches_host_entry(mixed):
    """Batch.host_call marshals the host arrays once; each call reads the current
    contents of theta and fills the same result arrays."""
    insts, hams, ans, B, theta = mixed
    n, M = len(insts), B.max_params
    th_h = torch.empty(n, M, dtype=torch.float64).pin_memory()
    e_h = torch.empty(n, dtype=torch.float64).pin_memory()
    g_h = torch.empty(n, M, dtype=torch.float64).pin_memory()
    ws = vq.alloc_workspace(B.host_workspace_bytes(True))
    call = B.host_call(th_h.numpy(), e_h.numpy(), g_h.numpy(), ws)
    e_ref = np.zeros(n)
    g_ref = np.zeros((n, M))
    ws2 = vq.alloc_workspace(B.host_workspace_bytes(True))
    for scale in (1.0, 0.5, 2.0):
        th_h.copy_(theta.cpu() * scale)
        call()
        B.energy_grad_host(np.ascontiguousarray(th_h.numpy()), e_ref, g_ref, ws2)
        assert np.array_equal(e_h.numpy(), e_ref), scale
        for i, a in enumerate(ans):
            assert np.array_equal(g_h.numpy()[i, :a.n_params], g_ref[i, :a.n_params]), (scale, i)


def test_persistent_batch_equals_single_calls_bitwise(mixed):
    """The streamed instances (14 and 16 qubits) run in the persistent launch;
    every energy and gradient equals vqe_energy_grad's bit for bit, for every
    launch shape."""
    insts, hams, ans, B, theta = mixed
    streamed = [i for i, (p, _, _) in enumerate(insts) if p.n_qubits >= 14]
    ref = []
    for i in streamed:
        m = ans[i].n_params
        e1, g1 = vq.energy_grad(hams[i], ans[i], theta[i, :m].contiguous())
        ref.append((e1.clone(), g1.clone()))
    for shape in ((0, 1024, 128), (1, 256, 128), (2, 4096, 128)):
        B.set_tuning(*shape)
        t = B.tuning()
        assert t["grid"] > 0 and t["n_tasks"] > 0
        e, g = B.energy_grad(theta)
        for (e1, g1), i in zip(ref, streamed):
            m = ans[i].n_params
            assert torch.equal(e[i], e1), (shape, i)
            assert torch.equal(g[i, :m], g1), (shape, i)
    B.set_tuning(0, 1024, 128)


def test_persistent_wait_runs_out_and_reports_timeout(mixed):
    """A task made to wait for a count that nothing reaches: its wait ends after
    the budget, the status word reports the task, every persistent output is
    NaN, the resident instances are untouched, the host-buffer call returns
    VQE_ERR_TIMEOUT, and the next normal call is correct again."""
    insts, hams, ans, B, theta = mixed
    streamed = [i for i, (p, _, _) in enumerate(insts) if p.n_qubits >= 14]
    resident = [i for i in range(len(insts)) if i not in streamed]
    e_ref, g_ref = [t.clone() for t in B.energy_grad(theta)]
    ws = vq.alloc_workspace(B.workspace_bytes(True))
    e = torch.zeros(len(insts), dtype=torch.float64, device="cuda")
    g = torch.zeros(len(insts), B.max_params, dtype=torch.float64, device="cuda")
    n_tasks = B.tuning()["n_tasks"]
    for probe in (0, n_tasks // 2):
        B.set_wait(budget_ns=2_000_000, probe_task=probe)
        try:
            B.energy_grad(theta, e, g, ws)
            with pytest.raises(vq.VQEError) as ex:
                B.status(ws)
            assert ex.value.code == 4 and "ran out" in str(ex.value)
            assert torch.isnan(e[streamed]).all()
            for i in resident:
                assert torch.equal(e[i], e_ref[i])
            n, M = len(insts), B.max_params
            th_h = theta.cpu().clone().pin_memory()
            e_h = torch.empty(n, dtype=torch.float64).pin_memory()
            g_h = torch.empty(n, M, dtype=torch.float64).pin_memory()
            wsh = vq.alloc_workspace(B.host_workspace_bytes(True))
            with pytest.raises(vq.VQEError) as ex:
                B.energy_grad_host(th_h.numpy(), e_h.numpy(), g_h.numpy(), wsh)
            assert ex.value.code == 4
        finally:
            B.set_wait(2_000_000_000, -1)
    B.energy_grad(theta, e, g, ws)
    B.status(ws)
    assert torch.equal(e, e_ref)
