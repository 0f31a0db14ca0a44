"""The allocation-free entry point (vqe_energy_grad_noalloc) against the regular one.

It is for callers that may not allocate device memory themselves; it runs the
same energy/gradient kernels on a static scratch array inside the library.
Here it is called twice in a row through the C ABI, and each time its energy
and gradient must match vqe_energy_grad on the same inputs within the parity
tolerances of the other GPU tests (1e-10 Ha, 1e-9 per component): first before
the regular call has built the pair's string or connectivity tables (the call
then scans every X-mask group), then after (the call uses those tables), with
real and with complex amplitudes. The device's free memory must not change
across the calls. This file sorts last so that a run stopping at the first
failure has run everything else.
"""
import numpy as np
import pytest
import torch

import synth
import paper_2311_01242_gb300 as vq
from paper_2311_01242_gb300.api import _ptr, _stream

pytestmark = pytest.mark.gpu

E_TOL = 1e-10
G_TOL = 1e-9


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    vq.build()
    return vq.load()


def _cases():
    w0 = synth.config0()
    yield w0.problems[0], w0.excitations[0], w0.thetas[0]
    w1 = synth.config1(2)
    yield w1.problems[1], w1.excitations[1], w1.thetas[1]
    ns, _ = synth.configs.config2_sizes()
    j = int(np.nonzero(ns == 16)[0][0])
    yield synth.config2_instance(j)


def _noalloc(lib, H, A, theta, with_grad=True):
    e = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
    g = torch.full((max(A.n_params, 1),), np.nan, dtype=torch.float64, device="cuda") if with_grad else None
    rc = lib.vqe_energy_grad_noalloc(H.handle, A.handle, _ptr(theta), _ptr(e), _ptr(g), _stream())
    assert rc == 0, lib.vqe_last_error()
    torch.cuda.synchronize()
    return e, g


@pytest.mark.parametrize("flags", [0, vq.VQE_FLAG_FORCE_COMPLEX], ids=["real", "complex"])
def test_noalloc_matches_regular_entry_on_two_calls(lib, flags):
    old = vq.set_flags(flags)
    try:
        for p, exc, th in _cases():
            H = vq.Hamiltonian.from_problem(p)
            A = vq.Ansatz(p.n_qubits, synth.hf_bitstring(p.n_elec), exc)
            rng = np.random.default_rng(p.n_qubits)
            for call in range(2):
                theta = torch.as_tensor(th + 0.1 * call * rng.normal(size=len(th))).cuda()
                # call 0 runs before the regular call has built the pair's tables
                e, g = _noalloc(lib, H, A, theta)
                e2, _ = _noalloc(lib, H, A, theta, with_grad=False)
                e_ref, g_ref = vq.energy_grad(H, A, theta)
                assert abs(float(e[0]) - float(e_ref)) <= E_TOL, (p.n_qubits, call)
                assert float((g - g_ref).abs().max()) <= G_TOL, (p.n_qubits, call)
                assert abs(float(e2[0]) - float(e_ref)) <= E_TOL
    finally:
        vq.set_flags(old)


def test_noalloc_allocates_no_device_memory(lib):
    vq.set_flags(0)
    ns, _ = synth.configs.config2_sizes()
    p, exc, th = synth.config2_instance(int(np.nonzero(ns == 16)[0][1]))
    theta = torch.as_tensor(th).cuda()
    e = torch.zeros(1, dtype=torch.float64, device="cuda")
    g = torch.zeros(len(th), dtype=torch.float64, device="cuda")
    for tables in (False, True):
        H = vq.Hamiltonian.from_problem(p)
        A = vq.Ansatz(p.n_qubits, synth.hf_bitstring(p.n_elec), exc)
        if tables:
            vq.workspace_bytes(H, A)  # builds the pair's string tables (an allocation of the regular path)
        # one call first: the first launch of a kernel may load its code onto the device
        assert lib.vqe_energy_grad_noalloc(H.handle, A.handle, _ptr(theta), _ptr(e), _ptr(g), _stream()) == 0
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        for _ in range(3):
            rc = lib.vqe_energy_grad_noalloc(H.handle, A.handle, _ptr(theta), _ptr(e), _ptr(g), _stream())
            assert rc == 0, lib.vqe_last_error()
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0, tables


def test_noalloc_rejects_instances_beyond_the_scratch(lib):
    n = 26  # 13 electrons: 1716 x 1716 sector states, 47 MB of real amplitudes > 16 MiB
    H = vq.Hamiltonian(n, [0], [1], [1.0])
    A = vq.Ansatz(n, synth.hf_bitstring(13), [[0, 14, -1, -1]])
    theta = torch.zeros(1, dtype=torch.float64, device="cuda")
    e = torch.zeros(1, dtype=torch.float64, device="cuda")
    g = torch.zeros(1, dtype=torch.float64, device="cuda")
    rc = lib.vqe_energy_grad_noalloc(H.handle, A.handle, _ptr(theta), _ptr(e), _ptr(g), _stream())
    assert rc == 1
    assert b"scratch" in lib.vqe_last_error()
