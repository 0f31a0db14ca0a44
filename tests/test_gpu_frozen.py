"""Frozen-core folding (Eq. 3, Sec. 2.1.3) through the whole GPU path.

With the frozen orbitals doubly occupied, a UCCSD state over the active
orbitals lives in the block where the full Hamiltonian equals the folded one,
so E and dE/dtheta of the folded problem (fewer qubits) must equal those of the
full problem with the same excitations moved to the active orbitals' qubits."""
import numpy as np
import pytest
import torch

import oracle
import synth
import paper_2311_01242_gb300 as vq

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    vq.build()
    vq.load()


@pytest.mark.parametrize("seed,n_s,n_elec,frozen", [(131, 6, 6, [0]), (132, 7, 8, [0, 1])])
def test_folded_problem_equals_full_problem(seed, n_s, n_elec, frozen):
    p = synth.random_problem(np.random.default_rng(seed), n_s, n_elec, 3)
    active = [q for q in range(n_s) if q not in frozen]
    h2, eri2, c2 = vq.fold_frozen(p.h, p.eri, p.c0, frozen, active)
    small = synth.Problem(len(active), n_elec - 2 * len(frozen), h2, eri2, c2)
    exc = synth.uccsd_pool(small.n_qubits, small.n_elec)
    th = np.random.default_rng(seed + 1).normal(0, 0.2, size=len(exc))
    e_s, g_s = vq.energy_grad(vq.Hamiltonian.from_problem(small),
                              vq.Ansatz(small.n_qubits, synth.hf_bitstring(small.n_elec), exc), th)
    shift = 2 * len(frozen)  # frozen orbitals are the lowest, so active qubit q is full qubit q + shift
    exc_full = np.where(exc >= 0, exc + shift, exc).astype(np.int32)
    e_f, g_f = vq.energy_grad(vq.Hamiltonian.from_problem(p), vq.Ansatz(2 * n_s, synth.hf_bitstring(n_elec), exc_full),
                              th)
    assert abs(float(e_s) - float(e_f)) <= 1e-10
    assert np.abs(g_s.cpu().numpy() - g_f.cpu().numpy()).max() <= 1e-9
    # and the folded problem against the oracle's own fold
    red = oracle.fold_frozen(p, frozen, active)
    e_o, _ = oracle.gradient_direct(oracle.EnergyModel.from_problem(red), synth.hf_bitstring(red.n_elec), exc, th)
    assert abs(float(e_s) - e_o) <= 1e-10
