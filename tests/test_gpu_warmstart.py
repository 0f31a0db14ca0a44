"""Learned warm start: exact energies, training along a scan, and the gain.

Uses a 12-qubit scan (6 spatial orbitals, 6 electrons, 117 UCCSD angles) so
the whole pipeline runs in seconds: plain VQE with continuation on every 4th
scan point trains the network, which then starts VQE at held-out points.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
import paper_2311_01242_gb300 as vq
from paper_2311_01242_gb300 import warmstart as ws

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def scan_setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    vq.load()
    rs = np.linspace(0.8, 3.0, 40)
    scan = synth.draw_scan(np.random.default_rng(41), 6, 6, 6, rs)
    A = vq.Ansatz(12, synth.hf_bitstring(6), synth.uccsd_pool(12, 6))
    return scan, A


def test_lanczos_matches_oracle_exact_energy(scan_setup):
    scan, A = scan_setup
    for r in (0.8, 2.1):
        p = scan.at(r)
        g = ws.Geometry(p, r, A)
        e_gpu = ws.lanczos_ground(g.H, A, 12, 6)
        e_o = oracle.exact_ground_energy(p)
        assert abs(e_gpu - e_o) <= 1e-9


def test_vqe_bfgs_reaches_converged_energy_bounded_below(scan_setup):
    scan, A = scan_setup
    p = scan.at(1.5)
    g = ws.Geometry(p, 1.5, A)
    th, e, hist = ws.vqe_bfgs(g.H, A, np.zeros(A.n_params), gtol=1e-7)
    e0 = oracle.exact_ground_energy(p)
    assert e >= e0 - 1e-10                      # variational bound
    assert e <= hist[0][0] - 1e-3               # improves on the HF energy
    e_o = oracle.energy(oracle.EnergyModel.from_problem(p), synth.hf_bitstring(6), A.excitations, th)
    assert abs(e - e_o) <= 1e-10


def test_network_start_beats_hf_start(scan_setup):
    scan, A = scan_setup
    rs = scan.rs
    train = list(range(0, len(rs), 4))
    held = [10, 22, 30]
    geoms = [ws.Geometry(scan.at(rs[i]), rs[i], A) for i in train]
    thetas, energies, evals = ws.training_set(geoms, gtol=1e-6)
    model = ws.WarmStart(geoms[0].features.size, A.n_params, hidden=256, seed=0)
    hist = model.fit(np.stack([g.features for g in geoms]), thetas, steps=1500, lr=1e-3)
    assert hist[-1] < 0.05 * hist[0]
    mlp_evals, hf_evals, mlp_hit, hf_hit = [], [], 0, 0
    for i in held:
        g = ws.Geometry(scan.at(rs[i]), rs[i], A)
        e0 = ws.lanczos_ground(g.H, A, 12, 6)
        pred = model.predict(g.features[None, :])[0]
        e_pred = float(vq.energy(g.H, A, pred))
        e_hf = float(vq.energy(g.H, A, np.zeros(A.n_params)))
        assert e_pred < e_hf
        res = ws.compare_starts(g, {"hf": np.zeros(A.n_params), "mlp": pred}, e0, gtol=1e-6)
        # target: E_exact + 1 mHa, or the best converged energy + 1 mHa; a start that
        # converges to a worse minimum counts with all the evaluations it spent
        for name, acc in (("mlp", mlp_evals), ("hf", hf_evals)):
            r = res[name]
            acc.append((r["evals"] if r["evals"] is not None else r["evals_total"]) + (2 if name == "mlp" else 0))
        mlp_hit += res["mlp"]["evals"] is not None
        hf_hit += res["hf"]["evals"] is not None
    assert mlp_hit >= hf_hit and mlp_hit >= 2
    assert np.mean(mlp_evals) < np.mean(hf_evals), (mlp_evals, hf_evals)
