"""CUDA-graph runner and autotuner for batched energy+gradient evaluation.

A batch of independent instances (geometries, molecules of uneven size) is
evaluated by libvqe in one resident launch for the instances that fit shared
memory and, for the others, in one persistent launch that works through a
device queue of per-instance tasks (gate rotations on ranges of pairs, H psi on
ranges of output strings, reductions), plus a small finalising launch.
GraphBatch captures that launch sequence once and replays it with new angles
written in place into the captured theta buffer. autotune() times the batch's
launch shapes (persistent CTAs per SM, amplitude pairs per gate task, resident
sweep width) and keeps the fastest, cached in a JSON file keyed by the batch's
sizes; results never depend on the launch shape.
"""
import hashlib
import json
import os

import torch

from . import api


class GraphBatch:
    def __init__(self, batch: api.Batch, with_grad=True, device="cuda"):
        self.batch = batch
        n, ld = batch.n_inst, max(batch.max_params, 1)
        self.theta = torch.zeros(n, ld, dtype=torch.float64, device=device)
        self.energies = torch.zeros(n, dtype=torch.float64, device=device)
        self.grads = torch.zeros(n, ld, dtype=torch.float64, device=device) if with_grad else None
        self.ws = api.alloc_workspace(batch.workspace_bytes(with_grad), device)
        self.with_grad = with_grad
        self._run()  # first call outside capture (loads kernels, sets shared-memory limits)
        torch.cuda.synchronize()
        side = torch.cuda.Stream(device=device)
        side.wait_stream(torch.cuda.current_stream())
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.stream(side):
            with torch.cuda.graph(self.graph, stream=side):
                self._run()
        torch.cuda.current_stream().wait_stream(side)

    def _run(self):
        self.batch.energy_grad(self.theta, self.energies, self.grads, self.ws, with_grad=self.with_grad)

    def __call__(self, theta=None):
        if theta is not None:
            self.theta[:, :theta.shape[1]].copy_(theta)
        self.graph.replay()
        return self.energies, self.grads


def signature(hams, ansatze):
    key = []
    for h, a in zip(hams, ansatze):
        hi, ai = h.info(), a.info()
        key.append((ai["n_qubits"], ai["n_params"], ai["sector_dim"], ai["n_pairs"], hi["n_groups"]))
    return hashlib.sha256(json.dumps(key).encode()).hexdigest()[:20]


def _time(batch, theta, energies, grads, ws, reps):
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    batch.energy_grad(theta, energies, grads, ws)
    torch.cuda.synchronize()
    start.record()
    for _ in range(reps):
        batch.energy_grad(theta, energies, grads, ws)
    end.record()
    torch.cuda.synchronize()
    return start.elapsed_time(end) / reps


def autotune(batch, theta, ctas_per_sm=(1, 2), gate_chunk=(512, 1024, 2048), sweep_threads=(128,), reps=5,
             cache_path=None):
    """Pick (ctas_per_sm, gate_chunk, sweep_threads) by timing; returns (choice, timings in ms)."""
    lib = api._lib()
    sig = signature(batch.hams, batch.ansatze)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
    if sig in cache:
        choice = tuple(cache[sig]["choice"])
        api._check(lib.vqe_batch_set_tuning(batch.handle, *choice))
        return choice, cache[sig]["timings"]
    energies = torch.empty(batch.n_inst, dtype=torch.float64, device=theta.device)
    grads = torch.empty(batch.n_inst, theta.shape[1], dtype=torch.float64, device=theta.device)
    ws = api.alloc_workspace(batch.workspace_bytes(True), theta.device)
    timings = {}
    for c in ctas_per_sm:
        for g in gate_chunk:
            for sw in sweep_threads:
                api._check(lib.vqe_batch_set_tuning(batch.handle, c, g, sw))
                timings[f"{c},{g},{sw}"] = _time(batch, theta, energies, grads, ws, reps)
    best = min(timings, key=timings.get)
    choice = tuple(int(v) for v in best.split(","))
    api._check(lib.vqe_batch_set_tuning(batch.handle, *choice))
    if cache_path:
        cache[sig] = {"choice": list(choice), "timings": timings}
        os.makedirs(os.path.dirname(os.path.abspath(cache_path)), exist_ok=True)
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1)
    return choice, timings
