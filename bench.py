#!/usr/bin/env python
"""Throughput of the VQE hot path: energy + adjoint-gradient evaluations per second.

Workload (default): the 12-qubit bond-stretch scan, 64 geometries batched in one
launch, 6 electrons, all 117 spin-conserving singles and doubles, theta ~ N(0, 0.05),
random integrals standing in for the molecule (synth.config1). A step evaluates
E(theta) and dE/dtheta for all 64 geometries.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank evaluates its own copy of the batch (weak
scaling, no collective on the data path); rank 0 prints one JSON line.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "energy+adjoint-grad evals/s & HBM GB/s at 12/20/30 qubits; time to 1 mHa vs plain"
UNIT = "evals/s"
WORKLOAD = "12 qubits, 6 electrons, 64-geometry scan r in [0.8,3.0], 117 UCCSD excitations"
# FP64 peak for the ALU roofline: 2 DFMA per clock per SM (measured by a DFMA
# throughput probe on this GB300: 600 GFMA/s at ~2.0 GHz) x 152 SMs x 2070 MHz
# x 2 flops per FMA.
FP64_DFMA_PER_CLK_SM = 2
N_SMS = 152
SM_MAX_MHZ = 2070.0
FP64_PEAK_TFLOPS = FP64_DFMA_PER_CLK_SM * N_SMS * SM_MAX_MHZ * 1e6 * 2 / 1e12
# 64-bit integer high multiplies (__umul64hi) sustained per clock per SM, measured
# by an integer throughput probe on this GB300 (the fixed-point kernels' multiply)
INT_MUL64_PER_CLK_SM = 6.7
# sources of the single-instance kernels (their ncu summaries name these files' sha256)
RESIDENT_SRC = ["vqe_kernels.cu", "vqe_device.cuh"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=None)
    ap.add_argument("--workload", choices=["scan12", "warmstart", "config3", "config2", "q24", "adapt30",
                                           "puccd11", "puccd24", "adapt24", "adapt12", "noalloc16", "hpsi30s", "q20"],
                    default="scan12",
                    help="scan12: the throughput line (default); warmstart: the 16-qubit learned-warm-start "
                         "comparison (time to 1 mHa vs the plain HF start); config3: one 30-qubit instance; "
                         "config2: 256 uneven 14-20-qubit instances replayed from a CUDA graph; q24: one 24-qubit "
                         "instance (10 electrons, 256 angles); adapt30: ADAPT-VQE screening of the full "
                         "3,500-operator pool at the 30-qubit state (adapt24: the same at the 24-qubit "
                         "state); adapt12: the whole ADAPT-VQE loop on one 12-qubit geometry (pool gradient "
                         "norm below 1e-3 or 60 operators); puccd11: pUCCD in the hard-core boson "
                         "form, 11 orbitals x 64 geometries in one launch; puccd24: one 24-orbital pUCCD "
                         "instance (12 pairs, 2.7M boson states); noalloc16: the allocation-free entry point "
                         "against vqe_energy_grad on one 16-qubit instance; hpsi30s: the 30-qubit Hamiltonian in "
                         "the 4-alpha/5-beta sector (4.1M states, the same wide block form of the string-driven "
                         "H psi as config3 on a smaller case, for full ncu captures); q20: one 20-qubit instance "
                         "(the first of config2's 20-qubit instances)")
    ap.add_argument("--held-out", type=int, default=24, help="warmstart: held-out scan points compared")
    ap.add_argument("--skip", nargs="*", default=[], choices=["config3", "config2", "q20", "warmstart", "complex"],
                    help="default line: leave these per-config entries out")
    ap.add_argument("--no-per-config", action="store_true", help="default line: headline only")
    ap.add_argument("--pool-ops", type=int, default=None,
                    help="adapt30/adapt24: screen only the first N pool operators (a small profiling case)")
    return ap.parse_args()


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu_index = gpu_index
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "20",
                 "-i", str(self.gpu_index)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()
        time.sleep(0.1)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def stop(self, t_begin=None, t_end=None):
        """Summary of the samples taken in [t_begin, t_end] (time.time(); all if None)."""
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.05)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lines = [(t, ln) for t, ln in self.lines
                 if (t_begin is None or t >= t_begin) and (t_end is None or t <= t_end)]
        if not lines:  # a region shorter than the sampling interval: the nearest samples
            lines = self.lines[-2:]
        for _, line in lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def gpu_index_for(local_rank):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    ids = [v.strip() for v in vis.split(",") if v.strip()]
    if ids and all(i.isdigit() for i in ids) and local_rank < len(ids):
        return int(ids[local_rank])
    return local_rank


# ------------------------------------------------------------------ CPU baseline (oracle)
_CACHE = {}


def _oracle_task(args):
    """One geometry: build the oracle's Hamiltonian (untimed, cached per process),
    then time its energy + gradient."""
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    i, n_comp = args
    import oracle
    import synth
    if "w" not in _CACHE:
        _CACHE["w"] = synth.config1()
    w = _CACHE["w"]
    if i not in _CACHE:
        _CACHE[i] = oracle.EnergyModel.from_problem(w.problems[i])
    model = _CACHE[i]
    exc, th = w.excitations[i], w.thetas[i]
    M = len(exc)
    idx = None if n_comp is None else list(range(M - n_comp, M))
    t0 = time.perf_counter()
    oracle.gradient_direct(model, synth.hf_bitstring(6), exc, th, idx)
    dt = time.perf_counter() - t0
    return dt, _work_fraction(M, idx)


def _work_fraction(M, idx):
    """Share of a full oracle E+g done, in gate applications (the oracle's unit of
    work): forward M gates + one H application (counted as one gate), then
    M - 1 - k gates and one generator per gradient component k."""
    full = M + 1 + sum(M - k for k in range(M))
    done = M + 1 + (sum(M - k for k in range(M)) if idx is None else sum(M - k for k in idx))
    return done / full


def cpu_baseline(n_geoms=None):
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    n = n_geoms or min(64, cores)
    ctx = mp.get_context("spawn")
    with ctx.Pool(processes=cores) as pool:
        pool.map(_noop, range(cores))  # start the workers (imports) outside the timing
        t0 = time.perf_counter()
        res = pool.map(_oracle_task, [(i, None) for i in range(n)])
        wall = time.perf_counter() - t0
    busy = sum(r[0] for r in res)
    used = min(cores, n)
    return {"value": n / wall, "unit": UNIT, "cores": used, "kind": "oracle",
            "sample": f"{n} of the 64 geometries, full energy+gradient each (oracle gradient_direct, "
                      f"Hamiltonian build untimed), one process per core; wall {wall:.1f} s, "
                      f"busy {busy:.1f} core-s"}


def _noop(_):
    import oracle  # noqa: F401
    import synth  # noqa: F401
    return 0


def run_reference(args, rank):
    if rank != 0:
        return
    import synth
    w = synth.config1()
    M = len(w.excitations[0])
    budget = 150.0
    per_step = max(0.05, budget / max(1, args.steps + args.warmup))
    # calibration (untimed): energy only, and the full energy + gradient
    dt_e, _ = _oracle_task((0, 0))
    dt_full, _ = _oracle_task((0, None))
    if dt_full <= per_step:
        n_comp = None
    else:
        # the c cheapest components (k = M-1, M-2, ...) cost c(c+1)/2 of the M(M+1)/2 units
        share = max(0.0, (per_step - dt_e) / max(dt_full - dt_e, 1e-9))
        n_comp = 0
        while n_comp < M and (n_comp + 1) * (n_comp + 2) / 2 <= share * M * (M + 1) / 2:
            n_comp += 1
    for s in range(args.warmup):
        _oracle_task((s % 4, n_comp))
    times, fracs = [], []
    t_start = time.perf_counter()
    for s in range(args.steps):
        dt, fr = _oracle_task((s % 4, n_comp))
        times.append(dt)
        fracs.append(fr)
    wall = time.perf_counter() - t_start
    tot = sum(times)
    value = sum(fracs) / tot
    sample = (f"per step one of geometries 0-3: energy + the {M if n_comp is None else n_comp} cheapest gradient "
              f"components of {M} (oracle gradient_direct), counted as full-evaluation equivalents by "
              f"gate applications; single process")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * tot / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": wall}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ ours
def reduce_max(value, world, device=None):
    """Max of a per-rank float over all ranks (identity for one rank)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def throughput(units_per_rank, world, steps, max_seconds):
    """Whole-job units per second: every rank did units_per_rank per step."""
    return units_per_rank * world * steps / max_seconds


def _timed(fn, steps, warmup, clocks_out=None):
    """Per-step CUDA-event times (ms) of fn() after warmup calls, flushing L2 between
    steps; SM clocks sampled during the timed steps are appended to clocks_out."""
    tm, clocks = _measure(fn, steps, warmup, 0)
    if clocks_out is not None:
        clocks_out.append(clocks)
    return tm["per_step"]


def run_large(args):
    """config3: 30 qubits, 10 electrons, 512 angles, energy + gradient per step.
    config2: 256 instances (14-20 qubits, 64-256 angles), one CUDA-graph replay
    of the gate-major batch per step (all energies and gradients)."""
    import numpy as np
    import torch

    import synth
    import paper_2311_01242_gb300 as vq
    from paper_2311_01242_gb300 import batch as vb

    torch.cuda.set_device(0)
    vq.load()
    steps, warmup = min(args.steps, 20), max(3, min(args.warmup, 5))
    clk = []
    t0 = time.perf_counter()
    if args.workload in ("puccd11", "puccd24"):
        if args.workload == "puccd11":
            w = synth.puccd_scan()
            pairs = synth.hcb_pairs_of(w.excitations[0])
            hams = [vq.Hamiltonian.from_problem_hcb(p) for p in w.problems]
            ans = [vq.Ansatz(11, 15, pairs, hcb=True)] * len(hams)
            thetas = np.stack(w.thetas)
            workload = "pUCCD hard-core boson form, 11 orbitals, 4 pairs, 28 angles, 64-geometry scan"
            units, unit = len(hams), "evals/s"
        else:
            w = synth.puccd_large()
            pairs = synth.hcb_pairs_of(w.excitations[0])
            hams = [vq.Hamiltonian.from_problem_hcb(w.problems[0])]
            ans = [vq.Ansatz(24, (1 << 12) - 1, pairs, hcb=True)]
            thetas = w.thetas[0][None, :]
            workload = "pUCCD hard-core boson form, 24 orbitals, 12 pairs (2.7M states), 144 angles"
            units, unit = 1, "evals/s"
        B = vq.Batch(hams, ans)
        theta = torch.as_tensor(thetas).cuda().contiguous()
        ws = vq.alloc_workspace(B.workspace_bytes(True))
        e_buf = torch.empty(len(hams), dtype=torch.float64, device="cuda")
        g_buf = torch.empty(len(hams), max(B.max_params, 1), dtype=torch.float64, device="cuda")
        t_create = time.perf_counter() - t0
        ms = _timed(lambda: B.energy_grad(theta, e_buf, g_buf, ws), steps, warmup, clk)
        flops = state_bytes = 0.0
        for h, a in zip(hams, ans):
            f, b = vq.work_estimate(h, a, True)
            flops += f
            state_bytes += b
        launches = None
    elif args.workload in ("config3", "q24", "hpsi30s", "q20"):
        hf = synth.hf_bitstring(10)
        if args.workload == "q20":
            ns, _ = synth.configs.config2_sizes()
            p, exc, th = synth.config2_instance(int(np.nonzero(ns == 20)[0][0]))
            drop, nq, hf = 1e-14, 20, synth.hf_bitstring(p.n_elec)
        elif args.workload == "config3":
            w = synth.config3()
            p, exc, th, drop, nq = w.problems[0], w.excitations[0], w.thetas[0], w.drop_tol, 30
        elif args.workload == "hpsi30s":
            # 4 alpha and 5 beta electrons: the 5-alpha/4-beta UCCSD pool with alpha and
            # beta qubits swapped (q -> q ^ 1), 256 of its excitations
            w = synth.config3()
            p, drop, nq = w.problems[0], w.drop_tol, 30
            rng = np.random.default_rng(30)
            pool = synth.uccsd_pool(30, 9)
            pool = np.where(pool >= 0, pool ^ 1, pool)
            exc = pool[rng.permutation(len(pool))[:256]]
            th = rng.normal(0.0, 0.05, size=256)
            hf = sum(1 << q for q in (0, 2, 4, 6, 1, 3, 5, 7, 9))
        else:
            rng = np.random.default_rng(24)
            p = synth.integrals.random_problem(rng, 12, 10, 6, label="q24")
            pool = synth.uccsd_pool(24, 10)
            exc = pool[rng.permutation(len(pool))[:256]]
            th, drop, nq = rng.normal(0.0, 0.05, size=256), 1e-14, 24
        H = vq.Hamiltonian.from_problem(p, drop)
        A = vq.Ansatz(nq, hf, exc)
        ws = vq.alloc_workspace(vq.workspace_bytes(H, A, vq.VQE_WS_GRAD))
        theta = torch.as_tensor(th).cuda()
        e_buf = torch.empty(1, dtype=torch.float64, device="cuda")
        g_buf = torch.empty(len(exc), dtype=torch.float64, device="cuda")
        t_create = time.perf_counter() - t0
        ms = _timed(lambda: vq.energy_grad(H, A, theta, workspace=ws, out=(e_buf, g_buf)), steps, warmup, clk)
        flops, state_bytes = vq.work_estimate(H, A, True)
        units, unit = 1, "evals/s"
        workload = {"config3": "30 qubits, 10 electrons, 512 UCCSD angles (9.0M sector amplitudes)",
                    "q24": "24 qubits, 10 electrons, 256 UCCSD angles (627k sector amplitudes)",
                    "hpsi30s": "30 qubits, 4 alpha + 5 beta electrons, 256 UCCSD angles (4.1M sector "
                               "amplitudes)",
                    "q20": f"20 qubits, {p.n_elec} electrons, {len(exc)} UCCSD angles (63,504 sector amplitudes)"
                    }[args.workload]
        launches = 2 * len(exc) + 8  # trig, init, gates, 4 H psi launches + energy sum, gates, gradient sums
    else:
        insts = [synth.config2_instance(j) for j in range(256)]
        hams = [vq.Hamiltonian.from_problem(p) for p, _, _ in insts]
        ans = [vq.Ansatz(p.n_qubits, synth.hf_bitstring(p.n_elec), e) for p, e, _ in insts]
        B = vq.Batch(hams, ans)
        theta = torch.zeros(256, B.max_params, dtype=torch.float64)
        for i, (_, _, t) in enumerate(insts):
            theta[i, :len(t)] = torch.as_tensor(t)
        theta = theta.cuda()
        vb.autotune(B, theta, reps=2)
        gb = vb.GraphBatch(B)
        gb(theta)
        t_create = time.perf_counter() - t0
        ms = _timed(lambda: gb(), steps, warmup, clk)
        flops = state_bytes = 0.0
        for h, a in zip(hams, ans):
            f, b = vq.work_estimate(h, a, True)
            flops += f
            state_bytes += b
        units, unit = 256, "instance-evals/s"
        workload = "256 instances, n in {14,16,18,20}, 64-256 UCCSD angles"
        launches = None
    ms_step = float(np.median(ms))
    achieved_tf = flops / (ms_step / 1e3) / 1e12
    line = {"metric": METRIC + f" [{args.workload}]", "value": units / (ms_step / 1e3), "unit": unit,
            "n_gpus": 1, "steps": steps, "warmup": warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload, "l2": "flushed between timed steps (512 MB write)",
                       "create_seconds": t_create},
            "roofline": {"bound": "alu", "achieved": achieved_tf, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": achieved_tf / FP64_PEAK_TFLOPS, "traffic": None,
                         "state_bytes_per_step": state_bytes,
                         "state_gbs": state_bytes / (ms_step / 1e3) / 1e9},
            "gpu_launches_per_step": launches, "clocks": clk[0] if clk else None}
    print(json.dumps(line), flush=True)


def run_noalloc(args):
    """noalloc16: one 16-qubit instance (8 electrons, the first such instance of the
    uneven batch), energy + gradient per step through vqe_energy_grad (caller's
    workspace) and through vqe_energy_grad_noalloc (the library's static scratch),
    the latter before and after the regular call has built the pair's string
    tables; CUDA-event timed, L2 flushed between steps."""
    import numpy as np
    import torch

    import synth
    import paper_2311_01242_gb300 as vq
    from paper_2311_01242_gb300.api import _ptr, _stream

    torch.cuda.set_device(0)
    lib = vq.load()
    steps, warmup = min(args.steps, 50), max(3, min(args.warmup, 5))
    ns, _ = synth.configs.config2_sizes()
    p, exc, th = synth.config2_instance(int(np.nonzero(ns == 16)[0][0]))
    theta = torch.as_tensor(th).cuda()
    e = torch.empty(1, dtype=torch.float64, device="cuda")
    g = torch.empty(len(th), dtype=torch.float64, device="cuda")

    def noalloc(H, A):
        rc = lib.vqe_energy_grad_noalloc(H.handle, A.handle, _ptr(theta), _ptr(e), _ptr(g), _stream())
        if rc != 0:
            raise RuntimeError(lib.vqe_last_error().decode(errors="replace"))

    clk = []
    # a fresh pair: no string or connectivity tables built yet
    H0 = vq.Hamiltonian.from_problem(p)
    A0 = vq.Ansatz(p.n_qubits, synth.hf_bitstring(p.n_elec), exc)
    ms_before = float(np.median(_timed(lambda: noalloc(H0, A0), steps, warmup, clk)))
    H = vq.Hamiltonian.from_problem(p)
    A = vq.Ansatz(p.n_qubits, synth.hf_bitstring(p.n_elec), exc)
    ws = vq.alloc_workspace(vq.workspace_bytes(H, A, vq.VQE_WS_GRAD))
    ms_reg = float(np.median(_timed(lambda: vq.energy_grad(H, A, theta, workspace=ws, out=(e, g)), steps, warmup,
                                    clk)))
    ms_after = float(np.median(_timed(lambda: noalloc(H, A), steps, warmup, clk)))
    line = {"metric": METRIC + " [noalloc16]", "value": 1e3 / ms_after, "unit": "evals/s", "n_gpus": 1,
            "steps": steps, "warmup": warmup, "ms_per_step": ms_after, "higher_is_better": True,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"16 qubits, {p.n_elec} electrons, {len(th)} UCCSD angles "
                                   f"({A.info()['sector_dim']} sector amplitudes), energy + gradient",
                       "l2": "flushed between timed steps (512 MB write)"},
            "energy_grad_ms": ms_reg, "noalloc_ms_tables_built": ms_after, "noalloc_ms_no_tables": ms_before,
            "ratio_tables_built": ms_after / ms_reg, "ratio_no_tables": ms_before / ms_reg,
            "clocks": clk[0] if clk else None}
    print(json.dumps(line), flush=True)


def measured_hbm_gbs():
    """Copy bandwidth measured on this GPU type (MEASURED_PEAKS.json), else the
    earlier GB300 measurement 6.8 TB/s; returns (GB/s, 'measured'|'fallback')."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def pool_profile_traffic(n_pairs):
    """DRAM bytes of one k_pool_grad launch over n_pairs, scaled from the committed
    ncu summary (5.33 GB for 137.4M pairs) if it was taken on the current source."""
    import re
    path = os.path.join(ROOT, "profiles", "k_pool_grad_adapt30.md")
    src = os.path.join(ROOT, "paper_2311_01242_gb300", "csrc", "vqe_pool.cu")
    try:
        text = open(path).read()
        with open(src, "rb") as f:
            cur = hashlib.sha256(f.read()).hexdigest()[:16]
    except OSError:
        return None
    sha = re.search(r"sha256 \(first 16 hex\): `([0-9a-f]+)`", text)
    if not sha or sha.group(1) != cur:
        return None
    return 5.33e9 * n_pairs / 137417280


def run_adapt(args):
    """ADAPT-VQE screening at 30 qubits: psi = U(theta)|HF> of the 512-angle
    state, lambda = H psi, and the gradient of every one of the 3,500 pool
    operators (one vqe_pool_gradients call per step); adapt24: the same at the
    24-qubit, 256-angle state with its full pool. The screening kernel's
    own time is the call's time minus that of vqe_energy on the same state
    (the same forward sweep and H psi launches), both CUDA-event timed."""
    import numpy as np
    import torch

    import synth
    import paper_2311_01242_gb300 as vq

    torch.cuda.set_device(0)
    vq.load()
    steps, warmup = min(args.steps, 10), max(3, min(args.warmup, 5))
    t0 = time.perf_counter()
    if args.workload == "adapt30":
        w = synth.config3()
        p, exc, th, drop, nq = w.problems[0], w.excitations[0], w.thetas[0], w.drop_tol, 30
        desc = "30 qubits, 10 electrons, 512-angle state, 3,500-operator UCCSD pool"
    else:
        rng = np.random.default_rng(24)
        p = synth.integrals.random_problem(rng, 12, 10, 6, label="q24")
        pool24 = synth.uccsd_pool(24, 10)
        exc = pool24[rng.permutation(len(pool24))[:256]]
        th, drop, nq = rng.normal(0.0, 0.05, size=256), 1e-14, 24
        desc = f"24 qubits, 10 electrons, 256-angle state, {len(pool24)}-operator UCCSD pool"
    pool = synth.uccsd_pool(nq, 10)
    if args.pool_ops is not None:
        pool = pool[:args.pool_ops]
        desc += f", first {len(pool)} operators screened"
    hf = synth.hf_bitstring(10)
    H = vq.Hamiltonian.from_problem(p, drop)
    A = vq.Ansatz(nq, hf, exc)
    P = vq.Ansatz(nq, hf, pool)
    t_create = time.perf_counter() - t0
    ws = vq.alloc_workspace(max(vq.pool_workspace_bytes(H, A, P), vq.workspace_bytes(H, A, vq.VQE_WS_ENERGY)))
    theta = torch.as_tensor(th).cuda()
    e_buf = torch.empty(1, dtype=torch.float64, device="cuda")
    g_buf = torch.empty(len(pool), dtype=torch.float64, device="cuda")
    clk = []
    ms_pool = _timed(lambda: vq.pool_gradients(H, A, P, theta, workspace=ws, out=(e_buf, g_buf)), steps, warmup, clk)
    ms_e = _timed(lambda: vq.energy(H, A, theta, workspace=ws), steps, warmup, clk)
    ms_step, ms_fwd_h = float(np.median(ms_pool)), float(np.median(ms_e))
    ms_screen = max(ms_step - ms_fwd_h, 1e-6)
    n_pairs = P.info()["n_pairs"]
    # per pair: its rank-pair record (8 B) and psi, lambda at both ranks (4 x 8 B);
    # the per-chunk partials (one double per 4,096 pairs) add under 0.01 %
    alg_bytes = n_pairs * 40
    achieved = alg_bytes / (ms_screen / 1e3) / 1e9
    peak, src = measured_hbm_gbs()
    line = {"metric": f"ADAPT pool screening passes/s [{args.workload}]", "value": 1e3 / ms_step, "unit": "screens/s",
            "n_gpus": 1, "steps": steps, "warmup": warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{desc} ({n_pairs} amplitude pairs)",
                       "l2": "flushed between timed steps (512 MB write)", "create_seconds": t_create,
                       "forward_and_hpsi_ms": ms_fwd_h, "screening_kernel_ms": ms_screen},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": pool_profile_traffic(n_pairs), "peak_source": src,
                         "kernel": "k_pool_grad + k_pool_finalize"},
            "gpu_launches_per_step": 2 * len(exc) + 8, "clocks": clk[0] if clk else None,
            "clocks_energy_only": clk[1] if len(clk) > 1 else None}
    print(json.dumps(line), flush=True)


def run_adapt_loop(args):
    """The ADAPT-VQE loop (screen the 117-operator UCCSD pool, append the largest
    gradient, re-optimise every angle with BFGS) on the first geometry of the
    12-qubit scan from the empty ansatz until the pool gradient norm is below
    1e-3 or 60 operators were added; wall-clock time, with the exact sector
    ground energy (Lanczos with the library's H psi) for reference."""
    import numpy as np
    import torch

    import synth
    import paper_2311_01242_gb300 as vq
    from paper_2311_01242_gb300 import adapt, warmstart

    torch.cuda.set_device(0)
    vq.load()
    w = synth.config1(1)
    p = w.problems[0]
    hf = synth.hf_bitstring(6)
    H = vq.Hamiltonian.from_problem(p)
    pool = synth.uccsd_pool(12, 6)
    adapt.adapt_vqe(H, 12, hf, pool, grad_tol=1e-1, max_ops=2)  # warm-up (library load, graph caches)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = adapt.adapt_vqe(H, 12, hf, pool, grad_tol=1e-3, max_ops=60)
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    e0 = warmstart.lanczos_ground(H, vq.Ansatz(12, hf, pool), 12, 6)
    e_hf = r.history[0][0]
    stop = ("pool gradient norm below 1e-3" if r.history[-1][1] < 1e-3 else
            f"{len(r.chosen)} operators (the cap) reached")
    line = {"metric": "ADAPT-VQE loop wall time (to a pool gradient norm below 1e-3, at most 60 operators) "
                      "[adapt12]", "value": secs,
            "unit": "s", "n_gpus": 1, "steps": 1, "warmup": 1, "ms_per_step": secs * 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "12 qubits, 6 electrons, scan geometry r = 0.8, 117-operator UCCSD pool, "
                                   "empty starting ansatz",
                       "operators_added": len(r.chosen), "distinct_operators": len(set(r.chosen)),
                       "energy_grad_evaluations": r.evaluations, "screening_calls": len(r.history),
                       "energy": r.energy, "hf_energy": e_hf, "exact_sector_energy": e0,
                       "error_ha": r.energy - e0, "final_pool_grad_norm": r.history[-1][1], "stopped_by": stop}}
    print(json.dumps(line), flush=True)


def warmstart_summary(args):
    """16 qubits, 8 electrons, 512-point scan r in [0.7, 4.0], 360 UCCSD angles:
    plain VQE with continuation on every 4th point trains the network; at
    held-out points, BFGS runs from the HF start, from the nearest earlier
    training point's angles (continuation), and from the network prediction
    (HF when the prediction's energy is not below HF). Per arm: evaluations and
    seconds until E <= E_exact + 1 mHa (exact: GPU Lanczos in the sector), or
    the best converged energy + 1 mHa where no start reaches that; a run that
    never reaches the target counts with every evaluation and second it spent."""
    import numpy as np
    import torch

    import synth
    import paper_2311_01242_gb300 as vq
    from paper_2311_01242_gb300 import warmstart as ws

    torch.cuda.set_device(0)
    vq.load()
    t_all = time.perf_counter()
    w = synth.config4()
    scan = w.scan
    rs = scan.rs
    n, ne = 2 * scan.n_spatial, scan.n_elec
    A = vq.Ansatz(n, synth.hf_bitstring(ne), w.excitations[0])
    train = list(range(0, len(rs), 4))
    rest = [i for i in range(len(rs)) if i % 4 != 0]
    held = rest[::max(1, len(rest) // args.held_out)][:args.held_out]
    t0 = time.perf_counter()
    geoms = [ws.Geometry(scan.at(rs[i]), rs[i], A, graph=True) for i in train]
    t_create = time.perf_counter() - t0
    t0 = time.perf_counter()
    thetas, energies, evals = ws.training_set(geoms, gtol=1e-6)
    t_data = time.perf_counter() - t0
    t0 = time.perf_counter()
    model = ws.WarmStart(geoms[0].features.size, A.n_params, hidden=256, seed=0)
    hist = model.fit(np.stack([g.features for g in geoms]), thetas, steps=3000, lr=1e-3)
    torch.cuda.synchronize()
    t_fit = time.perf_counter() - t0
    arms = {"hf": [], "continuation": [], "mlp": []}
    fallbacks, reached_exact = 0, 0
    for i in held:
        g = ws.Geometry(scan.at(rs[i]), rs[i], A, graph=True)
        e0 = ws.lanczos_ground(g.H, A, n, ne)
        prev = max(j for j, ti in enumerate(train) if ti < i)
        tp = time.perf_counter()
        pred = model.predict(g.features[None, :])[0]
        e_pred = float(vq.energy(g.H, A, pred))
        e_hf = float(vq.energy(g.H, A, np.zeros(A.n_params)))
        start = pred
        if not e_pred < e_hf:
            start = np.zeros(A.n_params)
            fallbacks += 1
        t_pred = time.perf_counter() - tp
        res = ws.compare_starts(g, {"hf": np.zeros(A.n_params), "continuation": thetas[prev], "mlp": start}, e0,
                                gtol=1e-6)
        reached_exact += int(res["reached_exact"])
        for name in arms:
            r = res[name]
            # the network arm also pays its prediction: two energy evaluations and the forward pass
            extra_e, extra_t = (2, t_pred) if name == "mlp" else (0, 0.0)
            hit = r["evals"] is not None
            arms[name].append((hit, (r["evals"] if hit else r["evals_total"]) + extra_e,
                               (r["seconds"] if hit else r["seconds_total"]) + extra_t))
    summary = {}
    for name, v in arms.items():
        ev = [e for _, e, _ in v]
        sec = [s for _, _, s in v]
        summary[name] = {"mean_evals": float(np.mean(ev)), "median_evals": float(np.median(ev)),
                         "mean_seconds": float(np.mean(sec)), "reached": int(sum(h for h, _, _ in v)),
                         "points": len(v)}
    return {"metric": "time to 1 mHa vs plain (learned warm start)", "value": summary["mlp"]["mean_seconds"],
            "unit": "s", "higher_is_better": False, "dtype": "f64 (VQE), bf16/f32 (network)",
            "workload": "16 qubits, 8 electrons, 512-point scan r in [0.7,4.0], 360 UCCSD angles",
            "train_points": len(train), "held_out_points": len(held),
            "target": "E_exact + 1 mHa (or best converged + 1 mHa where no start reaches it)",
            "averaging": "every held-out point in every arm; a run that never reaches the target counts "
                         "with all its evaluations and its whole wall time",
            "arms": summary, "fallbacks_to_hf": fallbacks, "held_out_reaching_exact": reached_exact,
            "training": {"vqe_seconds": t_data, "vqe_evals": int(np.sum(evals)), "fit_seconds": t_fit,
                         "fit_steps": 3000, "final_loss": float(hist[-1]), "create_seconds": t_create},
            "wall_s": time.perf_counter() - t_all}


def run_warmstart(args):
    s = warmstart_summary(args)
    line = {"metric": s["metric"], "value": s["value"], "unit": "s", "higher_is_better": False, "n_gpus": 1,
            "dtype": s["dtype"], "data": "synthetic",
            "config": {"workload": s["workload"], "train_points": s["train_points"],
                       "held_out_points": s["held_out_points"], "target": s["target"]},
            "arms": s["arms"], "fallbacks_to_hf": s["fallbacks_to_hf"],
            "held_out_reaching_exact": s["held_out_reaching_exact"], "training": s["training"]}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ per-config entries of the default line
def _measure(fn, steps, warmup, gpu_index):
    """CUDA-event time of fn() per step on torch's current stream (the library
    launches there), after max(3, warmup) untimed calls, with a 512 MB write
    (> the 129 MB L2) before each timed step; SM clocks are sampled during the
    timed region only. Returns (timing dict, clocks dict)."""
    import torch
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    warm = max(3, warmup)
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    sampler = ClockSampler(gpu_index)
    sampler.start()
    t0 = time.time()
    for i in range(steps):
        flush.fill_(float(i))
        starts[i].record(stream)
        fn()
        ends[i].record(stream)
    torch.cuda.synchronize()
    t1 = time.time()
    clocks = sampler.stop(t0, t1)
    per = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    return ({"ms_per_step": sum(per) / steps, "ms_median": statistics.median(per), "ms_min": min(per),
             "steps": steps, "warmup": warm, "per_step": per}, clocks)


def _e2e(call, steps, h2d, d2h, unit, units_per_call):
    """Wall-clock rate of a prepared host-buffer C-ABI call (copies from pinned
    host memory, launches, copies back, stream synchronised inside each call)."""
    for _ in range(3):
        call()
    t0 = time.perf_counter()
    for _ in range(steps):
        call()
    dt = time.perf_counter() - t0
    return {"value": units_per_call * steps / dt, "unit": unit, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "steps": steps, "ms_per_call": 1e3 * dt / steps}


def _profile_field(path, src_files, field):
    """A numeric field of a committed ncu summary, if the summary names the
    current sha256 of the kernel sources it was taken on; else None."""
    import re
    try:
        text = open(os.path.join(ROOT, "profiles", path)).read()
        h = hashlib.sha256()
        for f in src_files:
            with open(os.path.join(ROOT, "paper_2311_01242_gb300", "csrc", f), "rb") as fh:
                h.update(fh.read())
    except OSError:
        return None
    sha = re.search(r"sources sha256 \(first 16 hex\): `([0-9a-f]+)`", text)
    m = re.search(re.escape(field) + r": ([0-9.eE+-]+)", text)
    if not sha or not m or sha.group(1) != h.hexdigest()[:16]:
        return None
    return float(m.group(1))


def _oracle_rows_and_gate(xs, zs, cs, n, n_alpha, n_beta, exc, n_rows, gate_n=None, seed=0):
    """Seconds per output row of H psi (oracle.pauli_sum_row over every term,
    averaged over n_rows sampled sector rows) and per gate pass
    (oracle.apply_gate on a full 2^gate_n vector); the oracle as it stands."""
    import numpy as np
    import oracle
    sec = oracle.sector_basis(n, n_alpha, n_beta)
    rng = np.random.default_rng(seed)
    vals = rng.normal(size=len(sec))

    def amp(idx):
        pos = np.minimum(np.searchsorted(sec, idx), len(sec) - 1)
        return np.where(sec[pos] == idx, vals[pos], 0.0)

    rows = rng.choice(len(sec), size=min(n_rows, len(sec)), replace=False)
    t0 = time.perf_counter()
    for r in rows:
        oracle.pauli_sum_row(xs, zs, cs, int(sec[r]), amp)
    t_row = (time.perf_counter() - t0) / len(rows)
    gn = gate_n or n
    psi = rng.normal(size=1 << gn) + 0j
    t0 = time.perf_counter()
    oracle.apply_gate(psi, exc, 0.1)
    t_gate = time.perf_counter() - t0
    return t_row, t_gate, len(sec)


def _adjoint_seconds(t_row, t_gate, D, M):
    """One energy + adjoint gradient from the oracle's primitives: a forward
    sweep (M gate passes), H psi (D rows) and a reverse sweep that un-applies
    every gate to two vectors and applies one generator (counted as 3 gate
    passes per gate)."""
    return M * t_gate + D * t_row + 3 * M * t_gate


def cpu_baseline_config3(w, exc):
    import oracle
    import synth
    p = w.problems[0]
    t0 = time.perf_counter()
    xs, zs, cs = oracle.jordan_wigner(p, w.drop_tol)
    t_jw = time.perf_counter() - t0
    # a 30-qubit oracle gate pass needs ~60 GB of host arrays; its cost is linear in
    # 2^n, so a 24-qubit pass of a double excitation is timed and scaled by 2^6
    t_row, t_gate24, D = _oracle_rows_and_gate(xs, zs, cs, 30, 5, 5, [0, 1, 20, 21], 60, gate_n=24)
    t_gate = t_gate24 * 64
    secs = _adjoint_seconds(t_row, t_gate, D, len(exc))
    return {"value": 1.0 / secs, "unit": "evals/s", "cores": 1, "kind": "oracle", "extrapolated": True,
            "sample": f"oracle.pauli_sum_row on 60 sampled rows of the 30-qubit sector ({len(xs)} terms; "
                      f"{t_row * 1e3:.2f} ms/row) and one oracle.apply_gate pass over a full 2^24 vector "
                      f"({t_gate24:.2f} s, x64 for 2^30), extrapolated to 4 x 512 gate passes + {D} rows "
                      f"= {secs:.3g} s per energy+gradient; single process; the oracle's Jordan-Wigner "
                      f"mapping ({t_jw:.1f} s) untimed"}


def cpu_baseline_config2(insts, ns_all, ms_all):
    import numpy as np
    import oracle
    per_n = {}
    total = 0.0
    for n in (14, 16, 18, 20):
        j = int(np.nonzero(ns_all == n)[0][0])
        p, exc, _ = insts[j]
        xs, zs, cs = oracle.jordan_wigner(p)
        na, nb = (p.n_elec + 1) // 2, p.n_elec // 2
        t_row, t_gate, D = _oracle_rows_and_gate(xs, zs, cs, n, na, nb, exc[0], 40)
        per_n[n] = (t_row, t_gate, D)
    for i in range(len(insts)):
        n = int(ns_all[i])
        t_row, t_gate, D = per_n[n]
        total += _adjoint_seconds(t_row, t_gate, D, len(insts[i][1]))
    return {"value": len(insts) / total, "unit": "instance-evals/s", "cores": 1, "kind": "oracle",
            "extrapolated": True,
            "sample": "per qubit count (one instance each of 14/16/18/20 qubits): oracle.pauli_sum_row on 40 "
                      "sampled sector rows and one oracle.apply_gate pass over the full 2^n vector ("
                      + ", ".join(f"{n}q {v[0] * 1e3:.2f} ms/row, {v[1] * 1e3:.1f} ms/gate" for n, v in per_n.items())
                      + f"), extrapolated per instance to 4M gate passes + D rows and summed over the 256 "
                        f"instances = {total:.3g} s per batch; single process"}


def entry_config3(args, gpu_index):
    """30 qubits (config 3): one energy + adjoint gradient per step."""
    import numpy as np
    import torch

    import synth
    import paper_2311_01242_gb300 as vq

    steps, warmup = min(args.steps, 20), max(3, min(args.warmup, 5))
    w = synth.config3()
    p, exc, th = w.problems[0], w.excitations[0], w.thetas[0]
    t0 = time.perf_counter()
    H = vq.Hamiltonian.from_problem(p, w.drop_tol)
    A = vq.Ansatz(30, synth.hf_bitstring(10), exc)
    ws = vq.alloc_workspace(vq.workspace_bytes(H, A, vq.VQE_WS_GRAD))
    t_create = time.perf_counter() - t0
    theta = torch.as_tensor(th).cuda()
    e_buf = torch.empty(1, dtype=torch.float64, device="cuda")
    g_buf = torch.empty(len(exc), dtype=torch.float64, device="cuda")
    tm, clocks = _measure(lambda: vq.energy_grad(H, A, theta, workspace=ws, out=(e_buf, g_buf)), steps, warmup,
                          gpu_index)
    tm.pop("per_step")
    e_real = float(e_buf[0])
    flops, state_bytes = vq.work_estimate(H, A, True)
    counts = vq.work_counts(H, A)
    ms = tm["ms_per_step"]
    # A/B: the reverse sweep un-applying each gate to psi instead of reading the kept
    # forward outputs, and that path with each sweep as one persistent launch
    old = vq.set_flags(vq.VQE_FLAG_NO_PHI_STORE)
    try:
        e_u = torch.empty(1, dtype=torch.float64, device="cuda")
        g_u = torch.empty(len(exc), dtype=torch.float64, device="cuda")
        tu, clocks_u = _measure(lambda: vq.energy_grad(H, A, theta, workspace=ws, out=(e_u, g_u)), min(steps, 5), 3,
                                gpu_index)
    finally:
        vq.set_flags(old)
    old = vq.set_flags(vq.VQE_FLAG_PERSISTENT_SWEEPS)
    try:
        e_l = torch.empty(1, dtype=torch.float64, device="cuda")
        g_l = torch.empty(len(exc), dtype=torch.float64, device="cuda")
        tl, clocks_l = _measure(lambda: vq.energy_grad(H, A, theta, workspace=ws, out=(e_l, g_l)), min(steps, 5), 3,
                                gpu_index)
        same_bits = bool(torch.equal(e_l, e_u) and torch.equal(g_l, g_u))
    finally:
        vq.set_flags(old)
    # complex128 amplitudes and full complex coefficients (the same kernels' complex form)
    old = vq.set_flags(vq.VQE_FLAG_FORCE_COMPLEX)
    try:
        wsc = vq.alloc_workspace(vq.workspace_bytes(H, A, vq.VQE_WS_GRAD | vq.VQE_WS_COMPLEX))
        e_c = torch.empty(1, dtype=torch.float64, device="cuda")
        g_c = torch.empty(len(exc), dtype=torch.float64, device="cuda")
        tc, clocks_c = _measure(lambda: vq.energy_grad(H, A, theta, workspace=wsc, out=(e_c, g_c)), min(steps, 5),
                                3, gpu_index)
        tc.pop("per_step")
        d_e = abs(float(e_c[0]) - e_real)
        d_g = float((g_c - g_buf).abs().max())
        del wsc
    finally:
        vq.set_flags(old)
    # end to end through the host-buffer C entry point (a one-instance batch runs
    # the single-instance launches)
    B = vq.Batch([H], [A])
    th_h = torch.as_tensor(th, dtype=torch.float64).reshape(1, -1).pin_memory()
    e_h = torch.empty(1, dtype=torch.float64).pin_memory()
    g_h = torch.empty(1, len(exc), dtype=torch.float64).pin_memory()
    wsh = vq.alloc_workspace(B.host_workspace_bytes(True))
    th_np, e_np, g_np = th_h.numpy(), e_h.numpy(), g_h.numpy()
    e2e = _e2e(B.host_call(th_np, e_np, g_np, wsh), min(steps, 10), th_np.nbytes, e_np.nbytes + g_np.nbytes,
               "evals/s", 1)
    assert abs(float(e_np[0]) - e_real) <= 1e-12, "host-buffer and device calls disagree"
    del wsh, B
    peak_hbm, hbm_src = measured_hbm_gbs()
    # DRAM bytes of one whole evaluation (every kernel, warm L2 as in the timed steps),
    # else those of the H psi launch alone (cold L2)
    hpsi_dram = _profile_field("dram_config3_eval.md", RESIDENT_SRC + ["vqe_phi.cu"], "dram_bytes_per_eval")
    if hpsi_dram is None:
        hpsi_dram = _profile_field("k_hpsi_str_config3.md", RESIDENT_SRC, "dram_bytes_per_launch")
    achieved = flops / (ms / 1e3) / 1e12
    roof = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP64_PEAK_TFLOPS, "kernel": "k_hpsi_str (wide block form) + k_gate_fwd/k_gate_adj",
            "traffic": hpsi_dram,
            "dram_bytes_per_step": hpsi_dram,
            "hbm_gbs": None if hpsi_dram is None else hpsi_dram / (ms / 1e3) / 1e9,
            "hbm_frac": None if hpsi_dram is None else hpsi_dram / (ms / 1e3) / 1e9 / peak_hbm,
            "hbm_peak": peak_hbm, "hbm_peak_source": hbm_src,
            "state_bytes_per_step": state_bytes, "state_gbs": state_bytes / (ms / 1e3) / 1e9,
            "fp64_flops_per_step": flops, "hpsi_entries": counts["n_entries"], "amplitude_pairs": counts["n_pairs"],
            "binding": "FP64 pipe and instruction issue of the string-driven H psi (sector-compressed psi and "
                       "lambda, 72 MB each, stay in L2; DRAM carries the list entries and tables)"}
    cpu = cpu_baseline_config3(w, exc)
    return {"workload": "30 qubits, 10 electrons, 512 UCCSD angles (9.0M sector amplitudes), energy + adjoint "
                        "gradient", "metric": "energy+adjoint-grad evals/s", "value": 1e3 / ms, "unit": "evals/s",
            **tm, "dtype": "f64 (real amplitudes)", "create_seconds": t_create, "clocks": clocks, "roofline": roof,
            "e2e": e2e, "cpu_baseline": cpu,
            "complex128": {"value": 1e3 / tc["ms_per_step"], "unit": "evals/s", **tc, "clocks": clocks_c,
                           "abs_diff_energy_vs_real": d_e, "max_abs_diff_grad_vs_real": d_g},
            "reverse_sweep": {"kept_forward_outputs_ms_per_step": ms, "unapplying_ms_per_step": tu["ms_per_step"],
                              "energy_same_bits": bool(torch.equal(e_u, e_buf)),
                              "max_abs_diff_grad": float((g_u - g_buf).abs().max()), "clocks_unapplying": clocks_u},
            "gate_sweeps": {"one_launch_per_gate_ms_per_step": tu["ms_per_step"],
                            "persistent_ms_per_step": tl["ms_per_step"], "same_bits": same_bits,
                            "clocks_persistent": clocks_l},
            "l2": "flushed between timed steps (512 MB write)"}


def entry_q20(args, gpu_index):
    """One 20-qubit instance (the first of config 2's 20-qubit instances): one energy +
    adjoint gradient per step; HBM bytes per evaluation from the committed launch list
    of one evaluation (every kernel, warm L2 as in the timed steps)."""
    import numpy as np
    import torch

    import synth
    import paper_2311_01242_gb300 as vq

    steps, warmup = min(args.steps, 20), max(3, min(args.warmup, 5))
    ns, _ = synth.configs.config2_sizes()
    p, exc, th = synth.config2_instance(int(np.nonzero(ns == 20)[0][0]))
    H = vq.Hamiltonian.from_problem(p)
    A = vq.Ansatz(20, synth.hf_bitstring(p.n_elec), exc)
    ws = vq.alloc_workspace(vq.workspace_bytes(H, A, vq.VQE_WS_GRAD))
    theta = torch.as_tensor(th).cuda()
    e_buf = torch.empty(1, dtype=torch.float64, device="cuda")
    g_buf = torch.empty(len(exc), dtype=torch.float64, device="cuda")
    tm, clocks = _measure(lambda: vq.energy_grad(H, A, theta, workspace=ws, out=(e_buf, g_buf)), steps, warmup,
                          gpu_index)
    tm.pop("per_step")
    ms = tm["ms_per_step"]
    flops, state_bytes = vq.work_estimate(H, A, True)
    peak_hbm, hbm_src = measured_hbm_gbs()
    dram = _profile_field("dram_q20_eval.md", RESIDENT_SRC, "dram_bytes_per_eval")
    achieved = flops / (ms / 1e3) / 1e12
    roof = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP64_PEAK_TFLOPS, "kernel": "k_hpsi_str (warp form) + k_gate_fwd/k_gate_adj",
            "traffic": dram, "dram_bytes_per_step": dram,
            "hbm_gbs": None if dram is None else dram / (ms / 1e3) / 1e9,
            "hbm_frac": None if dram is None else dram / (ms / 1e3) / 1e9 / peak_hbm,
            "hbm_peak": peak_hbm, "hbm_peak_source": hbm_src,
            "state_bytes_per_step": state_bytes, "state_gbs": state_bytes / (ms / 1e3) / 1e9,
            "fp64_flops_per_step": flops}
    return {"workload": f"20 qubits, {p.n_elec} electrons, {len(exc)} UCCSD angles (63,504 sector amplitudes), "
                        "energy + adjoint gradient", "metric": "energy+adjoint-grad evals/s", "value": 1e3 / ms,
            "unit": "evals/s", **tm, "dtype": "f64 (real amplitudes)", "clocks": clocks, "roofline": roof,
            "l2": "flushed between timed steps (512 MB write)"}


def entry_config2(args, gpu_index):
    """256 uneven instances (config 2): one CUDA-graph replay of the batch per step."""
    import numpy as np
    import torch

    import synth
    import paper_2311_01242_gb300 as vq
    from paper_2311_01242_gb300 import batch as vb

    steps, warmup = min(args.steps, 20), max(3, min(args.warmup, 5))
    t0 = time.perf_counter()
    insts = [synth.config2_instance(j) for j in range(256)]
    hams = [vq.Hamiltonian.from_problem(p) for p, _, _ in insts]
    ans = [vq.Ansatz(p.n_qubits, synth.hf_bitstring(p.n_elec), e) for p, e, _ in insts]
    B = vq.Batch(hams, ans)
    theta = torch.zeros(256, B.max_params, dtype=torch.float64)
    for i, (_, _, t) in enumerate(insts):
        theta[i, :len(t)] = torch.as_tensor(t)
    theta_d = theta.cuda()
    choice, timings = vb.autotune(B, theta_d, reps=2)
    gb = vb.GraphBatch(B)
    gb(theta_d)
    t_create = time.perf_counter() - t0
    tm, clocks = _measure(lambda: gb(), steps, warmup, gpu_index)
    tm.pop("per_step")
    ms = tm["ms_per_step"]
    flops = state_bytes = 0.0
    n_entries = n_pairs = 0
    for h, a in zip(hams, ans):
        f, b = vq.work_estimate(h, a, True)
        c = vq.work_counts(h, a)
        flops += f
        state_bytes += b
        n_entries += c["n_entries"]
        n_pairs += c["n_pairs"]
    th_h = theta.clone().pin_memory()
    e_h = torch.empty(256, dtype=torch.float64).pin_memory()
    g_h = torch.empty(256, B.max_params, dtype=torch.float64).pin_memory()
    wsh = vq.alloc_workspace(B.host_workspace_bytes(True))
    th_np, e_np, g_np = th_h.numpy(), e_h.numpy(), g_h.numpy()
    e2e = _e2e(B.host_call(th_np, e_np, g_np, wsh), min(steps, 10), th_np.nbytes, e_np.nbytes + g_np.nbytes,
               "instance-evals/s", 256)
    e_dev, _ = gb()
    assert np.abs(e_np - e_dev.cpu().numpy()).max() <= 1e-12, "host-buffer and graph replay disagree"
    del wsh
    peak_hbm, hbm_src = measured_hbm_gbs()
    dram = _profile_field("k_batch_config2.md", ["vqe_batch.cu", "vqe_device.cuh"], "dram_bytes_per_launch")
    achieved = flops / (ms / 1e3) / 1e12
    roof = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP64_PEAK_TFLOPS, "kernel": "batched kernels of one graph replay",
            "traffic": dram, "dram_bytes_per_step": dram,
            "hbm_gbs": None if dram is None else dram / (ms / 1e3) / 1e9,
            "hbm_frac": None if dram is None else dram / (ms / 1e3) / 1e9 / peak_hbm,
            "hbm_peak": peak_hbm, "hbm_peak_source": hbm_src,
            "state_bytes_per_step": state_bytes, "state_gbs": state_bytes / (ms / 1e3) / 1e9,
            "fp64_flops_per_step": flops, "hpsi_entries": n_entries, "amplitude_pairs": n_pairs}
    ns_all, ms_all = synth.configs.config2_sizes()
    cpu = cpu_baseline_config2(insts, ns_all, ms_all)
    return {"workload": "256 instances, n in {14,16,18,20}, n/2 electrons, 64-256 UCCSD angles each, energy + "
                        "adjoint gradient of every instance per step (one CUDA-graph replay)",
            "metric": "energy+adjoint-grad instance-evals/s", "value": 256e3 / ms, "unit": "instance-evals/s",
            **tm, "dtype": "f64 (real amplitudes)", "create_seconds": t_create, "autotune": {"choice": choice},
            "clocks": clocks, "roofline": roof, "e2e": e2e, "cpu_baseline": cpu,
            "l2": "flushed between timed steps (512 MB write)"}


def entry_config1_complex(B, theta, n_inst, M, steps, warmup, gpu_index):
    """The 12-qubit scan with complex128 amplitudes (VQE_FLAG_FORCE_COMPLEX)."""
    import torch
    import paper_2311_01242_gb300 as vq
    old = vq.set_flags(vq.VQE_FLAG_FORCE_COMPLEX)
    try:
        e = torch.empty(n_inst, dtype=torch.float64, device="cuda")
        g = torch.empty(n_inst, M, dtype=torch.float64, device="cuda")
        ws = vq.alloc_workspace(B.workspace_bytes(True))
        tm, clocks = _measure(lambda: B.energy_grad(theta, e, g, ws), steps, warmup, gpu_index)
        tm.pop("per_step")
    finally:
        vq.set_flags(old)
    return {"workload": WORKLOAD + " (complex128 amplitudes and coefficients)", "value": n_inst * 1e3 / tm["ms_per_step"],
            "unit": UNIT, **tm, "clocks": clocks, "energies": e, "kernel": "k_resident (complex, one CTA per instance)"}


def per_config(args, gpu_index, extra=None):
    """The configurations besides the headline: each entry is timed on its own
    (CUDA events, L2 flushed, clocks sampled), with its roofline, an end-to-end
    figure through the host-buffer C entry point and the oracle's rate."""
    out = dict(extra or {})
    for name, fn in (("config3", lambda: entry_config3(args, gpu_index)),
                     ("config2", lambda: entry_config2(args, gpu_index)),
                     ("q20", lambda: entry_q20(args, gpu_index)),
                     ("warmstart", lambda: warmstart_summary(args))):
        if name in args.skip:
            continue
        t0 = time.perf_counter()
        try:
            out[name] = fn()
        except Exception as ex:  # keep the headline line even if one entry fails
            out[name] = {"error": f"{type(ex).__name__}: {ex}"}
        out[name]["entry_wall_s"] = time.perf_counter() - t0
        import torch
        torch.cuda.empty_cache()
    return out


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if args.workload == "warmstart":
        if rank == 0:
            run_warmstart(args)
        return
    if args.workload in ("config3", "config2", "q24", "puccd11", "puccd24", "hpsi30s", "q20"):
        if rank == 0:
            run_large(args)
        return
    if args.workload in ("adapt30", "adapt24"):
        if rank == 0:
            run_adapt(args)
        return
    if args.workload == "adapt12":
        if rank == 0:
            run_adapt_loop(args)
        return
    if args.workload == "noalloc16":
        if rank == 0:
            run_noalloc(args)
        return

    import numpy as np
    import torch
    import torch.distributed as dist

    torch.cuda.set_device(local_rank)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    def barrier():
        if world > 1:
            dist.barrier()

    import synth
    import paper_2311_01242_gb300 as vq

    vq.load()
    w = synth.config1()
    n_inst = len(w.problems)
    hams = [vq.Hamiltonian.from_problem(p) for p in w.problems]
    A = vq.Ansatz(12, synth.hf_bitstring(6), w.excitations[0])
    B = vq.Batch(hams, [A] * n_inst)
    M = B.max_params
    theta = torch.as_tensor(np.stack(w.thetas)).cuda().contiguous()
    energies = torch.empty(n_inst, dtype=torch.float64, device="cuda")
    grads = torch.empty(n_inst, M, dtype=torch.float64, device="cuda")
    ws = vq.alloc_workspace(B.workspace_bytes(True))
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    flops_per_eval = [vq.work_estimate(h, A, True)[0] for h in hams]
    flops_per_launch = float(sum(flops_per_eval))

    def step():
        B.energy_grad(theta, energies, grads, ws, stream)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()

    K = args.steps
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    sampler = ClockSampler(gpu_index_for(local_rank))
    sampler.start()
    barrier()
    torch.cuda.synchronize()
    t_wall0 = time.perf_counter()
    for i in range(K):
        flush.fill_(float(i))  # write 512 MB (> 129 MB L2) between timed launches
        starts[i].record(stream)
        step()
        ends[i].record(stream)
    torch.cuda.synchronize()
    barrier()
    t_wall = time.perf_counter() - t_wall0
    clocks = sampler.stop()
    per = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    dev_ms = reduce_max(sum(per), world, "cuda")
    ms_per_step = dev_ms / K
    value = throughput(n_inst, world, K, dev_ms / 1000.0)

    # e2e through the host-buffer C entry point (copies + sync inside the timed region)
    K2 = args.e2e_steps or min(K, 500)
    th_h = torch.empty(n_inst, M, dtype=torch.float64).pin_memory()
    th_h.copy_(theta.cpu())
    e_h = torch.empty(n_inst, dtype=torch.float64).pin_memory()
    g_h = torch.empty(n_inst, M, dtype=torch.float64).pin_memory()
    wsh = vq.alloc_workspace(B.host_workspace_bytes(True))
    th_np, e_np, g_np = th_h.numpy(), e_h.numpy(), g_h.numpy()
    call = B.host_call(th_np, e_np, g_np, wsh, stream)  # host arrays marshalled once, rewritten in place
    for _ in range(3):
        call()
    barrier()
    t0 = time.perf_counter()
    for _ in range(K2):
        call()
    t_e2e = reduce_max(time.perf_counter() - t0, world, "cuda")
    e2e_value = throughput(n_inst, world, K2, t_e2e)
    assert np.allclose(e_np, energies.cpu().numpy(), rtol=0, atol=0), "host and device entries disagree"

    achieved = flops_per_launch / (ms_per_step / 1000.0) / 1e12
    dram = _profile_field("k_resident_config1.md", RESIDENT_SRC, "dram_bytes_per_launch")
    units = _profile_field("k_resident_config1.md", RESIDENT_SRC, "units_per_launch")
    traffic = None if dram is None or not units else dram * n_inst / units
    probe = vq.probe_fp64()  # untimed: confirms the per-SM FP64 rate behind the peak
    # the resource the kernel actually uses: 64-bit integer multiplies (fixed-point
    # sweeps: 2 per lane forward, 3 per lane in reverse, two lanes per pair; H psi:
    # one per connected entry) against the probed __umul64hi rate, and issue slots
    wc = vq.work_counts(hams[0], A)
    muls = n_inst * (10 * wc["n_pairs"] + wc["n_entries"])
    mul_peak = INT_MUL64_PER_CLK_SM * N_SMS * SM_MAX_MHZ * 1e6
    issue_pct = _profile_field("k_resident_config1.md", RESIDENT_SRC, "issue_active_pct")
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
        "warmup": max(3, args.warmup), "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64 + i64 (fixed-point gate sweeps and H psi)",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "instances_per_gpu": n_inst, "qubits": 12, "params": M,
                   "l2": "flushed between timed launches (512 MB write)", "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved / FP64_PEAK_TFLOPS, "traffic": traffic,
                     "kernel": "k_resident (real amplitudes, cluster of two CTAs per instance, one launch "
                               "per step)",
                     "peak_source": "derived: 2 DFMA/clk/SM (probe) x 152 SMs x 2070 MHz x 2",
                     "fp64_flops_per_launch": flops_per_launch,
                     "note": "achieved counts the method's arithmetic as FP64-equivalent flops (vqe_work_estimate); "
                             "the gate sweeps and H psi run it on the integer pipe in 64-bit fixed point, the energy sum in FP64",
                     "probe": {"dfma_per_clock_per_sm": probe["dfma_per_clock_per_sm"],
                               "dependent_dfma_clocks": probe["dependent_dfma_clocks"],
                               "sm_count": probe["sm_count"]},
                     "int_mul64_per_launch": muls,
                     "int_mul64_frac": muls / (ms_per_step / 1000.0) / mul_peak,
                     "int_mul64_peak_per_s": mul_peak,
                     "issue_active_pct": issue_pct,
                     "hbm_gbs": None if traffic is None else traffic / (ms_per_step / 1000.0) / 1e9,
                     "hbm_frac": None if traffic is None else
                     traffic / (ms_per_step / 1000.0) / 1e9 / measured_hbm_gbs()[0],
                     "binding": "dependent latency of each instance's gate chain (fixed-point multiplies, "
                                "shared-memory loads and one barrier per gate); FP64-equivalent flops, integer "
                                "multiplies and DRAM bytes are all far below their peaks"},
        "clocks": clocks,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(th_np.nbytes),
                "d2h_bytes_per_step": int(e_np.nbytes + g_np.nbytes), "steps": K2},
        "gpu_launches": K,
        "wall_s_timed_region": t_wall,
    }
    if rank == 0 and world == 1 and not args.no_per_config:
        extra = {}
        if "complex" not in args.skip:
            c1 = entry_config1_complex(B, theta, n_inst, M, K, args.warmup, gpu_index_for(local_rank))
            c1["max_abs_diff_energy_vs_real"] = float((c1.pop("energies") - energies).abs().max())
            extra["config1_complex128"] = c1
        del wsh, ws
        torch.cuda.empty_cache()
        line["per_config"] = per_config(args, gpu_index_for(local_rank), extra)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
