"""The five seeded workloads (sizes of the paper's active spaces, random integrals).

config0: 4 qubits, 2 electrons, K=4, full UCCSD pool (3 excitations), seed 0.
config1: 12 qubits, 6 electrons, K=6, 64-point scan r in [0.8, 3.0], full pool
         (117 excitations), theta ~ N(0, 0.05) per geometry, seed 1.
config2: 256 instances, n uniform in {14,16,18,20}, n/2 electrons, K=n/2, the
         first M excitations (M uniform in [64, 256], capped at the pool size) of
         a seeded shuffle of the pool; instance j draws from default_rng([2, j]),
         (n_j, M_j) from default_rng(2).
config3: 30 qubits, 10 electrons, K=8, 512 excitations of a seeded shuffle of
         the 3500-excitation pool, theta ~ N(0, 0.05), seed 3; terms below 1e-8
         are dropped.
config4: 16 qubits, 8 electrons, K=8, 512-point scan r in [0.7, 4.0], full pool
         (360 excitations), seed 4.
puccd_scan: pUCCD at the CH3F frozen-core active-space size: 11 spatial
         orbitals, 8 electrons (4 pairs), K=6, 64-point scan r in [0.8, 3.0],
         the 28 pair excitations, theta ~ N(0, 0.05) per geometry, seed 5.
puccd_large: pUCCD, 24 spatial orbitals, 24 electrons (12 pairs, 2.7M boson
         states), K=8, the 144 pair excitations, theta ~ N(0, 0.05), seed 6.
"""
from dataclasses import dataclass, field
from typing import List

import numpy as np

from .integrals import Problem, random_problem, draw_scan, ScanProblem
from .pools import uccsd_pool, puccd_pool


@dataclass
class Workload:
    name: str
    problems: List[Problem]
    excitations: List[np.ndarray]
    thetas: List[np.ndarray]
    drop_tol: float = 1e-14
    scan: ScanProblem = None
    extra: dict = field(default_factory=dict)


def config0() -> Workload:
    rng = np.random.default_rng(0)
    p = random_problem(rng, 2, 2, 4, label="config0")
    exc = uccsd_pool(4, 2)
    theta = rng.normal(0.0, 0.05, size=len(exc))
    return Workload("4 qubits, 2 electrons, 3 excitations", [p], [exc], [theta])


def config1(n_geom: int = 64) -> Workload:
    rng = np.random.default_rng(1)
    rs = np.linspace(0.8, 3.0, 64)[:n_geom]
    scan = draw_scan(rng, 6, 6, 6, rs)
    exc = uccsd_pool(12, 6)
    thetas = rng.normal(0.0, 0.05, size=(64, len(exc)))[:n_geom]
    probs = scan.problems()
    return Workload("12 qubits x 64 geometries, 117 excitations", probs,
                    [exc] * len(probs), list(thetas), scan=scan)


def config2_sizes():
    rng = np.random.default_rng(2)
    ns = rng.choice(np.array([14, 16, 18, 20]), size=256)
    ms = rng.integers(64, 257, size=256)
    return ns, ms


def config2_instance(j: int):
    ns, ms = config2_sizes()
    n = int(ns[j])
    rng = np.random.default_rng([2, j])
    p = random_problem(rng, n // 2, n // 2, n // 2, label=f"config2[{j}]")
    pool = uccsd_pool(n, n // 2)
    perm = rng.permutation(len(pool))
    m = min(int(ms[j]), len(pool))
    exc = pool[perm[:m]]
    theta = rng.normal(0.0, 0.05, size=m)
    return p, exc, theta


def config2(indices=None) -> Workload:
    if indices is None:
        indices = range(256)
    probs, excs, ths = [], [], []
    for j in indices:
        p, e, t = config2_instance(j)
        probs.append(p)
        excs.append(e)
        ths.append(t)
    return Workload("uneven batch n in {14,16,18,20}", probs, excs, ths)


def config3(n_exc: int = 512) -> Workload:
    rng = np.random.default_rng(3)
    p = random_problem(rng, 15, 10, 8, label="config3")
    pool = uccsd_pool(30, 10)
    perm = rng.permutation(len(pool))
    exc = pool[perm[:n_exc]]
    theta = rng.normal(0.0, 0.05, size=n_exc)
    return Workload("30 qubits, 10 electrons, 512 excitations", [p], [exc], [theta],
                    drop_tol=1e-8)


def config4() -> Workload:
    rng = np.random.default_rng(4)
    rs = np.linspace(0.7, 4.0, 512)
    scan = draw_scan(rng, 8, 8, 8, rs)
    exc = uccsd_pool(16, 8)
    return Workload("16 qubits scan, 512 points", [], [exc], [], scan=scan)


def puccd_scan(n_geom: int = 64) -> Workload:
    rng = np.random.default_rng(5)
    rs = np.linspace(0.8, 3.0, 64)[:n_geom]
    scan = draw_scan(rng, 11, 8, 6, rs)
    exc = puccd_pool(22, 8)
    thetas = rng.normal(0.0, 0.05, size=(64, len(exc)))[:n_geom]
    probs = scan.problems()
    return Workload("pUCCD, 11 orbitals x 64 geometries, 28 pair excitations", probs,
                    [exc] * len(probs), list(thetas), scan=scan)


def puccd_large() -> Workload:
    rng = np.random.default_rng(6)
    p = random_problem(rng, 24, 24, 8, label="puccd_large")
    exc = puccd_pool(48, 24)
    theta = rng.normal(0.0, 0.05, size=len(exc))
    return Workload("pUCCD, 24 orbitals, 12 pairs, 144 pair excitations", [p], [exc], [theta])
