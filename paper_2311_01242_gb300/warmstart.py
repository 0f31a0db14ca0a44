"""Learned warm start for VQE along a bond-stretch scan.

The paper runs one VQE per geometry of a bond-stretch scan (Sec. 3.1, Figs.
7-8), each from the Hartree-Fock state (theta = 0) with BFGS (Sec. 3.1's
optimizer study). Here the angles that VQE converges to at a subset of scan
points train a small network (paper_2311_01242_gb300.mlp) that predicts the
angles at the other points from the geometry, r and diag h(r). A predicted
start is kept only when its energy is below the HF energy; otherwise the
plain HF start is used.

Pieces:
  vqe_bfgs         BFGS on the host over GPU energy+gradient evaluations
  lanczos_ground   exact sector ground energy: Lanczos with GPU H|v>
  WarmStart        features, training set, network fit and prediction
  compare_starts   evaluations and wall time to reach a target energy for the
                   HF start, previous-point continuation, and the network start
"""
import time

import numpy as np
import scipy.linalg as sla
import scipy.optimize as so
import torch

from . import api
from .mlp import WarmStartMLP


def sector_indices(n_qubits, n_elec):
    """Sorted basis indices of the (N, N_alpha) sector of the HF reference."""
    na = (n_elec + 1) // 2
    ks = np.arange(1 << n_qubits, dtype=np.int64)
    pc = np.zeros_like(ks)
    pa = np.zeros_like(ks)
    for q in range(n_qubits):
        bit = (ks >> q) & 1
        pc += bit
        if q % 2 == 0:
            pa += bit
    return ks[(pc == n_elec) & (pa == na)]


class Geometry:
    """Handles and features of one scan point; with graph=True the point's
    energy+gradient evaluation is captured once in a CUDA graph."""

    def __init__(self, problem, r, ansatz, drop_tol=1e-14, graph=False):
        self.problem = problem
        self.r = float(r)
        self.H = api.Hamiltonian.from_problem(problem, drop_tol)
        self.A = ansatz
        self.features = np.concatenate([[self.r], np.diag(problem.h)])
        self.evaluator = api.GraphEnergyGrad(self.H, self.A) if graph else None


def vqe_bfgs(H, A, theta0, workspace=None, gtol=1e-7, maxiter=3000, stop_below=None, evaluator=None):
    """BFGS from theta0. Returns (theta, E, history) with history a list of
    (energy, seconds since start) per energy+gradient evaluation. With
    stop_below, stops at the first evaluation whose energy is <= stop_below.
    evaluator: an api.GraphEnergyGrad for (H, A) to replay instead of launching."""
    if workspace is None and evaluator is None:
        workspace = api.alloc_workspace(api.workspace_bytes(H, A, api.VQE_WS_GRAD))
    hist = []
    t0 = time.perf_counter()
    th_dev = torch.empty(A.n_params, dtype=torch.float64, device="cuda")

    class _Stop(Exception):
        pass

    best = {"e": np.inf, "t": np.asarray(theta0, dtype=float).copy()}

    def fun(t):
        th_dev.copy_(torch.from_numpy(np.ascontiguousarray(t, dtype=np.float64)))
        if evaluator is not None:
            e, g = evaluator(th_dev)
        else:
            e, g = api.energy_grad(H, A, th_dev, workspace=workspace)
        ev = float(e)
        gg = g.cpu().numpy()
        hist.append((ev, time.perf_counter() - t0))
        if ev < best["e"]:
            best["e"], best["t"] = ev, np.array(t, dtype=float)
        if stop_below is not None and ev <= stop_below:
            raise _Stop()
        return ev, gg

    try:
        res = so.minimize(fun, np.asarray(theta0, dtype=float), jac=True, method="BFGS",
                          options={"gtol": gtol, "maxiter": maxiter})
        return res.x, float(res.fun), hist
    except _Stop:
        return best["t"], best["e"], hist


def lanczos_ground(H, A, n_qubits, n_elec, tol=1e-11, max_iter=400, seed=0):
    """Lowest eigenvalue of H in the reference's sector by Lanczos with full
    reorthogonalisation; H|v> is libvqe's X-mask-grouped kernel."""
    idx = sector_indices(n_qubits, n_elec)
    D = len(idx)
    rng = np.random.default_rng(seed)
    full = torch.zeros(1 << n_qubits, dtype=torch.complex128, device="cuda")
    idx_t = torch.as_tensor(idx, device="cuda")
    ws = api.alloc_workspace(api.workspace_bytes(H, A, api.VQE_WS_COMPLEX))

    def hv(v):
        full.zero_()
        full[idx_t] = torch.as_tensor(v, dtype=torch.complex128, device="cuda")
        lam, _ = api.apply_hamiltonian(H, A, full, workspace=ws)
        return lam[idx_t].real.cpu().numpy()

    V = np.zeros((min(max_iter, D) + 1, D))
    v = rng.normal(size=D)
    V[0] = v / np.linalg.norm(v)
    alpha, beta = [], []
    e_prev = np.inf
    for j in range(min(max_iter, D)):
        w = hv(V[j])
        a = float(V[j] @ w)
        alpha.append(a)
        w -= V[:j + 1].T @ (V[:j + 1] @ w)
        w -= V[:j + 1].T @ (V[:j + 1] @ w)
        b = float(np.linalg.norm(w))
        ev = sla.eigh_tridiagonal(np.array(alpha), np.array(beta), eigvals_only=True,
                                  select="i", select_range=(0, 0))[0] if j > 0 else a
        if abs(ev - e_prev) < tol or b < 1e-12 or j + 1 == D:
            return float(ev)
        e_prev = ev
        beta.append(b)
        V[j + 1] = w / b
    return float(e_prev)


class WarmStart:
    """Network from standardised features to standardised angles."""

    def __init__(self, n_features, n_params, hidden=256, seed=0):
        self.net = WarmStartMLP(n_features, hidden, n_params, seed=seed)
        self.n_params = n_params

    def fit(self, X, Y, steps=3000, lr=1e-3):
        X = np.asarray(X, dtype=np.float64)
        Y = np.asarray(Y, dtype=np.float64)
        self.xm, self.xs = X.mean(0), X.std(0) + 1e-12
        self.ym, self.ys = Y.mean(0), Y.std(0) + 1e-6
        Xs = ((X - self.xm) / self.xs).astype(np.float32)
        Ys = ((Y - self.ym) / self.ys).astype(np.float32)
        return self.net.fit(Xs, Ys, steps=steps, lr=lr, use_graph=True)

    def predict(self, X):
        Xs = ((np.atleast_2d(X) - self.xm) / self.xs).astype(np.float32)
        y = self.net.forward(Xs).cpu().numpy().astype(np.float64)
        return y * self.ys + self.ym


def training_set(geoms, gtol=1e-7, maxiter=3000):
    """Plain VQE at each training geometry in scan order, each started from the
    previous point's converged angles (the first from HF)."""
    thetas, energies, evals = [], [], []
    theta = np.zeros(geoms[0].A.n_params)
    for g in geoms:
        theta, e, hist = vqe_bfgs(g.H, g.A, theta, gtol=gtol, maxiter=maxiter, evaluator=g.evaluator)
        thetas.append(theta.copy())
        energies.append(e)
        evals.append(len(hist))
    return np.array(thetas), np.array(energies), np.array(evals)


def compare_starts(geom, starts, e_exact, gtol=1e-7, maxiter=3000, tol_ha=1e-3):
    """Run BFGS from each named start to convergence; the target is
    E_exact + tol_ha, or (when no run gets there) the best converged energy +
    tol_ha. Returns per start: evaluations and seconds until the target, and
    the converged energy."""
    runs = {name: vqe_bfgs(geom.H, geom.A, th, gtol=gtol, maxiter=maxiter, evaluator=geom.evaluator)
            for name, th in starts.items()}
    e_best = min(r[1] for r in runs.values())
    target = e_exact + tol_ha if e_best <= e_exact + tol_ha else e_best + tol_ha
    out = {"target": target, "e_exact": e_exact, "reached_exact": bool(e_best <= e_exact + tol_ha)}
    for name, (_, e, hist) in runs.items():
        k = next((i for i, (ev, _) in enumerate(hist) if ev <= target), None)
        out[name] = {"evals": None if k is None else k + 1, "seconds": None if k is None else hist[k][1],
                     "e_conv": e, "evals_total": len(hist), "seconds_total": hist[-1][1] if hist else 0.0}
    return out
