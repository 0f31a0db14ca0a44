"""ADAPT-VQE (Sec. 2.1.1, ADAPT-VQE) over the library's screening and
energy+gradient calls.

Each round screens the whole pool with one vqe_pool_gradients call (forward
sweep, H psi and every pool operator's gradient on the device), appends the
operator of largest |g_j| (lowest index on ties) at angle 0, and re-optimises
all angles with BFGS on the host from the previous optimum, each evaluation
one vqe_batch_energy_grad_host call on a one-instance batch (angles in, energy
and gradient out through pinned host arrays; graph-replayed). The paper takes
the pool gradients as the convergence measure without fixing a rule; here the
loop stops when their 2-norm falls below grad_tol, or after max_ops operators.
"""
from dataclasses import dataclass, field
from typing import List

import numpy as np
import scipy.optimize as so
import torch

from . import api


@dataclass
class AdaptResult:
    energy: float
    chosen: List[int]                       # pool indices, in ansatz order
    theta: np.ndarray
    history: List[tuple] = field(default_factory=list)  # per round (E, ||g||, argmax j)
    evaluations: int = 0                    # energy+gradient calls of the BFGS runs


def adapt_vqe(H, n_qubits, hf_bits, pool_excitations, grad_tol=1e-3, max_ops=None, gtol=1e-10,
              maxiter=2000, device="cuda"):
    pool_exc = np.ascontiguousarray(np.asarray(pool_excitations, dtype=np.int32).reshape(-1, 4))
    pool = api.Ansatz(n_qubits, hf_bits, pool_exc)
    chosen, theta, history, evals = [], np.zeros(0), [], 0
    g_buf = torch.empty(max(len(pool_exc), 1), dtype=torch.float64, device=device)
    e_buf = torch.empty(1, dtype=torch.float64, device=device)
    while True:
        A = api.Ansatz(n_qubits, hf_bits, pool_exc[chosen].reshape(-1, 4))
        e, g = api.pool_gradients(H, A, pool, theta, device=device, out=(e_buf, g_buf))
        g = g.cpu().numpy()
        gnorm = float(np.linalg.norm(g))
        j = int(np.argmax(np.abs(g))) if len(g) else -1
        history.append((float(e), gnorm, j))
        if gnorm < grad_tol or (max_ops is not None and len(chosen) >= max_ops) or j < 0:
            return AdaptResult(float(e), chosen, theta, history, evals)
        chosen.append(j)
        A = api.Ansatz(n_qubits, hf_bits, pool_exc[chosen])
        # one-instance batch evaluated from pinned host arrays: each BFGS
        # evaluation is one library call (copies, launch and synchronisation)
        B = api.Batch([H], [A])
        m = A.n_params
        th_h = torch.zeros(1, m, dtype=torch.float64).pin_memory()
        e_h = torch.zeros(1, dtype=torch.float64).pin_memory()
        g_h = torch.zeros(1, m, dtype=torch.float64).pin_memory()
        ws = api.alloc_workspace(B.host_workspace_bytes(True), device)
        th_np, e_np, g_np = th_h.numpy(), e_h.numpy(), g_h.numpy()
        call = B.host_call(th_np, e_np, g_np, ws)

        def fun(t):
            nonlocal evals
            evals += 1
            th_np[0, :] = t
            call()
            return float(e_np[0]), g_np[0].copy()

        res = so.minimize(fun, np.append(theta, 0.0), jac=True, method="BFGS",
                          options={"gtol": gtol, "maxiter": maxiter})
        theta = res.x
