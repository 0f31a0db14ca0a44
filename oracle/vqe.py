"""Energy (Eq. 1), its gradient, exact ground energies and a plain BFGS VQE loop.

E(theta) = Re <psi(theta)|H|psi(theta)> with psi(theta) = U_M ... U_1 |HF>.
The gradient is computed two independent ways:
 * directly from its definition, g_k = 2 Re <H psi | U_M ... U_{k+1} A_k U_k ... U_1 |HF>
   with A_k = T_k - T_k^dagger (dU_k/dtheta_k = A_k U_k), costing O(M^2) gates;
 * by the four-point shift rule, exact because E as a function of one theta_k is
   a0 + a1 cos t + b1 sin t + a2 cos 2t + b2 sin 2t (A_k has spectrum {0, +-i}):
   g_k = [E(t + pi/4) - E(t - pi/4)] - (sqrt(2) - 1)/2 [E(t + pi/2) - E(t - pi/2)].
Central finite differences are a sanity check only.

The exact energy E0 is the lowest eigenvalue of Eq. 2 in the reference's
(N, S_z) sector, the full-CI value the paper compares VQE against.
"""
import numpy as np
import scipy.linalg as sla
import scipy.optimize as so
import scipy.sparse.linalg as spla

from .ansatz import apply_gate, apply_generator, prepare_state
from .hamiltonian import hamiltonian_matrix, sector_basis, full_basis
from .pauli import pauli_sum_apply


class EnergyModel:
    """H acting on full 2^n state vectors, from integrals (route 1) or a Pauli sum (route 2)."""

    def __init__(self, n_qubits, apply_fn, label=""):
        self.n_qubits = n_qubits
        self._apply = apply_fn
        self.label = label

    @classmethod
    def from_problem(cls, problem, n_alpha=None, n_beta=None, full=None):
        """Route 1: Eq. 2 by literal ladder operators, on the full space (n <= 12 by
        default) or on the (N_alpha, N_beta) sector, in which case the state must
        vanish outside the sector (checked on every call)."""
        n = problem.n_qubits
        if full is None:
            full = n <= 12
        if full:
            basis = full_basis(n)
        else:
            if n_alpha is None:
                n_alpha, n_beta = (problem.n_elec + 1) // 2, problem.n_elec // 2
            basis = sector_basis(n, n_alpha, n_beta)
        H = hamiltonian_matrix(problem, basis)
        idx = basis.astype(np.int64)
        outside = np.ones(1 << n, dtype=bool)
        outside[idx] = False

        def apply(psi):
            if not full and np.any(psi[outside] != 0):
                raise ValueError("state has weight outside the sector basis")
            out = np.zeros(1 << n, dtype=complex)
            out[idx] = H @ psi[idx]
            return out

        m = cls(n, apply, "fermionic")
        m.matrix, m.basis = H, basis
        return m

    @classmethod
    def from_pauli(cls, n_qubits, xs, zs, cs):
        """Route 2: explicit Pauli action P|k> = i^{|x&z|} (-1)^{|k&z|} |k^x>."""
        return cls(n_qubits, lambda psi: pauli_sum_apply(xs, zs, cs, psi), "pauli")

    def apply(self, psi):
        return self._apply(psi)

    def expectation(self, psi):
        v = np.vdot(psi, self._apply(psi))
        return v.real, v.imag


def energy(model, hf_bits, excitations, thetas):
    psi = prepare_state(model.n_qubits, hf_bits, excitations, thetas)
    e, _ = model.expectation(psi)
    return e


def energy_pauli(n_qubits, xs, zs, cs, hf_bits, excitations, thetas):
    return energy(EnergyModel.from_pauli(n_qubits, xs, zs, cs), hf_bits, excitations, thetas)


def gradient_direct(model, hf_bits, excitations, thetas, indices=None):
    """g_k from the definition; indices selects a subset of k (all by default)."""
    thetas = np.asarray(thetas, dtype=float)
    M = len(excitations)
    states = [prepare_state(model.n_qubits, hf_bits, [], [])]
    for exc, th in zip(excitations, thetas):
        states.append(apply_gate(states[-1], exc, float(th)))
    psi = states[-1]
    hpsi = model.apply(psi)
    e = np.vdot(psi, hpsi).real
    ks = range(M) if indices is None else indices
    g = np.zeros(len(ks))
    for out, k in enumerate(ks):
        v = apply_generator(states[k + 1], excitations[k])
        for m in range(k + 1, M):
            v = apply_gate(v, excitations[m], float(thetas[m]))
        g[out] = 2.0 * np.vdot(hpsi, v).real
    return e, g


def gradient_shift(model, hf_bits, excitations, thetas, indices=None):
    thetas = np.asarray(thetas, dtype=float)
    ks = range(len(thetas)) if indices is None else indices
    w = (np.sqrt(2.0) - 1.0) / 2.0
    g = np.zeros(len(ks))
    for out, k in enumerate(ks):
        def e_at(shift):
            t = thetas.copy()
            t[k] += shift
            return energy(model, hf_bits, excitations, t)
        g[out] = (e_at(np.pi / 4) - e_at(-np.pi / 4)) - w * (e_at(np.pi / 2) - e_at(-np.pi / 2))
    return g


def gradient_fd(model, hf_bits, excitations, thetas, h=1e-5):
    thetas = np.asarray(thetas, dtype=float)
    g = np.zeros(len(thetas))
    for k in range(len(thetas)):
        tp = thetas.copy()
        tm = thetas.copy()
        tp[k] += h
        tm[k] -= h
        g[k] = (energy(model, hf_bits, excitations, tp)
                - energy(model, hf_bits, excitations, tm)) / (2 * h)
    return g


def exact_ground_energy(problem, n_alpha=None, n_beta=None):
    """Lowest eigenvalue of Eq. 2 in the (N_alpha, N_beta) sector."""
    if n_alpha is None:
        n_alpha, n_beta = (problem.n_elec + 1) // 2, problem.n_elec // 2
    basis = sector_basis(problem.n_qubits, n_alpha, n_beta)
    H = hamiltonian_matrix(problem, basis)
    if H.shape[0] <= 5000:
        return float(sla.eigh(H.toarray(), eigvals_only=True)[0])
    vals = spla.eigsh(H, k=1, which="SA", tol=1e-13, maxiter=100000)[0]
    return float(vals[0])


def run_bfgs(model, hf_bits, excitations, theta0, gtol=1e-10, maxiter=2000):
    """Plain BFGS VQE loop (Sec. 3.1's optimizer choice) on the oracle's E and g."""
    count = {"evals": 0}

    def fun(t):
        count["evals"] += 1
        e, g = gradient_direct(model, hf_bits, excitations, t)
        return e, g

    res = so.minimize(fun, np.asarray(theta0, dtype=float), jac=True, method="BFGS",
                      options={"gtol": gtol, "maxiter": maxiter})
    return res, count["evals"]
