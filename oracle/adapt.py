"""ADAPT-VQE operator screening and the adaptive loop (Sec. 2.1.1, ADAPT-VQE).

ADAPT grows the ansatz one operator at a time from a pool: each round it
measures, for every pool operator A_j = T_j - T_j^dagger, the derivative of the
energy with respect to that operator's angle when the operator is appended at
angle 0 after the current circuit,

    g_j = d/dt <psi| e^{-t A_j} H e^{t A_j} |psi> at t = 0
        = <psi| [H, A_j] |psi> = 2 Re <H psi| A_j |psi>,

appends the operator of largest |g_j|, and re-optimises every angle. The paper
names the pool gradients as the convergence measure without fixing the rule;
the reading taken here stops when the 2-norm of the pool gradient vector falls
below a given tolerance (or the ansatz reaches a given size).

hf_pool_gradients is the closed form of g_j at the reference state itself
(empty ansatz): for a pool of excitations out of the occupied set,
T_j^dagger |HF> = 0, so g_j = 2 <HF|H T_j|HF>, which the Slater-Condon rules
give in terms of the integrals (derived in its docstring).

Test infrastructure: plain numpy, no code shared with the CUDA library.
"""
import numpy as np
import scipy.optimize as so

from .ansatz import apply_generator, prepare_state
from .vqe import gradient_direct


def pool_gradients(model, hf_bits, excitations, thetas, pool):
    """(E(theta), g) with g_j = 2 Re <H psi| (T_j - T_j^dagger) |psi> for each
    pool excitation j, psi = U(theta)|HF> (the definition, operator by operator)."""
    psi = prepare_state(model.n_qubits, hf_bits, excitations, thetas)
    hpsi = model.apply(psi)
    e = float(np.vdot(psi, hpsi).real)
    g = np.array([2.0 * np.vdot(hpsi, apply_generator(psi, op)).real for op in pool])
    return e, g


def hf_pool_gradients(problem, hf_bits, pool):
    """g_j at psi = |HF> from the integrals.

    With spin orbitals P = (p, sP) (qubit 2p + sP) and the Hamiltonian of Eq. 2
    written as sum h a+_P a_Q + 1/2 sum <PQ|RS> a+_P a+_Q a_S a_R, where
    <PQ|RS> = (pr|qs) delta_{sP sR} delta_{sQ sS}:
      single T = a+_A a_I:           <HF|H T|HF> = h_ia + sum_{K occ} (<IK|AK> - <IK|KA>)
                                                 = h_ia + sum_K [(ia|kk) - delta_{sI sK} (ik|ka)];
      double T = a+_A a+_B a_J a_I:  <HF|H T|HF> = <IJ|AB> - <IJ|BA>
                                                 = (ia|jb) d_IA d_JB - (ib|ja) d_IB d_JA,
    (d_XY = delta of the spins), and g_j = 2 <HF|H T_j|HF>. Requires I, J
    occupied and A, B empty in hf_bits."""
    h, eri = problem.h, problem.eri
    occ = [q for q in range(problem.n_qubits) if (hf_bits >> q) & 1]
    g = np.zeros(len(pool))
    for n, op in enumerate(pool):
        e = [int(v) for v in op]
        if e[2] < 0:
            I, A = e[0], e[1]
            if not ((hf_bits >> I) & 1) or ((hf_bits >> A) & 1):
                raise ValueError("pool excitation is not out of the reference")
            if I % 2 != A % 2:
                continue
            i, a = I // 2, A // 2
            v = h[i, a]
            for K in occ:
                k = K // 2
                v += eri[i, a, k, k]
                if K % 2 == I % 2:
                    v -= eri[i, k, k, a]
            g[n] = 2.0 * v
        else:
            I, J, A, B = e
            if (not ((hf_bits >> I) & 1) or not ((hf_bits >> J) & 1)
                    or ((hf_bits >> A) & 1) or ((hf_bits >> B) & 1)):
                raise ValueError("pool excitation is not out of the reference")
            i, j, a, b = I // 2, J // 2, A // 2, B // 2
            v = 0.0
            if I % 2 == A % 2 and J % 2 == B % 2:
                v += eri[i, a, j, b]
            if I % 2 == B % 2 and J % 2 == A % 2:
                v -= eri[i, b, j, a]
            g[n] = 2.0 * v
    return g


def adapt_vqe(model, hf_bits, pool, grad_tol=1e-3, max_ops=None, gtol=1e-10, maxiter=2000):
    """The ADAPT-VQE loop: screen the pool, append the operator of largest |g_j|
    (lowest index on ties) at angle 0, re-optimise all angles with BFGS from the
    previous optimum, until ||g||_2 < grad_tol or max_ops operators were added.
    Returns (energy, chosen pool indices, angles, per-round (E, ||g||, j))."""
    pool = np.asarray(pool, dtype=np.int64).reshape(-1, 4)
    chosen, theta, history = [], np.zeros(0), []
    while True:
        exc = pool[chosen]
        e, g = pool_gradients(model, hf_bits, exc, theta, pool)
        gnorm = float(np.linalg.norm(g))
        j = int(np.argmax(np.abs(g)))
        history.append((e, gnorm, j))
        if gnorm < grad_tol or (max_ops is not None and len(chosen) >= max_ops):
            return e, chosen, theta, history
        chosen.append(j)
        exc = pool[chosen]

        def fun(t):
            return gradient_direct(model, hf_bits, exc, t)

        res = so.minimize(fun, np.append(theta, 0.0), jac=True, method="BFGS",
                          options={"gtol": gtol, "maxiter": maxiter})
        theta = res.x
