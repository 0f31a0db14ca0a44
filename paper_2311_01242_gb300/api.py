"""Python binding of libvqe: argument marshalling only.

Every computation runs in the CUDA library; torch supplies device memory and
the current stream. Names follow include/vqe.h.
"""
import ctypes

import numpy as np
import torch

from . import _native

VQE_WS_ENERGY, VQE_WS_GRAD, VQE_WS_COMPLEX = 0, 1, 2
VQE_FLAG_FORCE_COMPLEX, VQE_FLAG_FORCE_STREAMING, VQE_FLAG_NO_CLUSTER, VQE_FLAG_FP64_SWEEPS = 1, 2, 4, 8
VQE_FLAG_NO_STRINGS = 16
VQE_FLAG_PERSISTENT_SWEEPS = 32
VQE_FLAG_NO_PHI_STORE = 64


class VQEError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libvqe error {code}: {msg}")
        self.code = code


def _lib():
    return _native.load()


def _check(rc):
    if rc != 0:
        raise VQEError(rc, _lib().vqe_last_error().decode(errors="replace"))


def _ptr(a):
    """Address of a tensor's or array's data as an int (ctypes passes it as void*)."""
    if a is None:
        return None
    if isinstance(a, torch.Tensor):
        return a.data_ptr()
    return a.ctypes.data


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def set_flags(flags: int) -> int:
    return _lib().vqe_set_flags(int(flags))


def _mapped_terms(fn, n_spatial, h, eri, c0, drop_tol):
    h = np.ascontiguousarray(h, dtype=np.float64)
    eri = np.ascontiguousarray(eri, dtype=np.float64)
    n = ctypes.c_int64(0)
    rc = fn(int(n_spatial), _ptr(h), _ptr(eri), float(c0), float(drop_tol), 0, None, None, None, ctypes.byref(n))
    if rc not in (0, 1):
        _check(rc)
    cnt = n.value
    xs = np.zeros(cnt, dtype=np.uint64)
    zs = np.zeros(cnt, dtype=np.uint64)
    cs = np.zeros(cnt, dtype=np.float64)
    _check(fn(int(n_spatial), _ptr(h), _ptr(eri), float(c0), float(drop_tol), cnt, _ptr(xs), _ptr(zs), _ptr(cs),
              ctypes.byref(n)))
    return xs, zs, cs


def jordan_wigner(n_spatial, h, eri, c0=0.0, drop_tol=1e-14):
    """Pauli sum (x_masks, z_masks, coefs) of Eq. 2's Hamiltonian (library's own mapping)."""
    return _mapped_terms(_lib().vqe_jordan_wigner, n_spatial, h, eri, c0, drop_tol)


def fold_frozen(h, eri, c0, frozen, active):
    """Frozen-core folding of Eq. 3 (vqe_fold_frozen): (h', eri', c0') on the
    active orbitals, in the order given."""
    h = np.ascontiguousarray(h, dtype=np.float64)
    eri = np.ascontiguousarray(eri, dtype=np.float64)
    fr = np.ascontiguousarray(frozen, dtype=np.int32)
    ac = np.ascontiguousarray(active, dtype=np.int32)
    na = len(ac)
    h_out = np.zeros((na, na))
    eri_out = np.zeros((na,) * 4)
    c0_out = ctypes.c_double()
    _check(_lib().vqe_fold_frozen(h.shape[0], _ptr(h), _ptr(eri), float(c0), len(fr), _ptr(fr) if len(fr) else None,
                                  na, _ptr(ac) if na else None, _ptr(h_out), _ptr(eri_out), ctypes.byref(c0_out)))
    return h_out, eri_out, c0_out.value


def hcb_hamiltonian(n_spatial, h, eri, c0=0.0, drop_tol=1e-14):
    """Pauli sum on n_spatial qubits of Eq. 2's seniority-zero block (pUCCD's
    hard-core boson form, vqe_hcb_hamiltonian)."""
    return _mapped_terms(_lib().vqe_hcb_hamiltonian, n_spatial, h, eri, c0, drop_tol)


class Hamiltonian:
    """Qubit Hamiltonian handle (vqe_create_hamiltonian)."""

    def __init__(self, n_qubits, x_masks, z_masks, coefs, drop_tol=0.0):
        xs = np.ascontiguousarray(x_masks, dtype=np.uint64)
        zs = np.ascontiguousarray(z_masks, dtype=np.uint64)
        cs = np.ascontiguousarray(coefs, dtype=np.float64)
        if not (len(xs) == len(zs) == len(cs)):
            raise ValueError("mask and coefficient arrays differ in length")
        self._lib = _lib()
        h = ctypes.c_void_p()
        _check(self._lib.vqe_create_hamiltonian(int(n_qubits), len(xs), _ptr(xs), _ptr(zs), _ptr(cs),
                                                float(drop_tol), ctypes.byref(h)))
        self.handle = h
        self.n_qubits = int(n_qubits)

    @classmethod
    def from_integrals(cls, n_spatial, h, eri, c0=0.0, drop_tol=1e-14):
        xs, zs, cs = jordan_wigner(n_spatial, h, eri, c0, drop_tol)
        return cls(2 * n_spatial, xs, zs, cs, drop_tol)

    @classmethod
    def from_problem(cls, problem, drop_tol=1e-14):
        return cls.from_integrals(problem.n_spatial, problem.h, problem.eri, problem.c0, drop_tol)

    @classmethod
    def from_problem_hcb(cls, problem, drop_tol=1e-14):
        """Hard-core boson form on n_spatial qubits (pUCCD)."""
        xs, zs, cs = hcb_hamiltonian(problem.n_spatial, problem.h, problem.eri, problem.c0, drop_tol)
        return cls(problem.n_spatial, xs, zs, cs, drop_tol)

    def info(self):
        n = ctypes.c_int()
        t = ctypes.c_int64()
        g = ctypes.c_int64()
        r = ctypes.c_int()
        _check(self._lib.vqe_hamiltonian_info(self.handle, ctypes.byref(n), ctypes.byref(t), ctypes.byref(g),
                                              ctypes.byref(r)))
        return {"n_qubits": n.value, "n_terms": t.value, "n_groups": g.value, "is_real": bool(r.value)}

    def terms(self):
        """Kept (x_masks, z_masks, create-time coefs), in vqe_set_coefs order."""
        t = self.info()["n_terms"]
        xs = np.zeros(t, dtype=np.uint64)
        zs = np.zeros(t, dtype=np.uint64)
        cs = np.zeros(t, dtype=np.float64)
        _check(self._lib.vqe_hamiltonian_terms(self.handle, _ptr(xs), _ptr(zs), _ptr(cs)))
        return xs, zs, cs

    def set_coefs(self, coefs, stream=None):
        """New coefficients (device float64, kept-term order) for the same Pauli strings."""
        if not (isinstance(coefs, torch.Tensor) and coefs.is_cuda and coefs.dtype == torch.float64
                and coefs.is_contiguous()):
            raise TypeError("coefs must be a contiguous float64 CUDA tensor")
        if coefs.numel() != self.info()["n_terms"]:
            raise ValueError("coefs must hold one value per kept term")
        _check(self._lib.vqe_set_coefs(self.handle, _ptr(coefs), _stream(stream)))

    def set_coefs_from(self, x_masks, z_masks, coefs, stream=None):
        """set_coefs from a term list (e.g. jordan_wigner at a new geometry); the
        strings must equal the kept ones."""
        xs, zs, _ = self.terms()
        if not (np.array_equal(np.asarray(x_masks, dtype=np.uint64), xs)
                and np.array_equal(np.asarray(z_masks, dtype=np.uint64), zs)):
            raise ValueError("Pauli strings differ from the Hamiltonian's kept terms")
        c = torch.as_tensor(np.ascontiguousarray(coefs, dtype=np.float64)).cuda()
        self.set_coefs(c, stream)
        return c

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            self._lib.vqe_destroy_hamiltonian(h)
            self.handle = None


class Ansatz:
    """UCCSD-type ansatz handle (vqe_create_ansatz); with hcb=True, pair
    excitations (i, a) of pUCCD's hard-core boson form (vqe_create_ansatz_hcb)."""

    def __init__(self, n_qubits, hf_bits, excitations, hcb=False):
        exc = np.ascontiguousarray(np.asarray(excitations, dtype=np.int32).reshape(-1, 2 if hcb else 4))
        self._lib = _lib()
        a = ctypes.c_void_p()
        create = self._lib.vqe_create_ansatz_hcb if hcb else self._lib.vqe_create_ansatz
        _check(create(int(n_qubits), int(hf_bits), len(exc), _ptr(exc), ctypes.byref(a)))
        self.handle = a
        self.n_qubits = int(n_qubits)
        self.n_params = len(exc)
        self.excitations = exc

    def info(self):
        n = ctypes.c_int()
        m = ctypes.c_int32()
        d = ctypes.c_int64()
        p = ctypes.c_int64()
        _check(self._lib.vqe_ansatz_info(self.handle, ctypes.byref(n), ctypes.byref(m), ctypes.byref(d),
                                         ctypes.byref(p)))
        return {"n_qubits": n.value, "n_params": m.value, "sector_dim": d.value, "n_pairs": p.value}

    def __del__(self):
        a = getattr(self, "handle", None)
        if a is not None and a.value:
            self._lib.vqe_destroy_ansatz(a)
            self.handle = None


def workspace_bytes(h: Hamiltonian, a: Ansatz, mode=VQE_WS_GRAD) -> int:
    nb = _lib().vqe_workspace_bytes(h.handle, a.handle, int(mode))
    if nb == 0:
        msg = _lib().vqe_last_error().decode(errors="replace")
        if msg:
            raise VQEError(-1, msg)
    return int(nb)


def alloc_workspace(nbytes, device="cuda"):
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def _as_theta(theta, device):
    if not isinstance(theta, torch.Tensor):
        theta = torch.as_tensor(np.asarray(theta, dtype=np.float64))
    return theta.to(device=device, dtype=torch.float64).contiguous()


def energy(h, a, theta, workspace=None, stream=None, device="cuda"):
    theta = _as_theta(theta, device)
    if workspace is None:
        workspace = alloc_workspace(workspace_bytes(h, a, VQE_WS_ENERGY), theta.device)
    e = torch.empty(1, dtype=torch.float64, device=theta.device)
    _check(_lib().vqe_energy(h.handle, a.handle, _ptr(theta), _ptr(e), _ptr(workspace), workspace.numel(),
                             _stream(stream)))
    return e[0]


def energy_grad(h, a, theta, workspace=None, stream=None, device="cuda", out=None):
    """(E, dE/dtheta); out=(e[1], g[>=n_params]) reuses caller buffers."""
    theta = _as_theta(theta, device)
    if workspace is None:
        workspace = alloc_workspace(workspace_bytes(h, a, VQE_WS_GRAD), theta.device)
    if out is None:
        e = torch.empty(1, dtype=torch.float64, device=theta.device)
        g = torch.empty(max(a.n_params, 1), dtype=torch.float64, device=theta.device)
    else:
        e, g = out
    _check(_lib().vqe_energy_grad(h.handle, a.handle, _ptr(theta), _ptr(e), _ptr(g), _ptr(workspace),
                                  workspace.numel(), _stream(stream)))
    return e[0], g[:a.n_params]


def state(a, h, theta, workspace=None, stream=None, device="cuda"):
    """psi(theta) as a full 2^n complex128 vector."""
    theta = _as_theta(theta, device)
    if workspace is None:
        workspace = alloc_workspace(workspace_bytes(h, a, VQE_WS_GRAD), theta.device)
    out = torch.empty(2 * (1 << a.n_qubits), dtype=torch.float64, device=theta.device)
    _check(_lib().vqe_state(a.handle, h.handle, _ptr(theta), _ptr(out), _ptr(workspace), workspace.numel(),
                            _stream(stream)))
    return torch.view_as_complex(out.view(-1, 2))


def apply_hamiltonian(h, a, psi, workspace=None, stream=None):
    """(H psi restricted to the ansatz sector, Re <psi|H|psi>) for a complex128 psi."""
    psi = psi.to(dtype=torch.complex128).contiguous()
    if workspace is None:
        workspace = alloc_workspace(workspace_bytes(h, a, VQE_WS_COMPLEX), psi.device)
    lam = torch.empty_like(psi)
    e = torch.empty(1, dtype=torch.float64, device=psi.device)
    _check(_lib().vqe_apply_hamiltonian(h.handle, a.handle, _ptr(torch.view_as_real(psi)),
                                        _ptr(torch.view_as_real(lam)), _ptr(e), _ptr(workspace),
                                        workspace.numel(), _stream(stream)))
    return lam, e[0]


def apply_hamiltonian_sector(h, a, psi, workspace=None, stream=None):
    """(lambda, <psi|lambda>) for a real float64 CUDA vector psi compressed to the
    ansatz's sector (vqe_apply_hamiltonian_sector): the real-amplitude H psi
    kernels of the energy and gradient calls."""
    assert psi.dtype == torch.float64 and psi.is_cuda and psi.is_contiguous()
    if workspace is None:
        workspace = alloc_workspace(workspace_bytes(h, a, VQE_WS_ENERGY), psi.device)
    lam = torch.empty_like(psi)
    e = torch.empty(1, dtype=torch.float64, device=psi.device)
    _check(_lib().vqe_apply_hamiltonian_sector(h.handle, a.handle, _ptr(psi), _ptr(lam), _ptr(e), _ptr(workspace),
                                               workspace.numel(), _stream(stream)))
    return lam, e[0]


def pool_workspace_bytes(h, a, pool):
    nb = _lib().vqe_pool_workspace_bytes(h.handle, a.handle, pool.handle)
    if nb == 0:
        raise VQEError(1, _lib().vqe_last_error().decode(errors="replace"))
    return int(nb)


def pool_gradients(h, a, pool, theta, workspace=None, stream=None, device="cuda", out=None):
    """ADAPT screening (vqe_pool_gradients): (E(theta), g) with
    g[j] = 2 Re <H psi| T_j - T_j^dagger |psi> for each operator of the pool
    handle `pool` (an Ansatz over the same sector). out=(e[1], g[>=n_pool])."""
    theta = _as_theta(theta, device)
    if workspace is None:
        workspace = alloc_workspace(pool_workspace_bytes(h, a, pool), theta.device)
    if out is None:
        e = torch.empty(1, dtype=torch.float64, device=theta.device)
        g = torch.empty(max(pool.n_params, 1), dtype=torch.float64, device=theta.device)
    else:
        e, g = out
    _check(_lib().vqe_pool_gradients(h.handle, a.handle, pool.handle, _ptr(theta) if a.n_params else None,
                                     _ptr(e), _ptr(g), _ptr(workspace), workspace.numel(), _stream(stream)))
    return e[0], g[:pool.n_params]


def work_estimate(h, a, with_grad=True):
    f = ctypes.c_double()
    b = ctypes.c_double()
    _check(_lib().vqe_work_estimate(h.handle, a.handle, int(bool(with_grad)), ctypes.byref(f), ctypes.byref(b)))
    return f.value, b.value


def work_counts(h, a):
    """vqe_work_counts: {"n_pairs", "n_entries", "extra_adds"} of the pair (h, a)."""
    p, e, x = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_double()
    _check(_lib().vqe_work_counts(h.handle, a.handle, ctypes.byref(p), ctypes.byref(e), ctypes.byref(x)))
    return {"n_pairs": p.value, "n_entries": e.value, "extra_adds": x.value}


class Batch:
    """Independent instances evaluated together (vqe_create_batch)."""

    def __init__(self, hams, ansatze):
        if len(hams) != len(ansatze):
            raise ValueError("hams and ansatze differ in length")
        self._lib = _lib()
        self.hams = list(hams)
        self.ansatze = list(ansatze)
        hs = (ctypes.c_void_p * len(hams))(*[h.handle.value for h in hams])
        As = (ctypes.c_void_p * len(ansatze))(*[a.handle.value for a in ansatze])
        b = ctypes.c_void_p()
        _check(self._lib.vqe_create_batch(len(hams), hs, As, ctypes.byref(b)))
        self.handle = b
        self.n_inst = len(hams)
        self.max_params = int(self._lib.vqe_batch_max_params(b))

    def workspace_bytes(self, with_grad=True):
        return int(self._lib.vqe_batch_workspace_bytes(self.handle, int(bool(with_grad))))

    def host_workspace_bytes(self, with_grad=True):
        return int(self._lib.vqe_batch_host_workspace_bytes(self.handle, int(bool(with_grad))))

    def energy_grad(self, theta, energies=None, grads=None, workspace=None, stream=None, with_grad=True):
        """theta: (n_inst, ld) float64 CUDA tensor. Returns (energies, grads)."""
        assert theta.dtype == torch.float64 and theta.is_cuda and theta.is_contiguous()
        dev = theta.device
        if energies is None:
            energies = torch.empty(self.n_inst, dtype=torch.float64, device=dev)
        if with_grad and grads is None:
            grads = torch.empty(self.n_inst, max(self.max_params, 1), dtype=torch.float64, device=dev)
        if workspace is None:
            workspace = alloc_workspace(self.workspace_bytes(with_grad), dev)
        _check(self._lib.vqe_batch_energy_grad(
            self.handle, _ptr(theta), theta.shape[1], _ptr(energies), _ptr(grads) if with_grad else None,
            grads.shape[1] if with_grad else 0, _ptr(workspace), workspace.numel(), _stream(stream)))
        return energies, grads

    def energy_grad_host(self, theta_host, energies_host, grads_host, workspace, stream=None):
        """Host arrays in and out (copies inside the call; synchronises the stream)."""
        _check(self._lib.vqe_batch_energy_grad_host(
            self.handle, _ptr(theta_host), theta_host.shape[1], _ptr(energies_host), _ptr(grads_host),
            grads_host.shape[1] if grads_host is not None else 0, _ptr(workspace), workspace.numel(),
            _stream(stream)))

    def set_tuning(self, ctas_per_sm=0, gate_chunk=0, sweep_threads=0):
        """vqe_batch_set_tuning (0 keeps a value; ctas_per_sm 0 = as many as fit)."""
        _check(self._lib.vqe_batch_set_tuning(self.handle, int(ctas_per_sm), int(gate_chunk), int(sweep_threads)))

    def tuning(self):
        """{"ctas_per_sm", "gate_chunk", "grid", "n_tasks"} of the persistent launch."""
        c, g, gr = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        nt = ctypes.c_int64()
        _check(self._lib.vqe_batch_get_tuning(self.handle, ctypes.byref(c), ctypes.byref(g), ctypes.byref(gr),
                                              ctypes.byref(nt)))
        return {"ctas_per_sm": c.value, "gate_chunk": g.value, "grid": gr.value, "n_tasks": nt.value}

    def set_wait(self, budget_ns=2_000_000_000, probe_task=-1):
        """vqe_batch_set_wait: the persistent launch's wait bound (and the timeout probe)."""
        _check(self._lib.vqe_batch_set_wait(self.handle, int(budget_ns), int(probe_task)))

    def status(self, workspace, stream=None):
        """vqe_batch_status of the last persistent launch on `workspace` (raises VQEError on a timeout)."""
        _check(self._lib.vqe_batch_status(self.handle, _ptr(workspace), workspace.numel(), _stream(stream)))

    def host_call(self, theta_host, energies_host, grads_host, workspace, stream=None):
        """energy_grad_host on fixed host arrays, marshalled once: the returned
        callable runs one evaluation per call (for optimizer loops that rewrite
        theta_host in place and read the results from the same arrays)."""
        return HostCall(self, theta_host, energies_host, grads_host, workspace, stream)

    def __del__(self):
        b = getattr(self, "handle", None)
        if b is not None and b.value:
            self._lib.vqe_destroy_batch(b)
            self.handle = None


class HostCall:
    """A prepared vqe_batch_energy_grad_host call (Batch.host_call)."""

    def __init__(self, batch, theta_host, energies_host, grads_host, workspace, stream=None):
        self._keep = (batch, theta_host, energies_host, grads_host, workspace)
        self._fn = batch._lib.vqe_batch_energy_grad_host
        self._args = (batch.handle.value, _ptr(theta_host), theta_host.shape[1], _ptr(energies_host),
                      _ptr(grads_host), grads_host.shape[1] if grads_host is not None else 0, _ptr(workspace),
                      workspace.numel(), _stream(stream))

    def __call__(self):
        rc = self._fn(*self._args)
        if rc:
            _check(rc)


def _handle_arrays(hams, ansatze):
    if len(hams) != len(ansatze) or not hams:
        raise ValueError("hams and ansatze must be non-empty and of equal length")
    hs = (ctypes.c_void_p * len(hams))(*[h.handle.value for h in hams])
    As = (ctypes.c_void_p * len(ansatze))(*[a.handle.value for a in ansatze])
    return hs, As


def batched_workspace_bytes(hams, ansatze, with_grad=True):
    """vqe_batched_workspace_bytes (builds and caches the instance list's plan)."""
    hs, As = _handle_arrays(hams, ansatze)
    n = int(_lib().vqe_batched_workspace_bytes(len(hams), hs, As, int(bool(with_grad))))
    if n == 0:
        raise VQEError(1, _lib().vqe_last_error().decode(errors="replace"))
    return n


def energy_grad_batched(hams, ansatze, thetas, energies=None, grads=None, workspace=None, stream=None,
                        with_grad=True):
    """vqe_energy_grad_batched / vqe_energy_batched over per-instance angle
    tensors (float64 CUDA, one per instance). Returns (energies, list of grads)."""
    hs, As = _handle_arrays(hams, ansatze)
    n = len(hams)
    if len(thetas) != n:
        raise ValueError("one theta per instance")
    thetas = [t if (t.dtype == torch.float64 and t.is_cuda and t.is_contiguous()) else
              torch.as_tensor(t, dtype=torch.float64).cuda().contiguous() for t in thetas]
    for t, a in zip(thetas, ansatze):
        if t.numel() < a.n_params:
            raise ValueError("theta shorter than the ansatz's parameter count")
    dev = thetas[0].device
    if energies is None:
        energies = torch.empty(n, dtype=torch.float64, device=dev)
    if with_grad and grads is None:
        grads = [torch.empty(max(a.n_params, 1), dtype=torch.float64, device=dev) for a in ansatze]
    if workspace is None:
        workspace = alloc_workspace(batched_workspace_bytes(hams, ansatze, with_grad), dev)
    tp = (ctypes.c_void_p * n)(*[t.data_ptr() for t in thetas])
    if with_grad:
        gp = (ctypes.c_void_p * n)(*[g.data_ptr() for g in grads])
        _check(_lib().vqe_energy_grad_batched(n, hs, As, tp, _ptr(energies), gp, _ptr(workspace),
                                              workspace.numel(), _stream(stream)))
        return energies, [g[:a.n_params] for g, a in zip(grads, ansatze)]
    _check(_lib().vqe_energy_batched(n, hs, As, tp, _ptr(energies), _ptr(workspace), workspace.numel(),
                                     _stream(stream)))
    return energies, None


class GraphEnergyGrad:
    """vqe_energy_grad of one (Hamiltonian, ansatz) pair captured once in a CUDA
    graph and replayed with new angles copied into the captured buffer (the
    streaming path issues two launches per gate; replay removes their host cost)."""

    def __init__(self, h, a, device="cuda"):
        self.h, self.a = h, a
        m = max(a.n_params, 1)
        self.theta = torch.zeros(m, dtype=torch.float64, device=device)
        self.e = torch.zeros(1, dtype=torch.float64, device=device)
        self.g = torch.zeros(m, dtype=torch.float64, device=device)
        self.ws = alloc_workspace(workspace_bytes(h, a, VQE_WS_GRAD), device)
        self._run()
        torch.cuda.synchronize()
        side = torch.cuda.Stream(device=device)
        side.wait_stream(torch.cuda.current_stream())
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.stream(side):
            with torch.cuda.graph(self.graph, stream=side):
                self._run()
        torch.cuda.current_stream().wait_stream(side)

    def _run(self):
        energy_grad(self.h, self.a, self.theta[:self.a.n_params] if self.a.n_params else self.theta,
                    workspace=self.ws, out=(self.e, self.g))

    def __call__(self, theta):
        if self.a.n_params:
            self.theta[:self.a.n_params].copy_(torch.as_tensor(theta, dtype=torch.float64))
        self.graph.replay()
        return self.e, self.g[:self.a.n_params]


def probe_fp64():
    """FP64 throughput/latency and device limits measured by vqe_probe_fp64."""
    r = [ctypes.c_double(), ctypes.c_double(), ctypes.c_double()]
    i = [ctypes.c_int(), ctypes.c_int()]
    sm = ctypes.c_size_t()
    l2 = ctypes.c_int()
    _check(_lib().vqe_probe_fp64(ctypes.byref(r[0]), ctypes.byref(r[1]), ctypes.byref(r[2]), ctypes.byref(i[0]),
                                 ctypes.byref(i[1]), ctypes.byref(sm), ctypes.byref(l2)))
    return {"dfma_per_sec": r[0].value, "dfma_per_clock_per_sm": r[1].value, "dependent_dfma_clocks": r[2].value,
            "sm_count": i[0].value, "sm_clock_khz": i[1].value, "smem_optin": sm.value, "l2_bytes": l2.value}
