"""GB300-native state-vector VQE: energy E(theta) = <psi|H|psi> (Eq. 1) and its
adjoint gradient for Jordan-Wigner Hamiltonians (Sec. 2.1.1) and UCCSD
excitation ansatze (Sec. 2.1.2), computed by the CUDA library libvqe."""
from ._native import build, load
from .api import (Hamiltonian, Ansatz, Batch, VQEError, energy, energy_grad, state,
                  apply_hamiltonian, apply_hamiltonian_sector, jordan_wigner, hcb_hamiltonian, fold_frozen, workspace_bytes, alloc_workspace,
                  work_estimate, work_counts, set_flags, VQE_WS_ENERGY, VQE_WS_GRAD, VQE_WS_COMPLEX,
                  VQE_FLAG_FORCE_COMPLEX, VQE_FLAG_FORCE_STREAMING, VQE_FLAG_NO_CLUSTER, VQE_FLAG_FP64_SWEEPS,
                  VQE_FLAG_NO_STRINGS, VQE_FLAG_PERSISTENT_SWEEPS, VQE_FLAG_NO_PHI_STORE,
                  probe_fp64,
                  GraphEnergyGrad, batched_workspace_bytes, energy_grad_batched,
                  pool_workspace_bytes, pool_gradients)
from .autograd import VQEEnergy, vqe_energy

__all__ = [
    "build", "load", "Hamiltonian", "Ansatz", "Batch", "VQEError", "energy", "energy_grad",
    "state", "apply_hamiltonian", "apply_hamiltonian_sector", "jordan_wigner", "hcb_hamiltonian", "fold_frozen", "workspace_bytes", "alloc_workspace",
    "work_estimate", "work_counts", "set_flags", "VQEEnergy", "vqe_energy", "VQE_WS_ENERGY", "VQE_WS_GRAD",
    "VQE_WS_COMPLEX", "VQE_FLAG_FORCE_COMPLEX", "VQE_FLAG_FORCE_STREAMING", "VQE_FLAG_NO_CLUSTER", "VQE_FLAG_FP64_SWEEPS", "VQE_FLAG_NO_STRINGS", "VQE_FLAG_PERSISTENT_SWEEPS", "VQE_FLAG_NO_PHI_STORE",
    "probe_fp64",
    "GraphEnergyGrad", "batched_workspace_bytes", "energy_grad_batched",
    "pool_workspace_bytes", "pool_gradients",
]
