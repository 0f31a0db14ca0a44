"""E(theta) as a differentiable torch function backed by the adjoint kernel.

forward runs vqe_energy_grad once (energy and the full gradient from one
forward sweep, one H psi and one reverse sweep); backward scales the stored
gradient by the incoming grad_output. No intermediate states are kept.
"""
import torch

from . import api


class VQEEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, h, a, workspace):
        e, g = api.energy_grad(h, a, theta, workspace=workspace)
        ctx.save_for_backward(g)
        return e.clone()

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        return grad_out * g, None, None, None


def vqe_energy(theta, h, a, workspace=None):
    """Differentiable E(theta) for a float64 CUDA tensor theta."""
    if workspace is None:
        workspace = api.alloc_workspace(api.workspace_bytes(h, a, api.VQE_WS_GRAD), theta.device)
    return VQEEnergy.apply(theta, h, a, workspace)
