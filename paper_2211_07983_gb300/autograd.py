"""`MPSEnergy`: E(theta) as a torch.autograd.Function whose backward is the library's adjoint.

forward() runs mps_energy_grad (energy, cotangent and the full reverse pass in one call) and
keeps dE/dtheta; backward() scales it by the incoming gradient.  No autograd tape lives in
Python: the cost of the gradient does not grow with the number of parameters (Sec. 4).
"""
from __future__ import annotations

import torch

from . import api


class MPSEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta: torch.Tensor, state0: "api.State", circuit: "api.Circuit",
                ham: "api.Hamiltonian") -> torch.Tensor:
        th = theta.detach().to(torch.float64).contiguous()
        E = torch.zeros(1, dtype=torch.float64, device=th.device)
        g = torch.zeros(th.numel(), dtype=torch.float64, device=th.device)
        if th.is_cuda:
            api.energy_grad(state0, circuit, th, ham, out=(E, g))
        else:
            e, gn = api.energy_grad(state0, circuit, th.numpy(), ham)
            E[0] = e
            g.copy_(torch.from_numpy(gn))
        ctx.save_for_backward(g)
        return E[0].to(theta.dtype)

    @staticmethod
    def backward(ctx, grad_E: torch.Tensor):
        (g,) = ctx.saved_tensors
        return (grad_E * g).to(grad_E.dtype), None, None, None


def mps_energy(theta: torch.Tensor, state0, circuit, ham) -> torch.Tensor:
    """E(theta) with dE/dtheta available through torch.autograd."""
    return MPSEnergy.apply(theta, state0, circuit, ham)
