"""`MPSEnergy`: E(theta) as a torch.autograd.Function whose backward is the library's adjoint.

forward() runs mps_energy_grad (energy, cotangent and the full reverse pass in one call) and
keeps dE/dtheta; backward() scales it by the incoming gradient.  No autograd tape lives in
Python: the cost of the gradient does not grow with the number of parameters (Sec. 4).

A batched state (n_inst instances) takes theta of shape [n_inst, n_theta] and returns E of
shape [n_inst]; a single-instance state takes [n_theta] and returns a 0-d tensor.
"""
from __future__ import annotations

import torch

from . import api


class MPSEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta: torch.Tensor, state0: "api.State", circuit: "api.Circuit",
                ham: "api.Hamiltonian") -> torch.Tensor:
        th = theta.detach().to(torch.float64).contiguous()
        n_inst = state0.n_inst
        batched = th.dim() == 2
        if n_inst > 1 and (not batched or th.shape[0] != n_inst):
            raise ValueError(f"theta must have shape [{n_inst}, n_theta] for a state of {n_inst} instances")
        if not batched and th.dim() != 1:
            raise ValueError("theta must be 1-d (one instance) or 2-d (one row per instance)")
        # one energy per instance and one gradient row per instance: the library writes exactly
        # n_inst values of E and n_inst x n_theta values of the gradient
        E = torch.zeros(n_inst, dtype=torch.float64, device=th.device)
        g = torch.zeros(th.shape, dtype=torch.float64, device=th.device)
        api.energy_grad(state0, circuit, th, ham, out=(E, g))
        ctx.save_for_backward(g)
        ctx.batched = batched
        out = E if batched else E[0]
        return out.to(theta.dtype)

    @staticmethod
    def backward(ctx, grad_E: torch.Tensor):
        (g,) = ctx.saved_tensors
        gE = grad_E.to(torch.float64)
        if ctx.batched:
            gth = gE.reshape(-1, 1) * g          # one incoming gradient per instance
        else:
            gth = gE * g
        return gth.to(grad_E.dtype), None, None, None


def mps_energy(theta: torch.Tensor, state0, circuit, ham) -> torch.Tensor:
    """E(theta) with dE/dtheta available through torch.autograd."""
    return MPSEnergy.apply(theta, state0, circuit, ham)
