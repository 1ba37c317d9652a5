"""The variational loop around the energy and its gradient (Sec. 5 of the paper).

The paper minimises E(theta) with gradient-based optimisers (BFGS-type and Adam) and stops when
the energy change between iterations falls below 1e-6, the gradient norm below 1e-5, or after
100 iterations.  `minimize` runs that loop with torch.optim on any energy-and-gradient callable;
`mps_objective` supplies E and dE/dtheta from the library (MPSEnergy: one energy + reverse pass
per evaluation, whatever the number of parameters).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable

import torch

from . import autograd


@dataclass
class VQEResult:
    theta: torch.Tensor
    energy: float
    grad_norm: float
    iterations: int
    evaluations: int
    reason: str                       # "energy", "gradient" or "iterations"
    history: list = field(default_factory=list)   # (E, |g|) per iteration


def mps_objective(state0, circuit, ham) -> Callable[[torch.Tensor], torch.Tensor]:
    """E(theta) as a differentiable torch function evaluated by the library."""
    def f(theta: torch.Tensor) -> torch.Tensor:
        return autograd.mps_energy(theta, state0, circuit, ham)
    return f


def minimize(energy: Callable[[torch.Tensor], torch.Tensor], theta0, method: str = "lbfgs",
             max_iter: int = 100, e_tol: float = 1e-6, g_tol: float = 1e-5, lr: float | None = None,
             device=None) -> VQEResult:
    """Minimise energy(theta) from theta0.

    method: "lbfgs" (torch.optim.LBFGS, strong-Wolfe line search, one outer iteration per step)
    or "adam".  Stops when |E_k - E_{k-1}| < e_tol, ||dE/dtheta|| < g_tol, or after max_iter
    iterations (the paper's criteria).
    """
    theta = torch.as_tensor(theta0, dtype=torch.float64, device=device).clone().requires_grad_(True)
    if method == "lbfgs":
        opt = torch.optim.LBFGS([theta], lr=1.0 if lr is None else lr, max_iter=20,
                                line_search_fn="strong_wolfe", tolerance_grad=g_tol, tolerance_change=1e-12)
    elif method == "adam":
        opt = torch.optim.Adam([theta], lr=0.05 if lr is None else lr)
    else:
        raise ValueError('method must be "lbfgs" or "adam"')
    n_eval = 0

    def closure():
        nonlocal n_eval
        opt.zero_grad()
        E = energy(theta)
        E.backward()
        n_eval += 1
        return E

    history = []
    E_prev = None
    reason = "iterations"
    it = 0
    if method == "adam":
        closure()                           # the gradient at the starting point
    for it in range(1, max_iter + 1):
        if method == "lbfgs":
            opt.step(closure)
        else:
            opt.step()
        E_now = float(closure())            # E and gradient at the new point (Adam's next step uses it)
        gn = float(theta.grad.norm())
        history.append((E_now, gn))
        if gn < g_tol:
            reason = "gradient"
            break
        if E_prev is not None and abs(E_now - E_prev) < e_tol:
            reason = "energy"
            break
        E_prev = E_now
    return VQEResult(theta=theta.detach(), energy=history[-1][0], grad_norm=history[-1][1], iterations=it,
                     evaluations=n_eval, reason=reason, history=history)
