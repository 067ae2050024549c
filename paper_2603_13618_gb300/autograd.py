"""``torch.autograd`` front end of the adjoint entry points (include/kss.h).

``kl_objective(rho0, tau, ux0, uy0, nsteps)`` returns the sensor objective
J = sum_x W(x) eps_KL(x) of step ``nsteps`` (the KL sensor, Eq. HKL-sensor, of a
periodic lattice started from f^eq(rho0, u0)) as a differentiable scalar tensor: its
backward pass is the hand-written discrete adjoint in the CUDA library, which returns
dJ/drho0 (u0 held fixed) and dJ/dtau.  Marshalling only: all arithmetic runs in the
library's kernels.
"""
from __future__ import annotations

import torch

from . import kss


class KLObjective(torch.autograd.Function):
    """J(rho0, tau); ux0, uy0 and the weights are constants."""

    @staticmethod
    def forward(ctx, rho0, tau, ux0, uy0, weight, nsteps, precision, checkpoint_every):
        ny, nx = rho0.shape
        adj = kss.Adjoint(nx, ny, int(nsteps), precision=precision,
                          checkpoint_every=int(checkpoint_every))
        args = [t.detach().to(device="cuda", dtype=torch.float64).contiguous()
                for t in (rho0, ux0, uy0)]
        w = None if weight is None else weight.detach().to(
            device="cuda", dtype=torch.float64).contiguous()
        J = adj.forward(*args, float(tau), weight=w)
        ctx.adj = adj
        ctx.rho_meta = (rho0.dtype, rho0.device)
        ctx.tau_meta = (tau.dtype, tau.device) if torch.is_tensor(tau) else None
        return torch.tensor(J, dtype=torch.float64, device=rho0.device)

    @staticmethod
    def backward(ctx, gJ):
        g, gt = ctx.adj.backward(device=True)
        ctx.adj.close()
        dtype, device = ctx.rho_meta
        grad_rho = (gJ.to(torch.float64) * g).to(dtype=dtype, device=device)
        grad_tau = None
        if ctx.tau_meta is not None:
            grad_tau = (gJ.to(torch.float64) * gt).to(dtype=ctx.tau_meta[0],
                                                      device=ctx.tau_meta[1])
        return grad_rho, grad_tau, None, None, None, None, None, None


def kl_objective(rho0, tau, ux0, uy0, nsteps: int, weight=None, precision: str = "fp32",
                 checkpoint_every: int = 20):
    """Differentiable J = sum W eps_KL of step nsteps (see the module docstring)."""
    return KLObjective.apply(rho0, tau, ux0, uy0, weight, nsteps, precision, checkpoint_every)
