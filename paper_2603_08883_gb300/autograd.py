"""torch.autograd bindings of the dressed QMF energy.

``dressed_energy(H, theta, phi, tau=None, gx=None, gz=None)`` returns the
energy of Eq. 12 for the product state of Eq. 3 (after one generator P at
amplitude tau when given, Eq. 5) as a 0-dim float64 tensor whose backward is
the library's adjoint kernel (``iqcc_energy_gradients``): one pass over H
gives the energy and every dE/dtheta_j, dE/dphi_j and dE/dtau, so joint
optimisation of the angles and the amplitude runs with any torch optimiser.
The angle tensors may live on any device; they are copied to the host (n
values each) for the call.
"""
from __future__ import annotations

import torch

from . import iqcc


class DressedQMFEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, phi, tau, H, gx, gz):
        t = theta.detach().to("cpu", torch.float64).numpy()
        p = phi.detach().to("cpu", torch.float64).numpy()
        tv = float(tau.detach()) if tau is not None else 0.0
        e, dt, dp, dtau = iqcc.iqcc_energy_gradients(H, t, p, gx, gz, tv)
        ctx.save_for_backward(torch.from_numpy(dt).to(theta.device), torch.from_numpy(dp).to(phi.device),
                              torch.tensor(dtau, dtype=torch.float64))
        ctx.tau_device = tau.device if tau is not None else None
        return torch.tensor(e, dtype=torch.float64, device=theta.device)

    @staticmethod
    def backward(ctx, grad_out):
        dt, dp, dtau = ctx.saved_tensors
        g = grad_out.to(torch.float64)
        gtau = (g.cpu() * dtau).to(ctx.tau_device) if ctx.tau_device is not None else None
        return g * dt, g * dp, gtau, None, None, None


def dressed_energy(H, theta: torch.Tensor, phi: torch.Tensor, tau: torch.Tensor | None = None, gx=None, gz=None):
    """E(theta, phi[, tau]) as a differentiable 0-dim tensor (float64)."""
    if (tau is None) != (gx is None) or (gx is None) != (gz is None):
        raise ValueError("tau, gx and gz go together")
    return DressedQMFEnergy.apply(theta, phi, tau, H, gx, gz)
