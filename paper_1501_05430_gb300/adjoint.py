"""Differentiable simulation: the final density as a function of the bottom
wall's angles and the EOS temperature, with the gradient computed by the
library's hand-written discrete adjoint (lbm_adjoint_record /
lbm_adjoint_backward).

    rho = final_density(theta_bottom, T, nx=..., ny=..., eos=..., tau=...,
                        params=..., f0=..., steps=2000, checkpoint_every=100)
    loss = some_function(rho)          # any torch expression of rho
    loss.backward()                    # -> theta_bottom.grad, T.grad

Argument marshalling only: the forward steps, the tape and the reverse sweep
run in liblbm's CUDA kernels.  The initial state f0 is held fixed (no gradient
flows to it); the top wall keeps the angles given in ``theta_top``.
"""
from __future__ import annotations

import numpy as np
import torch

from . import lbm as L


class FinalDensity(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta_bottom, T, spec):
        nx, ny = spec["nx"], spec["ny"]
        theta = np.full((ny, nx), np.pi / 2)
        theta[0] = theta_bottom.detach().cpu().double().numpy()
        if spec.get("theta_top") is not None:
            theta[-1] = np.broadcast_to(np.asarray(spec["theta_top"], dtype=float), (nx,))
        sim = L.Lbm(nx, ny, spec["eos"], float(T.detach().cpu()), spec["tau"], theta=theta, params=spec["params"],
                    stream=spec.get("stream"), torch_state=False)
        sim.set_f(spec["f0"])
        L.lbm_adjoint_record(sim.ctx, spec["steps"], spec.get("checkpoint_every", 100))
        rho = sim.rho()
        ctx.sim = sim
        ctx.like = (theta_bottom, T)
        return torch.as_tensor(rho, dtype=torch.float64, device=theta_bottom.device)

    @staticmethod
    def backward(ctx, grad_rho):
        sim = ctx.sim
        dth, dT, _ = L.lbm_adjoint_backward(sim.ctx, grad_rho.detach().cpu().double().numpy())
        L.lbm_adjoint_release(sim.ctx)
        sim.close()
        tb, T = ctx.like
        return (torch.as_tensor(dth[0], dtype=tb.dtype, device=tb.device),
                torch.as_tensor(dT, dtype=T.dtype, device=T.device), None)


def final_density(theta_bottom: torch.Tensor, T: torch.Tensor, *, nx, ny, eos, tau, params, f0, steps,
                  checkpoint_every=100, theta_top=None, stream=None) -> torch.Tensor:
    """[ny, nx] float64 density after ``steps`` steps from the distributions
    ``f0`` ([9, ny, nx]), differentiable w.r.t. theta_bottom ([nx], radians)
    and T (scalar, absolute temperature of the EOS)."""
    spec = dict(nx=nx, ny=ny, eos=eos, tau=tau, params=params, f0=f0, steps=steps,
                checkpoint_every=checkpoint_every, theta_top=theta_top, stream=stream)
    return FinalDensity.apply(theta_bottom, T, spec)
