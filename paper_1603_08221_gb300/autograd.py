"""torch.autograd.Function over the library's adjoint: the separation degree
CL (or the light species' outlet flux) of a channel after a fixed number of
steps as a differentiable function of the pressure ratio theta, the outlet
Knudsen number and the per-wall-node accommodation field.

Forward and backward both run in the CUDA library (lbm_adj_forward,
lbm_adj_gradient); this module only marshals tensors.
"""
from __future__ import annotations

import torch

from . import binding


class ChannelObjective(torch.autograd.Function):
    """objective(theta, Kn_out, alpha) for fixed gases, C_l, N, L/H and step
    count.  theta and Kn_out are 0-d tensors, alpha a [2, N_x] tensor
    (bottom wall, then top).  Returns a 0-d float64 tensor."""

    @staticmethod
    def forward(ctx, theta, kn_out, alpha, params: dict, nsteps: int,
                checkpoint_every: int = 70, objective: int = binding.LBM_ADJ_CL):
        p = dict(params)
        p["theta"] = float(theta)
        p["Kn_out"] = float(kn_out)
        adj = binding.LbmAdjoint(p, nsteps, checkpoint_every,
                                 alpha=alpha.detach().to("cpu", torch.float64).numpy())
        cl, flux = adj.forward()
        ctx.adj = adj
        ctx.objective = objective
        ctx.alpha_meta = (alpha.device, alpha.dtype, alpha.shape)
        value = cl if objective == binding.LBM_ADJ_CL else flux
        return torch.tensor(value, dtype=torch.float64)

    @staticmethod
    def backward(ctx, grad_out):
        g = ctx.adj.gradient(ctx.objective)
        dev, dt, shape = ctx.alpha_meta
        scale = float(grad_out)
        d_theta = torch.tensor(scale * g["theta"], dtype=torch.float64)
        d_kn = torch.tensor(scale * g["Kn_out"], dtype=torch.float64)
        d_alpha = (scale * torch.from_numpy(g["alpha"])).reshape(shape).to(dev, dt)
        return d_theta, d_kn, d_alpha, None, None, None, None


def channel_objective(theta, kn_out, alpha, params: dict, nsteps: int,
                      checkpoint_every: int = 70, objective: int = binding.LBM_ADJ_CL):
    return ChannelObjective.apply(theta, kn_out, alpha, params, nsteps, checkpoint_every,
                                  objective)
