"""torch.autograd bridge for the reverse mode of libmc.

RolloutFn.apply(theta0, spec, n_steps, ckpt_every, stored) runs a rollout of
the world described by `spec` with its static rest angles replaced by
`theta0` (a CUDA float32 tensor [J]) and returns the beads' displacement
after n_steps, a CUDA tensor [N, 2].  Its backward calls mc_rollout_backward,
the hand-written adjoint with checkpoint-and-recompute (or, with stored=True,
over every step's record kept by the forward); there is no autograd graph of
the simulation itself.
"""
from __future__ import annotations

import dataclasses

import torch

from .world import World


class RolloutFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta0: torch.Tensor, spec, n_steps: int, ckpt_every: int = 100, stored: bool = False):
        sp = dataclasses.replace(spec, theta0=theta0.detach().float().cpu().numpy())
        world = World(sp)
        world.rollout_forward(n_steps, ckpt_every, stored=stored)
        disp = world.state_device()["disp"]
        ctx.world = world
        return disp

    @staticmethod
    def backward(ctx, grad_disp: torch.Tensor):
        g = grad_disp.contiguous().float()
        dtheta0 = ctx.world.rollout_backward(g[:, 0], g[:, 1])
        ctx.world.close()
        return dtheta0, None, None, None, None


def rollout_displacement(theta0: torch.Tensor, spec, n_steps: int, ckpt_every: int = 100,
                         stored: bool = False) -> torch.Tensor:
    return RolloutFn.apply(theta0, spec, n_steps, ckpt_every, stored)
