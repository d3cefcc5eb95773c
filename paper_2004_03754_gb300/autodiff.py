"""torch.autograd front ends of libpic's hand-written adjoint (FP64).

Both functions run the forward simulation and its reverse sweep (with
checkpointing every ``checkpoint_every`` steps and recomputation of each
segment) inside one C call; the gradients are handed to autograd in backward().
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import pic as P


class LaserEnergy(torch.autograd.Function):
    """J(a0, phase) = mean final (gamma - 1) of the electrons after nsteps steps.

    sim: an FP64 2D ``pic.Simulation`` (Boris or analytic pusher); laser: dict of the other
    pic_laser fields; x, u: host particle arrays (ndim*n, 3*n); w: host weights (n,), or
    None for test electrons (weight 0).  Electrons of non-zero weight deposit current, and
    the gradient includes their current's effect on the fields."""

    @staticmethod
    def forward(ctx, a0, phase, sim, laser, x, u, nsteps, checkpoint_every=100, w=None):
        las = P.pic_laser(float(a0), laser.get("k0", 1.0), float(phase), laser["L_env"],
                          laser["x_front"], laser.get("w0", 0.0), laser["x2c"], laser.get("x3c", 0.0))
        if w is None:
            J, ga, gp = P.pic_adjoint_laser_energy(sim.ctx, las, x, u, nsteps, checkpoint_every)
        else:
            J, ga, gp = P.pic_adjoint_laser_energy_w(sim.ctx, las, x, u, w, nsteps, checkpoint_every)
        ctx.g = (ga, gp)
        return torch.tensor(J, dtype=torch.float64)

    @staticmethod
    def backward(ctx, gJ):
        ga, gp = ctx.g
        return gJ * ga, gJ * gp, None, None, None, None, None, None, None


class DispersionError(torch.autograd.Function):
    """J(C^E, C^B) = 1/2 |E2^N - target|^2 of a vacuum pulse after nsteps field steps."""

    @staticmethod
    def forward(ctx, cE, cB, n, dx, dt, e2_0, b3_0, target, nsteps, checkpoint_every=100):
        ce = cE.detach().cpu().numpy().astype(np.float64)
        cb = cB.detach().cpu().numpy().astype(np.float64)
        sim = P.Simulation(n, dx, dt, ce, cb, precision="fp64", pusher="boris")
        try:
            J, gE, gB = P.pic_adjoint_dispersion(sim.ctx, e2_0, b3_0, target, nsteps, ce.size,
                                                 checkpoint_every)
        finally:
            sim.close()
        ctx.g = (torch.from_numpy(gE), torch.from_numpy(gB))
        return torch.tensor(J, dtype=torch.float64)

    @staticmethod
    def backward(ctx, gJ):
        gE, gB = ctx.g
        return gJ * gE, gJ * gB, None, None, None, None, None, None, None, None
