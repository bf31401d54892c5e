"""``torch.autograd.Function`` around the library's forward recording and
hand-written adjoint: J = sum_m c_m W(E^m), by default the time-integrated
electric energy tau * sum_m W(E^m), as a function of the initial f.
"""
from __future__ import annotations

import numpy as np
import torch

from .solver import Sldg


class TimeIntegratedEnergy(torch.autograd.Function):
    """forward(f0, solver, nsteps, ckpt_every, cW=None) -> J (float64 scalar).

    The forward copies f0 into the solver's state (a device copy in the
    library), records nsteps Strang steps with a checkpoint every
    ckpt_every steps, and returns J.  The backward runs the library's
    adjoint (sldg_backward) with the weights scaled by the incoming
    gradient, so the returned dJ/df0 needs no further arithmetic."""

    @staticmethod
    def forward(ctx, f0, solver: Sldg, nsteps: int, ckpt_every: int, cW=None):
        solver.set_f(f0.detach().contiguous())
        W = solver.record(nsteps, ckpt_every)
        c = np.full(nsteps, solver.cfg.dt) if cW is None else np.asarray(cW, dtype=np.float64)
        ctx.solver = solver
        ctx.c = c
        ctx.W = W
        J = float(np.dot(c, W))
        return torch.tensor(J, dtype=torch.float64)

    @staticmethod
    def backward(ctx, gJ):
        c = ctx.c * float(gJ)
        _, grad = ctx.solver.backward(c)
        return grad, None, None, None, None


def time_integrated_energy(f0, solver: Sldg, nsteps: int, ckpt_every: int, cW=None):
    return TimeIntegratedEnergy.apply(f0, solver, nsteps, ckpt_every, cW)
