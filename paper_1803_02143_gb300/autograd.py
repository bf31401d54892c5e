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
    ckpt_every steps, and returns J as the library computes it.  The
    backward runs the library's adjoint (sldg_backward) with the weights
    scaled by the incoming gradient, so the returned dJ/df0 needs no further
    arithmetic.  A solver holds one recording: a backward after another
    forward on the same solver raises instead of returning the gradient of
    the later recording."""

    @staticmethod
    def forward(ctx, f0, solver: Sldg, nsteps: int, ckpt_every: int, cW=None):
        solver.set_f(f0.detach().contiguous())
        solver.record(nsteps, ckpt_every)
        c = None if cW is None else np.ascontiguousarray(cW, dtype=np.float64)
        if c is not None and c.size != nsteps:
            raise ValueError("cW needs one weight per step")
        ctx.solver = solver
        ctx.c = c
        ctx.recording = solver.recording
        J = solver.objective(c)
        return torch.tensor(J, dtype=torch.float64)

    @staticmethod
    def backward(ctx, gJ):
        if ctx.solver.recording != ctx.recording:
            raise RuntimeError("the solver recorded again since this forward; its adjoint "
                               "would be that of the later recording")
        nsteps = ctx.solver.record_steps
        c = np.full(nsteps, ctx.solver.cfg.dt) if ctx.c is None else ctx.c
        _, grad = ctx.solver.backward(c * float(gJ))
        return grad, None, None, None, None


def time_integrated_energy(f0, solver: Sldg, nsteps: int, ckpt_every: int, cW=None):
    return TimeIntegratedEnergy.apply(f0, solver, nsteps, ckpt_every, cW)
