"""Python front end of libsldg: device memory and streams from PyTorch, every
computation in the library's CUDA kernels (through ``_native``).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import torch

from . import _native as N


@dataclass
class Config:
    """Grid and time step of a 2D2V run (directions x1, x2, v1, v2).

    ``degree`` is the polynomial degree l per cell (the scheme dG(l+1));
    ``precision`` is "fp64" or "fp32" (storage and sweeps of f)."""

    degree: int
    ncell: tuple
    lo: tuple
    hi: tuple
    dt: float
    precision: str = "fp64"
    vbc: int = N.SLDG_VBC_ZERO_INFLOW
    poisson_kmax: int = -1
    flags: int = 0  # N.SLDG_FLAG_NATIVE_FP64: FP64 sweeps with FP64 FMA

    def c(self) -> N.sldg_config:
        c = N.sldg_config()
        c.degree = int(self.degree)
        for d in range(4):
            c.ncell[d] = int(self.ncell[d])
            c.lo[d] = float(self.lo[d])
            c.hi[d] = float(self.hi[d])
        c.dt = float(self.dt)
        c.precision = N.SLDG_FP64 if self.precision == "fp64" else N.SLDG_FP32
        c.vbc = int(self.vbc)
        c.poisson_kmax = int(self.poisson_kmax)
        c.flags = int(self.flags)
        return c

    @property
    def n(self):
        return self.degree + 1

    def D(self, d):
        return int(self.ncell[d]) * self.n

    @property
    def shape(self):
        """Shape of f as a tensor: (v2, v1, x2, x1), x1 contiguous."""
        return (self.D(3), self.D(2), self.D(1), self.D(0))

    @property
    def xshape(self):
        return (self.D(1), self.D(0))

    @property
    def numel(self):
        return self.D(0) * self.D(1) * self.D(2) * self.D(3)

    @property
    def dtype(self):
        return torch.float64 if self.precision == "fp64" else torch.float32


class Sldg:
    """One SLDG context bound to a caller-owned device tensor ``f``.

    The tensor must be contiguous on the current CUDA device with the
    layout ``Config.shape``; all work runs on ``stream`` (default: the
    current torch stream)."""

    _recordings = 0  # recordings made by any context (identifiers)

    def __init__(self, cfg: Config, f: torch.Tensor | None = None, stream=None):
        N.load()
        self.cfg = cfg
        if f is None:
            f = torch.empty(cfg.shape, dtype=cfg.dtype, device="cuda")
        if not (f.is_cuda and f.is_contiguous() and f.dtype == cfg.dtype and f.numel() == cfg.numel):
            raise ValueError("f must be a contiguous CUDA tensor of the configured shape and dtype")
        self.f = f
        self.stream = stream if stream is not None else torch.cuda.current_stream(f.device)
        self._ctx = N.sldg_init(cfg.c(), f.data_ptr(), self.stream.cuda_stream)
        self.recording = 0  # increments with every record(); 0: none yet

    # ---- life cycle -------------------------------------------------------
    def close(self):
        if self._ctx is not None:
            N.sldg_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def ctx(self):
        return self._ctx

    # ---- state --------------------------------------------------------------
    def set_initial(self, kind: int, params):
        N.sldg_set_initial(self._ctx, kind, params)

    def set_f(self, src: torch.Tensor, t: float = 0.0, step: int = 0):
        assert src.dtype == self.cfg.dtype and src.numel() == self.cfg.numel and src.is_contiguous()
        N.sldg_set_f(self._ctx, src.data_ptr(), src.is_cuda, t, step)

    def get_f(self, dst: torch.Tensor):
        assert dst.dtype == self.cfg.dtype and dst.numel() == self.cfg.numel and dst.is_contiguous()
        N.sldg_get_f(self._ctx, dst.data_ptr(), dst.is_cuda)

    # ---- hot path -----------------------------------------------------------
    def step(self, nsteps: int = 1, history: bool = False):
        W = np.zeros(max(nsteps, 1)) if history else None
        N.sldg_step(self._ctx, nsteps, W)
        return W[:nsteps] if history else None

    def step_host_batches(self, host: torch.Tensor, nbatch: int | None = None):
        """One Strang step for each state in ``host`` (a CPU tensor, pinned
        for overlapped copies): shape ``(nbatch,) + Config.shape`` or
        ``Config.shape`` with ``nbatch`` repeats of the same state.  Returns
        W of each batch's step; ``f`` ends as the last batch's stepped state."""
        assert not host.is_cuda and host.dtype == self.cfg.dtype and host.is_contiguous()
        if nbatch is None:
            assert host.numel() % self.cfg.numel == 0
            nbatch, stride = host.numel() // self.cfg.numel, self.cfg.numel * host.element_size()
        else:
            assert host.numel() == self.cfg.numel
            stride = 0
        W = np.zeros(nbatch)
        N.sldg_step_host_batches(self._ctx, host.data_ptr(), stride, nbatch, W)
        return W

    def sweep(self, dim: int, frac: float):
        N.sldg_sweep(self._ctx, dim, frac)

    def drift(self, frac: float):
        """X1 then X2 by frac * dt: the drift kernels of a Strang step."""
        N.sldg_drift(self._ctx, frac)

    def compute_fields(self):
        N.sldg_compute_fields(self._ctx)

    def set_field(self, E1: torch.Tensor, E2: torch.Tensor):
        E1 = E1.to(torch.float64).contiguous()
        E2 = E2.to(torch.float64).contiguous()
        if E1.is_cuda:
            N.sldg_set_field(self._ctx, E1.data_ptr(), E2.data_ptr(), True)
            torch.cuda.current_stream().synchronize()
        else:
            N.sldg_set_field(self._ctx, E1.data_ptr(), E2.data_ptr(), False)

    def fields(self):
        """(rho, E1, E2) as float64 numpy arrays of shape (D_x2, D_x1)."""
        out = [np.zeros(self.cfg.xshape) for _ in range(3)]
        N.sldg_fields(self._ctx, *(o.ctypes.data for o in out), False)
        return tuple(out)

    def diagnostics(self) -> dict:
        d = N.sldg_diagnostics(self._ctx)
        return {k: getattr(d, k) for k in ("t", "step", "mass", "l1", "l2sq", "kinetic",
                                           "electric", "total")}

    # ---- adjoint ------------------------------------------------------------
    def sweep_adjoint(self, dim: int, frac: float, lam: torch.Tensor, g: torch.Tensor | None = None,
                      Ebar: torch.Tensor | None = None):
        N.sldg_sweep_adjoint(self._ctx, dim, frac, lam.data_ptr(),
                             None if g is None else g.data_ptr(),
                             None if Ebar is None else Ebar.data_ptr())

    def record(self, nsteps: int, ckpt_every: int):
        """Record nsteps Strang steps for backward(); returns W of each step.
        ``recording`` identifies this recording (it replaces any earlier one)."""
        self.recording = 0
        W = np.zeros(nsteps)
        N.sldg_record(self._ctx, nsteps, ckpt_every, W)
        Sldg._recordings += 1
        self.recording = Sldg._recordings
        self.record_steps = nsteps
        return W

    def objective(self, cW=None) -> float:
        """J = sum_m cW[m] W_m of the last recording (cW = dt: the
        time-integrated electric energy), computed by the library."""
        c = None if cW is None else np.ascontiguousarray(cW, dtype=np.float64)
        return N.sldg_objective(self._ctx, c)

    def backward(self, cW=None, grad: torch.Tensor | None = None):
        if grad is None:
            grad = torch.empty_like(self.f)
        c = None if cW is None else np.ascontiguousarray(cW, dtype=np.float64)
        J = N.sldg_backward(self._ctx, c, grad.data_ptr())
        return J, grad

    def set_slot_limit(self, max_slots: int):
        N.sldg_set_slot_limit(self._ctx, max_slots)

    def backward_stats(self):
        """(Strang steps recomputed by the last backward, recomputation slots held)."""
        return N.sldg_backward_stats(self._ctx)

    def initial_param_grad(self, kind: int, params, grad: torch.Tensor) -> float:
        return N.sldg_initial_param_grad(self._ctx, kind, params, grad.data_ptr())

    # ---- measurement --------------------------------------------------------
    @property
    def launch_count(self) -> int:
        return N.sldg_launch_count(self._ctx)

    @property
    def x_pass_shape(self):
        """(CTAs per x-plane, lanes per x1 line pair) of the last fused x pass."""
        return N.sldg_x_pass_shape(self._ctx)

    def timing(self, enable: bool):
        N.sldg_timing(self._ctx, enable)

    def timing_read(self) -> dict:
        return N.sldg_timing_read(self._ctx)
