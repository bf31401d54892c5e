"""The workloads: the paper's Landau damping and two-stream problems
(Sec. 4, Eq. (iv-nl); Sec. 5, Eq. (iv-tsi)) at the sizes this library is
measured on, and the paper's own dG4 runs (Sec. 4, Sec. 5, Table 1).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

from . import _native as N
from .solver import Config

LANDAU_LO = (0.0, 0.0, -6.0, -6.0)
LANDAU_HI = (4 * math.pi, 4 * math.pi, 6.0, 6.0)
TSI_LO = (0.0, 0.0, -9.0, -9.0)
TSI_HI = (10 * math.pi, 10 * math.pi, 9.0, 9.0)
TSI_PAPER_LO = (0.0, 0.0, -6.0, -6.0)
TSI_PAPER_HI = (10 * math.pi, 10 * math.pi, 6.0, 6.0)


@dataclass(frozen=True)
class Workload:
    name: str
    cfg: Config
    kind: int
    params: tuple
    steps: int
    ckpt: int = 0  # checkpoint interval of the adjoint workloads


def _landau(degree, nc, dt, eps, precision="fp64"):
    return Config(degree=degree, ncell=(nc,) * 4, lo=LANDAU_LO, hi=LANDAU_HI, dt=dt,
                  precision=precision)


WORKLOADS = {
    # linear Landau damping, 16^4 cells, degree 1, dt 0.1, 50 steps
    "linear_landau_16": Workload("linear_landau_16", _landau(1, 16, 0.1, 0.01), N.SLDG_INIT_LANDAU,
                                 (0.01, 0.5, 0.5), 50),
    # nonlinear Landau damping, 64^4 cells, degree 2 (1.36e9 dofs), dt 0.05 to T = 20
    "nonlinear_landau_64": Workload("nonlinear_landau_64", _landau(2, 64, 0.05, 0.5),
                                    N.SLDG_INIT_LANDAU, (0.5, 0.5, 0.5), 400),
    # the same problem at 48^4 cells (4.3e8 dofs: larger than L2, a few GB) for
    # profiling captures
    "nonlinear_landau_48": Workload("nonlinear_landau_48", _landau(2, 48, 0.05, 0.5),
                                    N.SLDG_INIT_LANDAU, (0.5, 0.5, 0.5), 400),
    # the 64^4 workload's x-grid with 32^2 v-cells (3.4e8 dofs, 2.7 GB FP64): same x1
    # and x2 lines as the bench workload, for profiling captures
    "nonlinear_landau_64x32": Workload(
        "nonlinear_landau_64x32",
        Config(degree=2, ncell=(64, 64, 32, 32), lo=LANDAU_LO, hi=LANDAU_HI, dt=0.05),
        N.SLDG_INIT_LANDAU, (0.5, 0.5, 0.5), 400),
    # two-stream instability, 64^2 x 128^2 cells, degree 2 (5.4e9 dofs), dt 0.05 to T = 40
    "two_stream_64x128": Workload(
        "two_stream_64x128",
        Config(degree=2, ncell=(64, 64, 128, 128), lo=TSI_LO, hi=TSI_HI, dt=0.05),
        N.SLDG_INIT_TWO_STREAM, (1e-3, 0.2, 3.0), 800),
    # the two-stream workload's x-grid (64^2 cells, degree 2: the same x-planes
    # and x-lines) with 16^2 v-cells (8.5e7 dofs, 0.68 GB FP64, larger than
    # L2) for profiling captures
    "two_stream_64x16": Workload(
        "two_stream_64x16",
        Config(degree=2, ncell=(64, 64, 16, 16), lo=TSI_LO, hi=TSI_HI, dt=0.05),
        N.SLDG_INIT_TWO_STREAM, (1e-3, 0.2, 3.0), 800),
    # the paper's dG4 (degree 3) runs of Sec. 4 and Table 1: nonlinear Landau
    # damping, dt 0.1 to T = 50, at 64, 128 and 144 nodal values per direction
    "landau_dg4_16": Workload("landau_dg4_16", _landau(3, 16, 0.1, 0.5), N.SLDG_INIT_LANDAU,
                              (0.5, 0.5, 0.5), 500),
    "landau_dg4_32": Workload("landau_dg4_32", _landau(3, 32, 0.1, 0.5), N.SLDG_INIT_LANDAU,
                              (0.5, 0.5, 0.5), 500),
    "landau_dg4_36": Workload("landau_dg4_36", _landau(3, 36, 0.1, 0.5), N.SLDG_INIT_LANDAU,
                              (0.5, 0.5, 0.5), 500),
    # the paper's two-stream instability (Sec. 5, Eq. (iv-tsi): eps 1e-3, k 0.2,
    # v0 2.4 on [0, 10 pi]^2 x [-6, 6]^2), dG4 at 32, 64 and 128 nodal values
    # per direction, dt 0.1 to T = 250 (quiescent to t ~ 175, growth to ~ 225)
    **{f"two_stream_paper_dg4_{nc}": Workload(
        f"two_stream_paper_dg4_{nc}",
        Config(degree=3, ncell=(nc,) * 4, lo=TSI_PAPER_LO, hi=TSI_PAPER_HI, dt=0.1),
        N.SLDG_INIT_TWO_STREAM_PAPER, (1e-3, 0.2, 2.4), 2500) for nc in (8, 16, 32)},
    # the cubic-spline comparison method of Sec. 3 (Table 1: 64 and 128 grid
    # points per direction) on nonlinear Landau damping, dt 0.1, periodic v
    **{f"spline_landau_{n}": Workload(
        f"spline_landau_{n}",
        Config(degree=0, ncell=(n,) * 4, lo=LANDAU_LO, hi=LANDAU_HI, dt=0.1, vbc=1,
               flags=N.SLDG_FLAG_SPLINE),
        N.SLDG_INIT_LANDAU, (0.5, 0.5, 0.5), 500) for n in (64, 128)},
    # adjoint of nonlinear Landau damping, 32^4 cells, degree 1, dt 0.1, 100 steps, ckpt 10
    "adjoint_landau_32": Workload("adjoint_landau_32", _landau(1, 32, 0.1, 0.5), N.SLDG_INIT_LANDAU,
                                  (0.5, 0.5, 0.5), 100, ckpt=10),
    # mixed precision forward+adjoint, 128^4 cells, degree 1 (4.3e9 dofs), fp32 f
    "mixed_landau_128": Workload("mixed_landau_128", _landau(1, 128, 0.05, 0.5, "fp32"),
                                 N.SLDG_INIT_LANDAU, (0.5, 0.5, 0.5), 200, ckpt=25),
    # its x-planes and x-lines (128^2 x-cells, degree 1) over 16^2 v-cells:
    # 6.7e7 dofs, 268 MB in FP32 (beyond L2), the profiling case of that grid
    "mixed_landau_128x16": Workload(
        "mixed_landau_128x16",
        Config(degree=1, ncell=(128, 128, 16, 16), lo=LANDAU_LO, hi=LANDAU_HI, dt=0.05,
               precision="fp32"),
        N.SLDG_INIT_LANDAU, (0.5, 0.5, 0.5), 200),
}


def workload(name: str, precision: str | None = None, flags: int = 0) -> Workload:
    """The named workload, in another storage precision and with more
    configuration flags (added to the workload's own) if given."""
    w = WORKLOADS[name]
    flags = flags | w.cfg.flags
    if (precision is None or precision == w.cfg.precision) and flags == w.cfg.flags:
        return w
    c = w.cfg
    return Workload(w.name, Config(c.degree, c.ncell, c.lo, c.hi, c.dt, precision or c.precision,
                                   c.vbc, c.poisson_kmax, flags), w.kind, w.params, w.steps,
                    w.ckpt)
