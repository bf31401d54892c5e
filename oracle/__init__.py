"""Plain FP64 CPU oracle of the SLDG Vlasov-Poisson step (arXiv 1803.02143).

TEST INFRASTRUCTURE ONLY.  The oracle is the independent checker of the CUDA
library: only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU
baseline / reference arm may import it.  It shares no code with the CUDA path
(``paper_1803_02143_gb300``) and neither side imports the other.

The arithmetic lives in ``sldg_oracle.c`` (plain C, FP64, every function
citing the section or equation of the paper it follows); this module only
compiles it with gcc and marshals numpy arrays through ctypes.

Parity pins (see ``tests/test_oracle_*.py``): Gauss-Legendre nodes against
numpy and closed forms; the projection matrices against exact rational
polynomial integration (40-digit mpmath), donor-cell upwinding at degree 0, the identity at
theta = 0 and 1, the column mass identity and finite differences of their
theta-derivatives; the sweep against integer-cell permutation, polynomial
reproduction, mass conservation and the two-cell stencil; the Poisson map
against closed-form fields; the full step against the free-streaming closed
form, the convergence order l+1 and the linear Landau damping rate from the
dispersion relation; the adjoint against dot-product identities and central
finite differences; the splitting compositions (order 4, merged drifts)
against the tabulated triple-jump weights, the convergence orders of an
exactly split pendulum, free streaming and linear Landau damping; the
cubic-spline advection against scipy's periodic CubicSpline, a dense
solve of its cyclic system, permutations, conservation, fourth-order
convergence and free streaming.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sldg_oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile ``sldg_oracle.c`` into ``liboracle.so`` (gcc, OpenMP if present).

    ``-ffp-contract=off`` keeps every multiply and add separately rounded on
    both x86-64 and aarch64, so the oracle gives the same bits on both hosts.
    """
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    base = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off",
            "-fno-fast-math", _SRC, "-o", _SO + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_SO + ".tmp", _SO)
    return _SO


class _CGrid(ctypes.Structure):
    _fields_ = [
        ("deg", ctypes.c_int),
        ("nc", ctypes.c_int * 4),
        ("lo", ctypes.c_double * 4),
        ("hi", ctypes.c_double * 4),
        ("dt", ctypes.c_double),
        ("vbc", ctypes.c_int),
        ("kmax", ctypes.c_int),
        ("spline", ctypes.c_int),
    ]


_DP = ctypes.POINTER(ctypes.c_double)
_IP = ctypes.POINTER(ctypes.c_int)


def _lib_handle():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        G = ctypes.POINTER(_CGrid)
        sig = {
            "orc_gauss_legendre": (ctypes.c_int, [ctypes.c_int, _DP, _DP]),
            "orc_lagrange": (ctypes.c_double, [ctypes.c_int, _DP, ctypes.c_int, ctypes.c_double]),
            "orc_lagrange_d": (ctypes.c_double, [ctypes.c_int, _DP, ctypes.c_int, ctypes.c_double]),
            "orc_matrices": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, _DP, _DP, _DP, _DP]),
            "orc_advect_line": (None, [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_int, _DP, _DP]),
            "orc_advect_line_adj": (None, [ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_int, _DP, _DP]),
            "orc_advect_line_dshift": (ctypes.c_double, [ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                                         ctypes.c_double, ctypes.c_int, _DP, _DP]),
            "orc_numel": (ctypes.c_long, [G]),
            "orc_sweep": (ctypes.c_int, [G, ctypes.c_int, _DP, ctypes.c_double, _DP, _DP]),
            "orc_sweep_adj": (ctypes.c_int, [G, ctypes.c_int, _DP, ctypes.c_double, _DP, _DP, _DP,
                                             _DP]),
            "orc_rho": (ctypes.c_int, [G, _DP, _DP]),
            "orc_rho_adj": (ctypes.c_int, [G, _DP, _DP]),
            "orc_rho_column": (ctypes.c_double, [G, _DP]),
            "orc_poisson": (ctypes.c_int, [G, _DP, _DP, _DP]),
            "orc_poisson_adj": (ctypes.c_int, [G, _DP, _DP, _DP]),
            "orc_electric_energy": (ctypes.c_double, [G, _DP, _DP]),
            "orc_diagnostics": (ctypes.c_int, [G, _DP, _DP, _DP, _DP]),
            "orc_init": (ctypes.c_int, [G, ctypes.c_int, _DP, _DP]),
            "orc_step": (ctypes.c_int, [G, _DP, ctypes.c_int, ctypes.c_int, _DP, _DP, _DP]),
            "orc_fields_of": (ctypes.c_int, [G, _DP, _DP, _DP, _DP]),
            "orc_spline_coeffs": (ctypes.c_int, [ctypes.c_long, _DP, _DP]),
            "orc_spline_line": (ctypes.c_int, [ctypes.c_long, ctypes.c_double, ctypes.c_double,
                                               _DP, _DP]),
            "orc_split_stages": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _IP,
                                                _DP, ctypes.c_int]),
            "orc_step_split": (ctypes.c_int, [G, _DP, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                              ctypes.c_int, _DP, _DP, _DP]),
            "orc_backward": (ctypes.c_int, [G, _DP, ctypes.c_int, ctypes.c_int, _DP, _DP, _DP,
                                            _DP]),
            "orc_threads": (ctypes.c_int, []),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _p(a):
    """Pointer to a C-contiguous float64 numpy array (or NULL for None)."""
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_DP)


@dataclass
class Grid:
    """Phase-space grid: directions x1, x2, v1, v2; ``deg`` is the degree l."""

    deg: int
    nc: tuple
    lo: tuple
    hi: tuple
    dt: float
    vbc: int = 0
    kmax: int = -1
    spline: int = 0  # 1: cubic-spline sweeps (degree 0, periodic v)
    _c: _CGrid = field(default=None, repr=False, compare=False)

    def c(self):
        g = _CGrid()
        g.deg = self.deg
        for d in range(4):
            g.nc[d] = int(self.nc[d])
            g.lo[d] = float(self.lo[d])
            g.hi[d] = float(self.hi[d])
        g.dt = float(self.dt)
        g.vbc = int(self.vbc)
        g.kmax = int(self.kmax)
        g.spline = int(self.spline)
        self._c = g
        return ctypes.byref(g)

    @property
    def n(self):
        return self.deg + 1

    def D(self, d):
        return self.nc[d] * self.n

    @property
    def shape(self):
        """numpy shape of f: (v2, v1, x2, x1)."""
        return (self.D(3), self.D(2), self.D(1), self.D(0))

    @property
    def xshape(self):
        return (self.D(1), self.D(0))

    def h(self, d):
        return (self.hi[d] - self.lo[d]) / self.nc[d]

    def nodes(self, d):
        xi, _ = gauss_legendre(self.n)
        c = np.repeat(np.arange(self.nc[d]), self.n)
        j = np.tile(np.arange(self.n), self.nc[d])
        return self.lo[d] + (c + xi[j]) * self.h(d)

    def weights(self, d):
        _, w = gauss_legendre(self.n)
        return np.tile(w, self.nc[d]) * self.h(d)


def threads() -> int:
    return _lib_handle().orc_threads()


def gauss_legendre(n: int):
    xi = np.zeros(n)
    w = np.zeros(n)
    if _lib_handle().orc_gauss_legendre(n, _p(xi), _p(w)) != 0:
        raise ValueError("unsupported node count")
    return xi, w


def lagrange(n, j, t, derivative=False):
    xi, _ = gauss_legendre(n)
    fn = _lib_handle().orc_lagrange_d if derivative else _lib_handle().orc_lagrange
    return fn(n, _p(xi), j, float(t))


def matrices(deg: int, theta: float, deriv: bool = False):
    n = deg + 1
    A = np.zeros((n, n))
    B = np.zeros((n, n))
    dA = np.zeros((n, n)) if deriv else None
    dB = np.zeros((n, n)) if deriv else None
    _lib_handle().orc_matrices(deg, float(theta), _p(A), _p(B), _p(dA), _p(dB))
    return (A, B, dA, dB) if deriv else (A, B)


def advect_line(deg, nc, h, a, periodic, u):
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.zeros_like(u)
    _lib_handle().orc_advect_line(deg, nc, float(h), float(a), int(periodic), _p(u), _p(out))
    return out


def advect_line_adj(deg, nc, h, a, periodic, lam):
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    out = np.zeros_like(lam)
    _lib_handle().orc_advect_line_adj(deg, nc, float(h), float(a), int(periodic), _p(lam), _p(out))
    return out


def advect_line_dshift(deg, nc, h, a, periodic, lam, u):
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    return _lib_handle().orc_advect_line_dshift(deg, nc, float(h), float(a), int(periodic),
                                                 _p(lam), _p(u))


def _f(g: Grid, f):
    f = np.ascontiguousarray(f, dtype=np.float64)
    assert f.size == int(np.prod(g.shape))
    return f


def sweep(g: Grid, d: int, f, Ed=None, frac: float = 1.0):
    """One 1D sweep along direction d (0..3). Ed is E1 or E2 for d = 2, 3."""
    f = _f(g, f)
    out = np.empty_like(f)
    Ed = None if Ed is None else np.ascontiguousarray(Ed, dtype=np.float64)
    rc = _lib_handle().orc_sweep(g.c(), d, _p(Ed), float(frac), _p(f), _p(out))
    if rc != 0:
        raise ValueError("orc_sweep failed")
    return out


def sweep_adj(g: Grid, d: int, lam, Ed=None, frac: float = 1.0, gfwd=None):
    """Transposed sweep; with gfwd returns (lam_in, Ebar) for v-sweeps."""
    lam = _f(g, lam)
    out = np.empty_like(lam)
    Ed = None if Ed is None else np.ascontiguousarray(Ed, dtype=np.float64)
    Ebar = np.zeros(g.xshape) if gfwd is not None else None
    gfwd = None if gfwd is None else _f(g, gfwd)
    rc = _lib_handle().orc_sweep_adj(g.c(), d, _p(Ed), float(frac), _p(lam), _p(out), _p(gfwd),
                                     _p(Ebar))
    if rc != 0:
        raise ValueError("orc_sweep_adj failed")
    return (out, Ebar) if Ebar is not None else out


def rho(g: Grid, f):
    f = _f(g, f)
    r = np.zeros(g.xshape)
    _lib_handle().orc_rho(g.c(), _p(f), _p(r))
    return r


def rho_column(g: Grid, col):
    """v-quadrature of one x-node's v-plane col (shape (D_v2, D_v1))."""
    c = np.ascontiguousarray(col, dtype=np.float64)
    assert c.size == g.D(2) * g.D(3)
    return _lib_handle().orc_rho_column(g.c(), _p(c))


def rho_adj(g: Grid, rhobar, lam=None):
    lam = np.zeros(g.shape) if lam is None else np.array(lam, dtype=np.float64, copy=True)
    rb = np.ascontiguousarray(rhobar, dtype=np.float64)
    _lib_handle().orc_rho_adj(g.c(), _p(rb), _p(lam))
    return lam


def poisson(g: Grid, rho_):
    r = np.ascontiguousarray(rho_, dtype=np.float64)
    E1 = np.zeros(g.xshape)
    E2 = np.zeros(g.xshape)
    _lib_handle().orc_poisson(g.c(), _p(r), _p(E1), _p(E2))
    return E1, E2


def poisson_adj(g: Grid, E1bar, E2bar):
    a = np.ascontiguousarray(E1bar, dtype=np.float64)
    b = np.ascontiguousarray(E2bar, dtype=np.float64)
    rb = np.zeros(g.xshape)
    _lib_handle().orc_poisson_adj(g.c(), _p(a), _p(b), _p(rb))
    return rb


def electric_energy(g: Grid, E1, E2):
    a = np.ascontiguousarray(E1, dtype=np.float64)
    b = np.ascontiguousarray(E2, dtype=np.float64)
    return _lib_handle().orc_electric_energy(g.c(), _p(a), _p(b))


DIAG_KEYS = ("mass", "l1", "l2sq", "kinetic", "electric", "total")


def diagnostics(g: Grid, f, E1=None, E2=None):
    f = _f(g, f)
    out = np.zeros(6)
    a = None if E1 is None else np.ascontiguousarray(E1, dtype=np.float64)
    b = None if E2 is None else np.ascontiguousarray(E2, dtype=np.float64)
    _lib_handle().orc_diagnostics(g.c(), _p(f), _p(a), _p(b), _p(out))
    return dict(zip(DIAG_KEYS, out.tolist()))


LANDAU, TWO_STREAM, TWO_STREAM_PAPER = 0, 1, 2


def init(g: Grid, kind: int, params):
    f = np.zeros(g.shape)
    p = np.ascontiguousarray(params, dtype=np.float64)
    if _lib_handle().orc_init(g.c(), int(kind), _p(p), _p(f)) != 0:
        raise ValueError("unknown initial value kind")
    return f


def step(g: Grid, f, nsteps: int = 1, kick: bool = True):
    """Advance a copy of f by nsteps Strang steps. Returns (f, W_hist, E1, E2)."""
    f = np.array(_f(g, f), copy=True)
    W = np.zeros(max(nsteps, 1))
    E1 = np.zeros(g.xshape)
    E2 = np.zeros(g.xshape)
    rc = _lib_handle().orc_step(g.c(), _p(f), int(nsteps), int(kick), _p(W), _p(E1), _p(E2))
    if rc != 0:
        raise MemoryError("orc_step failed")
    return f, W[:nsteps], E1, E2


def spline_coeffs(u):
    """B-spline coefficients of the periodic cubic interpolant of u."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    w = np.zeros_like(u)
    if _lib_handle().orc_spline_coeffs(u.size, _p(u), _p(w)) != 0:
        raise ValueError("orc_spline_coeffs failed")
    return w


def spline_line(h: float, a: float, u):
    """The periodic cubic-spline advection of Sec. 3: out_i = u~(x_i - a)."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.empty_like(u)
    if _lib_handle().orc_spline_line(u.size, float(h), float(a), _p(u), _p(out)) != 0:
        raise ValueError("orc_spline_line failed")
    return out


def split_stages(order: int, nsteps: int, merge: bool = False):
    """The stage list of nsteps steps of the splitting of the given order:
    (kinds, fracs), kind 0 = drift, 1 = kick, 2 = first kick of a step."""
    cap = 9 * nsteps + 2
    kind = np.zeros(cap, dtype=np.int32)
    frac = np.zeros(cap)
    n = _lib_handle().orc_split_stages(int(order), int(nsteps), int(bool(merge)),
                                       kind.ctypes.data_as(_IP), _p(frac), cap)
    if n < 0:
        raise ValueError("unsupported splitting order")
    return kind[:n].copy(), frac[:n].copy()


def step_split(g: Grid, f, nsteps: int = 1, order: int = 2, merge: bool = False,
               kick: bool = True):
    """Advance a copy of f by nsteps steps of the order-2 or order-4 splitting,
    optionally with merged drifts. Returns (f, W_hist, E1, E2)."""
    f = np.array(_f(g, f), copy=True)
    W = np.zeros(max(nsteps, 1))
    E1 = np.zeros(g.xshape)
    E2 = np.zeros(g.xshape)
    rc = _lib_handle().orc_step_split(g.c(), _p(f), int(nsteps), int(order), int(bool(merge)),
                                      int(kick), _p(W), _p(E1), _p(E2))
    if rc != 0:
        raise ValueError("orc_step_split failed")
    return f, W[:nsteps], E1, E2


def fields(g: Grid, f):
    f = _f(g, f)
    r = np.zeros(g.xshape)
    E1 = np.zeros(g.xshape)
    E2 = np.zeros(g.xshape)
    _lib_handle().orc_fields_of(g.c(), _p(f), _p(r), _p(E1), _p(E2))
    return r, E1, E2


def backward(g: Grid, f0, nsteps: int, ckpt: int, cW=None):
    """Gradient of J = sum_m cW[m] W(E^m) (cW = dt: time-integrated W).

    Returns (J, grad dJ/df0, W_hist)."""
    f0 = _f(g, f0)
    grad = np.zeros_like(f0)
    J = np.zeros(1)
    W = np.zeros(max(nsteps, 1))
    c = None if cW is None else np.ascontiguousarray(cW, dtype=np.float64)
    rc = _lib_handle().orc_backward(g.c(), _p(f0), int(nsteps), int(ckpt), _p(c), _p(grad),
                                    _p(J), _p(W))
    if rc != 0:
        raise MemoryError("orc_backward failed")
    return float(J[0]), grad, W[:nsteps]


def step_inplace(g: Grid, f, nsteps: int = 1, kick: bool = True):
    """Advance f (float64, C-contiguous, modified in place) by nsteps steps."""
    assert f.dtype == np.float64 and f.flags["C_CONTIGUOUS"]
    rc = _lib_handle().orc_step(g.c(), _p(f), int(nsteps), int(kick), None, None, None)
    if rc != 0:
        raise MemoryError("orc_step failed")
    return f
