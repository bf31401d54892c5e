"""Pins of the oracle's Strang step (Sec. 2) against physics it must reproduce.

- Free streaming (field off): every line is translated exactly in the
  continuum, so rho(t) has the closed form 1 + eps exp(-k^2 t^2/2)(...) and
  the nodal values converge to f0(x - v t, v).
- Linear Landau damping (eps = 0.01, k = 0.5): the decay rate and frequency
  of the electric energy match the root of the dispersion relation
  1 + (1 + zeta Z(zeta))/k^2 = 0, solved here with scipy's Faddeeva function.
- Mass is conserved to round-off with periodic v (Sec. 1).
- Nonlinear Landau damping at tau = 0.1 keeps the energy error near 1e-3
  (Sec. 4), a loose band.
"""
import numpy as np
import pytest

from conftest import golden_kv
from inputs import LANDAU_HI, LANDAU_LO


def _grid(orc, deg, nc, dt, vbc=0):
    return orc.Grid(deg=deg, nc=nc, lo=LANDAU_LO, hi=LANDAU_HI, dt=dt, vbc=vbc)


def test_free_streaming_density_closed_form(orc):
    # rho(t,x) = int f0(x - v t, v) dv = 1 + eps exp(-k^2 t^2/2) cos(k x1)
    # (+ the constant eps from k2 = 0), for the Gaussian in v.
    g = _grid(orc, 2, (16, 1, 24, 8), dt=0.25)
    eps, k = 0.05, 0.5
    f0 = orc.init(g, orc.LANDAU, [eps, k, 0.0])
    nsteps = 8
    f, _, _, _ = orc.step(g, f0, nsteps, kick=False)
    t = nsteps * g.dt
    r = orc.rho(g, f)
    r0 = orc.rho(g, f0)
    base = r0.mean()  # discrete Gaussian mass times (1 + eps), identical at all times
    X1 = np.broadcast_to(g.nodes(0), r.shape)
    expect = base + eps * np.exp(-(k * t) ** 2 / 2) * np.cos(k * X1) * (base / (1 + eps))
    np.testing.assert_allclose(r, expect, rtol=0, atol=2e-4 * eps)
    # a wrong sign of the x-shift or of t would not damp the mode
    assert np.abs(r - base).max() < 0.7 * eps


@pytest.mark.parametrize("deg", [1, 2])
def test_free_streaming_nodal_convergence(orc, deg):
    # f(t) = f0(x - v t, v) at the nodes; error decreases at order >= l+1 in x
    # (v is not advected when the field is off).
    eps, k, T = 0.3, 0.5, 1.0
    errs = []
    for ncx in (8, 16):
        g = _grid(orc, deg, (ncx, ncx, 4, 4), dt=T / 4)
        f0 = orc.init(g, orc.LANDAU, [eps, k, k])
        f, _, _, _ = orc.step(g, f0, 4, kick=False)
        V2, V1, X2, X1 = np.meshgrid(g.nodes(3), g.nodes(2), g.nodes(1), g.nodes(0), indexing="ij")
        ex = (1 + eps * (np.cos(k * (X1 - V1 * T)) + np.cos(k * (X2 - V2 * T)))) * \
            np.exp(-(V1 ** 2 + V2 ** 2) / 2) / (2 * np.pi)
        errs.append(np.abs(f.reshape(g.shape) - ex).max())
    rate = np.log2(errs[0] / errs[1])
    assert rate > deg + 1 - 0.4, (errs, rate)


def _dispersion_root(k):
    from scipy.optimize import fsolve
    from scipy.special import wofz

    def F(z):
        w = z[0] + 1j * z[1]
        zeta = w / (k * np.sqrt(2))
        Z = 1j * np.sqrt(np.pi) * wofz(zeta)
        r = 1 + (1 + zeta * Z) / k ** 2
        return [r.real, r.imag]

    w = fsolve(F, [1.4, -0.15], xtol=1e-14)
    return w[0], w[1]


def test_dispersion_root_textbook_value():
    ref = golden_kv("landau_dispersion_k05.txt")
    om, ga = _dispersion_root(ref["k"])
    assert abs(om - ref["omega_r"]) < ref["abs_tol"] and abs(ga - ref["gamma"]) < ref["abs_tol"]


def test_linear_landau_damping_rate(orc):
    # 2D2V linear Landau damping: the (1,0) and (0,1) modes each damp at the
    # 1D rate; W ~ exp(2 gamma t) cos^2(omega t + phi).  The v-grid has 32
    # cells (h_v = 0.375) so the resonant velocity omega/k ~ 2.8 is resolved.
    om, ga = _dispersion_root(0.5)
    g = _grid(orc, 1, (16, 16, 32, 32), dt=0.1)
    f0 = orc.init(g, orc.LANDAU, [0.01, 0.5, 0.5])
    n = 205
    _, W, _, _ = orc.step(g, f0, n)
    t = (np.arange(n) + 0.5) * g.dt  # the field is taken after the first half drift
    lw = np.log(W)
    tp, lp = [], []
    for i in range(1, n - 1):
        if lw[i] > lw[i - 1] and lw[i] > lw[i + 1] and 1.0 <= t[i] <= 20.0:
            a, b, c = lw[i - 1], lw[i], lw[i + 1]
            d = 0.5 * (a - c) / (a - 2 * b + c)
            tp.append(t[i] + d * g.dt)
            lp.append(b - 0.25 * (a - c) * d)
    slope = np.polyfit(tp, lp, 1)[0]
    assert abs(slope / 2 - ga) < 0.005, (slope / 2, ga)
    assert abs(np.pi / np.mean(np.diff(tp)) - om) < 0.01


def test_mass_conserved_with_periodic_v(orc):
    g = _grid(orc, 2, (6, 5, 6, 7), dt=0.2, vbc=1)
    f0 = orc.init(g, orc.LANDAU, [0.5, 0.5, 0.5])
    f, _, _, _ = orc.step(g, f0, 5)
    m0 = orc.diagnostics(g, f0)["mass"]
    m1 = orc.diagnostics(g, f)["mass"]
    assert abs(m1 - m0) < 1e-13 * m0


def test_nonlinear_landau_energy_error_band(orc):
    # Sec. 4: at tau = 0.1 the relative error in the total energy is of order
    # 1e-3 after the transient and comes from the time integration: within a
    # factor 3 of that order here (6.2e-4 on this grid, the same to 2% on
    # grids up to 16^2 x 24^2 cells), and halving tau over the same time span
    # divides it by about 4 (the second order of Strang splitting; a
    # spatial error would not shrink with tau).
    ref = golden_kv("nonlinear_landau_energy_error.txt")

    def energy_error(tau, nsteps):
        g = _grid(orc, 2, (8, 8, 16, 16), dt=tau)
        f0 = orc.init(g, orc.LANDAU, [ref["eps"], ref["k"], ref["k"]])
        _, E1, E2 = orc.fields(g, f0)
        d0 = orc.diagnostics(g, f0, E1, E2)
        f, _, _, _ = orc.step(g, f0, nsteps)
        _, E1, E2 = orc.fields(g, f)
        d1 = orc.diagnostics(g, f, E1, E2)
        return abs(d1["total"] - d0["total"]) / d0["total"]

    err = energy_error(ref["tau"], 40)
    order = ref["energy_error_order"]
    assert order / 3 < err < 3 * order, err
    ratio = energy_error(ref["tau"] / 2, 80) / err
    assert 1 / 5 < ratio < 1 / 3, ratio
