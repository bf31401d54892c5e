"""The oracle's cubic-spline advection (the spline method of Sec. 3: the
periodic cubic B-spline interpolant of the point values, evaluated at the
shifted points), pinned against mathematics and libraries that do not come
from the oracle.

- Against scipy's periodic CubicSpline (the same unique periodic cubic
  interpolant, built by a different algorithm) for shifts of either sign,
  fractional and integer, and beyond one period.
- Integer shifts are permutations; the sum of the point values is
  conserved (the B-splines are a partition of unity and the system's
  columns sum to one); a smooth wave is advected with fourth-order error.
- In 4D on a degree-0 grid (one point per cell, periodic v), free
  streaming keeps the closed-form density.
"""
import math

import numpy as np
import pytest

from inputs import rng


def _scipy_shift(u, L, a):
    from scipy.interpolate import CubicSpline

    n = u.size
    x = np.arange(n) * (L / n)
    cs = CubicSpline(np.append(x, L), np.append(u, u[0]), bc_type="periodic")
    return cs(np.mod(x - a, L))


@pytest.mark.parametrize("n", [3, 8, 37, 128])
def test_spline_line_matches_scipy_periodic_spline(orc, n):
    L = 3.0
    h = L / n
    u = rng(n).standard_normal(n)
    for sig in (0.0, 0.31, -0.77, 1.5, -2.25, 4.0, n + 0.4, -3 * n - 0.6):
        out = orc.spline_line(h, sig * h, u)
        ref = _scipy_shift(u, L, sig * h)
        assert np.abs(out - ref).max() < 1e-13 * np.abs(u).max(), sig


def test_spline_coefficients_solve_the_cyclic_system(orc):
    # (w_{i-1} + 4 w_i + w_{i+1})/6 = u_i, checked with a dense solve
    n = 11
    u = rng(5).standard_normal(n)
    M = np.zeros((n, n))
    for i in range(n):
        M[i, i] = 4 / 6
        M[i, (i - 1) % n] += 1 / 6
        M[i, (i + 1) % n] += 1 / 6
    np.testing.assert_allclose(orc.spline_coeffs(u), np.linalg.solve(M, u), rtol=0, atol=1e-14)


def test_integer_shift_is_a_permutation_and_sum_is_conserved(orc):
    n, h = 40, 0.1
    u = rng(7).standard_normal(n)
    for s in (-3, 0, 1, 17, 45):
        np.testing.assert_allclose(orc.spline_line(h, s * h, u), np.roll(u, s), rtol=0, atol=1e-14)
    for sig in (0.5, -1.3, 7.9):
        assert abs(orc.spline_line(h, sig * h, u).sum() - u.sum()) < 1e-13 * np.abs(u).sum()


def test_fourth_order_advection_of_a_wave(orc):
    # the shift is 2.5 points at every resolution (theta = 1/2, where the
    # interpolation error is largest)
    L = 2 * math.pi
    errs = []
    for n in (16, 32, 64):
        x = np.arange(n) * (L / n)
        a = 2.5 * L / n
        out = orc.spline_line(L / n, a, np.sin(3 * x))
        errs.append(np.abs(out - np.sin(3 * (x - a))).max())
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 3.7), (errs, rates)


def test_spline_free_streaming_density_closed_form(orc):
    from inputs import LANDAU_HI, LANDAU_LO

    g = orc.Grid(deg=0, nc=(32, 4, 48, 8), lo=LANDAU_LO, hi=LANDAU_HI, dt=0.25, vbc=1, spline=1)
    eps, k = 0.05, 0.5
    f0 = orc.init(g, orc.LANDAU, [eps, k, 0.0])
    nsteps = 8
    f, _, _, _ = orc.step(g, f0, nsteps, kick=False)
    t = nsteps * g.dt
    r = orc.rho(g, f)
    base = orc.rho(g, f0).mean()
    X1 = np.broadcast_to(g.nodes(0), r.shape)
    expect = base + eps * np.exp(-(k * t) ** 2 / 2) * np.cos(k * X1) * (base / (1 + eps))
    np.testing.assert_allclose(r, expect, rtol=0, atol=2e-4 * eps)


def test_spline_grid_needs_periodic_lines_of_three(orc):
    from inputs import LANDAU_HI, LANDAU_LO

    g = orc.Grid(deg=0, nc=(8, 4, 6, 6), lo=LANDAU_LO, hi=LANDAU_HI, dt=0.1, vbc=0, spline=1)
    f = orc.init(g, orc.LANDAU, [0.1, 0.5, 0.5])
    with pytest.raises(ValueError):
        orc.sweep(g, 2, f, Ed=np.zeros(g.xshape))
    g = orc.Grid(deg=0, nc=(8, 2, 6, 6), lo=LANDAU_LO, hi=LANDAU_HI, dt=0.1, vbc=1, spline=1)
    with pytest.raises(ValueError):
        orc.sweep(g, 1, orc.init(g, orc.LANDAU, [0.1, 0.5, 0.5]))
