"""Pins of the oracle's 1D advection and 4D sweeps (Sec. 2-3, Eq. (AB-sldg)).

Checks that fix the sweep from outside: an integer-cell shift is an exact
cyclic permutation; a polynomial of degree l is translated exactly (the
projection is the only approximation, Sec. 2); periodic mass is conserved
(Sec. 1); only the two cells i*, i*+1 feed an output cell (Sec. 3); the
direction of the shift matches u(x - a) of Eq. (1d-advection); and the 4D
sweep shifts each line by its own node velocity (x) or field value (v).
"""
import numpy as np
import pytest

from inputs import LANDAU_HI, LANDAU_LO, random_f, random_field


def _nodes1d(orc, deg, nc, h, lo=0.0):
    xi, _ = orc.gauss_legendre(deg + 1)
    c = np.repeat(np.arange(nc), deg + 1)
    j = np.tile(np.arange(deg + 1), nc)
    return lo + (c + xi[j]) * h


@pytest.mark.parametrize("deg", [0, 1, 2, 3])
@pytest.mark.parametrize("k", [-3, -1, 0, 1, 2, 7])
def test_integer_shift_is_cyclic_permutation(orc, deg, k):
    nc, h = 9, 0.25  # binary h: a/h is exactly k
    u = random_f((nc * (deg + 1),), seed=deg * 10 + k + 50)
    out = orc.advect_line(deg, nc, h, k * h, True, u)
    expect = np.roll(u.reshape(nc, deg + 1), k, axis=0).ravel()
    np.testing.assert_array_equal(out, expect)


@pytest.mark.parametrize("deg", [1, 2, 3])
@pytest.mark.parametrize("a", [0.37, -0.81, 1.93, -2.4])
def test_polynomial_translated_exactly(orc, deg, a):
    # A global polynomial of degree <= l is in the approximation space; its
    # translate is too, so P T u = T u exactly away from the zero inflow.
    nc, h = 12, 0.5
    z = _nodes1d(orc, deg, nc, h)
    coef = np.array([0.3, -1.1, 0.7, 0.25][: deg + 1])
    p = lambda x: np.polyval(coef, x)
    out = orc.advect_line(deg, nc, h, a, False, p(z))
    s = int(np.floor(a / h))
    inner = slice((max(s + 1, 0)) * (deg + 1), (nc + min(s, 0)) * (deg + 1))
    np.testing.assert_allclose(out[inner], p(z - a)[inner], rtol=0, atol=2e-13)


@pytest.mark.parametrize("deg", [0, 1, 2, 3])
@pytest.mark.parametrize("a", [0.123, -0.77, 2.9])
def test_periodic_mass_conservation(orc, deg, a):
    nc, h = 11, 0.25
    _, w = orc.gauss_legendre(deg + 1)
    W = np.tile(w, nc) * h
    u = random_f((nc * (deg + 1),), seed=7 + deg)
    out = orc.advect_line(deg, nc, h, a, True, u)
    assert abs(W @ out - W @ u) < 1e-14 * np.abs(u).sum()


@pytest.mark.parametrize("deg", [1, 2])
@pytest.mark.parametrize("a", [0.31, -0.52, 1.2])
def test_two_cell_stencil(orc, deg, a):
    nc, h, n = 10, 0.4, deg + 1
    s = int(np.floor(a / h))
    for k in range(nc):
        e = np.zeros(nc * n)
        e[k * n:(k + 1) * n] = 1.0
        out = orc.advect_line(deg, nc, h, a, True, e).reshape(nc, n)
        touched = {c for c in range(nc) if np.any(out[c] != 0.0)}
        assert touched <= {(k + s) % nc, (k + s + 1) % nc}


@pytest.mark.parametrize("deg", [1, 2, 3])
def test_shift_direction_and_accuracy(orc, deg):
    # out(x) approximates u(x - a): compare with the exact translate of a
    # smooth periodic function; the wrong sign would give u(x + a).
    nc, L = 32, 2 * np.pi
    h = L / nc
    z = _nodes1d(orc, deg, nc, h)
    a = 0.7
    out = orc.advect_line(deg, nc, h, a, True, np.sin(z))
    err = np.abs(out - np.sin(z - a)).max()
    assert err < 5e-3 ** (deg / 2 + 0.5)
    assert np.abs(out - np.sin(z + a)).max() > 0.5


@pytest.mark.parametrize("deg", [1, 2, 3])
def test_convergence_order(orc, deg):
    # Repeated translation of a smooth periodic profile: error ~ h^(l+1)
    # (Sec. 3: "the resulting scheme has order l+1").
    L, T, steps = 2 * np.pi, 1.0, 10
    errs = []
    for nc in (8, 16, 32):
        h = L / nc
        z = _nodes1d(orc, deg, nc, h)
        u = np.exp(np.sin(z))
        for _ in range(steps):
            u = orc.advect_line(deg, nc, h, T / steps, True, u)
        errs.append(np.abs(u - np.exp(np.sin(z - T))).max())
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates[-1] > deg + 1 - 0.35, (errs, rates)


def _grid(orc, deg=1, nc=(4, 5, 6, 3), vbc=0, dt=0.37):
    return orc.Grid(deg=deg, nc=nc, lo=LANDAU_LO, hi=LANDAU_HI, dt=dt, vbc=vbc)


@pytest.mark.parametrize("d", [0, 1, 2, 3])
@pytest.mark.parametrize("vbc", [0, 1])
def test_4d_sweep_shifts_each_line_by_its_parameter(orc, d, vbc):
    # The 4D sweep is the 1D advection along direction d with shift
    # v1*dt*frac (d=0), v2*dt*frac (d=1), E1(x)*dt*frac (d=2), E2(x)*dt*frac (d=3);
    # shifts are taken from numpy's node coordinates, lines from numpy axes.
    g = _grid(orc, vbc=vbc)
    f = random_f(g.shape, seed=11 + d)
    Ed = random_field(g.xshape, seed=3 + d, scale=3.0) if d >= 2 else None
    frac = 0.5 if d < 2 else 1.0
    out = orc.sweep(g, d, f, Ed=Ed, frac=frac).reshape(g.shape)
    F = f.reshape(g.shape)
    axis = 3 - d  # numpy axis of direction d in (v2, v1, x2, x1)
    xs = np.moveaxis(F, axis, -1)
    ys = np.moveaxis(out, axis, -1)
    x1n, x2n, v1n, v2n = (np.asarray(x) for x in (
        np.arange(g.D(0)), np.arange(g.D(1)), g.nodes(2), g.nodes(3)))
    periodic = d < 2 or vbc == 1
    for idx in np.ndindex(xs.shape[:-1]):
        full = list(idx)
        full.insert(axis, None)  # position along d
        i_v2, i_v1, i_x2, i_x1 = full
        if d == 0:
            a = v1n[i_v1] * g.dt * frac
        elif d == 1:
            a = v2n[i_v2] * g.dt * frac
        else:
            a = Ed[i_x2, i_x1] * g.dt * frac
        line = orc.advect_line(g.deg, g.nc[d], g.h(d), a, periodic, xs[idx])
        np.testing.assert_array_equal(ys[idx], line)


def test_v_sweep_zero_inflow_loses_mass_only_at_boundary(orc):
    # With zero inflow, a shift that moves mass out of [-vmax, vmax] loses
    # exactly the outflowing cells' mass; with periodic v, none.
    g = _grid(orc, deg=2, nc=(2, 2, 8, 2), vbc=1)
    f = (np.abs(random_f(g.shape, seed=5)) + 0.1).ravel()
    E = np.full(g.xshape, 0.9 * g.h(2) / g.dt)
    W = np.einsum("a,b,c,d->abcd", g.weights(3), g.weights(2), g.weights(1), g.weights(0)).ravel()
    out = orc.sweep(g, 2, f, Ed=E)
    assert abs(W @ out - W @ f) < 1e-13 * (W @ f)
    g0 = _grid(orc, deg=2, nc=(2, 2, 8, 2), vbc=0)
    out0 = orc.sweep(g0, 2, f, Ed=E)
    assert W @ out0 < W @ f - 1e-3
