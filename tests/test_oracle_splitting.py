"""The oracle's splitting compositions (order 2: the Strang step of Sec. 2;
order 4: the triple jump of Strang steps; merged drifts), pinned against
mathematics that does not come from the oracle.

- The stage fractions of one order-4 step are the tabulated triple-jump
  weights.
- On a pendulum split into its two exactly solvable flows (drift x' = v, kick
  v' = -sin x; the same splitting as Vlasov-Poisson in one particle), the
  oracle's stage lists converge at orders 2 and 4 to an adaptive
  high-order ODE solution, and merged drifts give the unmerged result
  (exact drifts compose exactly).
- In 4D: free streaming at order 4 keeps the closed-form density, and
  linear Landau damping at order 4 with a larger step damps at the rate of
  the dispersion relation.
"""
import numpy as np
import pytest

from conftest import golden_kv
from inputs import LANDAU_HI, LANDAU_LO


def test_order4_weights_are_the_triple_jump(orc):
    ref = golden_kv("triple_jump_weights.txt")
    kind, frac = orc.split_stages(4, 1)
    assert list(kind) == [0, 2, 0, 0, 1, 0, 0, 1, 0]
    kicks = frac[kind != 0]
    tol = ref["abs_tol"]
    assert abs(kicks[0] - ref["w1"]) < tol and abs(kicks[1] - ref["w0"]) < tol
    assert abs(kicks[2] - ref["w1"]) < tol
    np.testing.assert_allclose(frac[kind == 0], np.repeat(kicks, 2) / 2, rtol=0, atol=tol)
    # the order-2 list is the Strang step
    kind, frac = orc.split_stages(2, 2)
    assert list(kind) == [0, 2, 0, 0, 2, 0] and list(frac) == [0.5, 1.0, 0.5] * 2


def _pendulum(orc, order, merge, tau, T, y0):
    x, v = y0
    n = int(round(T / tau))
    kind, frac = orc.split_stages(order, n, merge)
    for k, fr in zip(kind, frac):
        if k == 0:
            x = x + fr * tau * v
        else:
            v = v - fr * tau * np.sin(x)
    return np.array([x, v])


def _pendulum_exact(y0, T):
    from scipy.integrate import solve_ivp

    r = solve_ivp(lambda t, y: [y[1], -np.sin(y[0])], (0, T), y0, method="DOP853", rtol=1e-13,
                  atol=1e-14)
    return r.y[:, -1]


@pytest.mark.parametrize("order", [2, 4])
def test_pendulum_convergence_order_and_merge(orc, order):
    y0, T = (1.0, 0.5), 4.0
    ex = _pendulum_exact(y0, T)
    errs = []
    for tau in (0.2, 0.1, 0.05):
        a = _pendulum(orc, order, False, tau, T, y0)
        b = _pendulum(orc, order, True, tau, T, y0)
        assert np.abs(a - b).max() < 1e-12
        errs.append(np.abs(a - ex).max())
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(rates - order) < 0.25), (errs, rates)


def _grid(orc, deg, nc, dt):
    return orc.Grid(deg=deg, nc=nc, lo=LANDAU_LO, hi=LANDAU_HI, dt=dt)


@pytest.mark.parametrize("merge", [False, True])
def test_order4_free_streaming_density_closed_form(orc, merge):
    # as for the Strang step: rho(t, x1) = base (1 + eps exp(-k^2 t^2/2) cos(k x1)/(1+eps))
    g = _grid(orc, 2, (16, 1, 24, 8), dt=0.5)
    eps, k = 0.05, 0.5
    f0 = orc.init(g, orc.LANDAU, [eps, k, 0.0])
    nsteps = 4
    f, _, _, _ = orc.step_split(g, f0, nsteps, order=4, merge=merge, kick=False)
    t = nsteps * g.dt
    r = orc.rho(g, f)
    base = orc.rho(g, f0).mean()
    X1 = np.broadcast_to(g.nodes(0), r.shape)
    expect = base + eps * np.exp(-(k * t) ** 2 / 2) * np.cos(k * X1) * (base / (1 + eps))
    np.testing.assert_allclose(r, expect, rtol=0, atol=5e-4 * eps)
    # drift weights summing to anything but one step per step move the
    # damping factor exp(-k^2 t^2/2) by far more than the tolerance
    wrong = base + eps * np.exp(-(k * 1.1 * t) ** 2 / 2) * np.cos(k * X1) * (base / (1 + eps))
    assert np.abs(wrong - expect).max() > 20 * 5e-4 * eps


def test_order4_strang_order2_are_the_same_step(orc):
    # order 2 through the stage executor is the oracle's Strang step
    g = _grid(orc, 1, (6, 5, 6, 7), dt=0.2)
    f0 = orc.init(g, orc.LANDAU, [0.5, 0.5, 0.5])
    a, Wa, _, _ = orc.step(g, f0, 3)
    b, Wb, _, _ = orc.step_split(g, f0, 3, order=2)
    assert np.array_equal(a, b) and np.array_equal(Wa, Wb)


def test_order4_linear_landau_damping_rate(orc):
    # as the Strang test: W ~ exp(2 gamma t) cos^2(omega t + phi), here with
    # the order-4 composition at a 2.5x larger step
    from test_oracle_step import _dispersion_root

    om, ga = _dispersion_root(0.5)
    g = _grid(orc, 1, (16, 16, 32, 32), dt=0.25)
    f0 = orc.init(g, orc.LANDAU, [0.01, 0.5, 0.5])
    n = 82
    _, W, _, _ = orc.step_split(g, f0, n, order=4)
    # W of step m is taken at its first kick, after the drift g1 tau / 2
    g1 = 1.0 / (2.0 - 2.0 ** (1.0 / 3.0))
    t = (np.arange(n) + 0.5 * g1) * g.dt
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
