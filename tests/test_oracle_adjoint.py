"""Pins of the oracle's adjoint: the transposed sweeps, the shift derivative
of the v-sweeps, and the gradient of the time-integrated electric energy.

Every operator's transpose is checked by the dot-product identity
<lam, S g> = <S^T lam, g>; the shift derivative and the full gradient against
central finite differences of the forward oracle (h = 1e-6), along seeded
random directions and for the perturbation amplitude eps.
"""
import numpy as np
import pytest

from inputs import LANDAU_HI, LANDAU_LO, random_f, random_field


def _grid(orc, deg=1, nc=(4, 5, 6, 4), vbc=0, dt=0.3):
    return orc.Grid(deg=deg, nc=nc, lo=LANDAU_LO, hi=LANDAU_HI, dt=dt, vbc=vbc)


@pytest.mark.parametrize("d", [0, 1, 2, 3])
@pytest.mark.parametrize("vbc", [0, 1])
@pytest.mark.parametrize("deg", [1, 2])
def test_sweep_transpose_dot_product(orc, d, vbc, deg):
    g = _grid(orc, deg=deg, vbc=vbc)
    f = random_f(g.shape, seed=20 + d)
    lam = random_f(g.shape, seed=30 + d)
    Ed = random_field(g.xshape, seed=40 + d, scale=4.0) if d >= 2 else None
    Sf = orc.sweep(g, d, f, Ed=Ed, frac=0.5)
    STl = orc.sweep_adj(g, d, lam, Ed=Ed, frac=0.5)
    lhs, rhs = np.sum(lam * Sf), np.sum(STl * f)
    assert abs(lhs - rhs) < 1e-13 * np.sqrt(np.sum(lam ** 2) * np.sum(f ** 2))


@pytest.mark.parametrize("deg", [1, 2, 3])
@pytest.mark.parametrize("a", [0.37, -0.45, 1.3])
def test_line_shift_derivative_fd(orc, deg, a):
    nc, h = 7, 0.5
    u = random_f((nc * (deg + 1),), seed=1)
    lam = random_f((nc * (deg + 1),), seed=2)
    e = 1e-6
    fp = lam @ orc.advect_line(deg, nc, h, a + e, False, u)
    fm = lam @ orc.advect_line(deg, nc, h, a - e, False, u)
    d = orc.advect_line_dshift(deg, nc, h, a, False, lam, u)
    assert abs(d - (fp - fm) / (2 * e)) < 1e-7 * (abs(d) + 1)


@pytest.mark.parametrize("d", [2, 3])
def test_v_sweep_field_derivative_fd(orc, d):
    # Ebar[x] = d/dE(x) <lam, V(E) g>, checked at a few x-nodes.
    g = _grid(orc, deg=2)
    f = random_f(g.shape, seed=50)
    lam = random_f(g.shape, seed=51)
    E = random_field(g.xshape, seed=52, scale=1.5)
    _, Ebar = orc.sweep_adj(g, d, lam, Ed=E, frac=1.0, gfwd=f)
    e = 1e-6
    for p in [(0, 0), (3, 7), (g.xshape[0] - 1, 2)]:
        Ep, Em = E.copy(), E.copy()
        Ep[p] += e
        Em[p] -= e
        fd = (np.sum(lam * orc.sweep(g, d, f, Ed=Ep)) - np.sum(lam * orc.sweep(g, d, f, Ed=Em))) / (2 * e)
        assert abs(Ebar[p] - fd) < 1e-6 * (abs(fd) + 1), (p, Ebar[p], fd)


def _J(orc, g, f0, n):
    _, W, _, _ = orc.step(g, f0, n)
    return g.dt * W.sum()


@pytest.fixture(scope="module")
def adj_case(orc):
    g = orc.Grid(deg=1, nc=(4, 4, 6, 6), lo=LANDAU_LO, hi=LANDAU_HI, dt=0.1)
    eps, k = 0.5, 0.5
    f0 = orc.init(g, orc.LANDAU, [eps, k, k])
    n = 6
    J, grad, W = orc.backward(g, f0, n, ckpt=4)
    return g, f0, n, J, grad, W, eps, k


def test_backward_J_matches_forward(orc, adj_case):
    g, f0, n, J, grad, W, *_ = adj_case
    assert abs(J - _J(orc, g, f0, n)) < 1e-14 * abs(J)


@pytest.mark.parametrize("seed", range(8))
def test_backward_directional_fd(orc, adj_case, seed):
    g, f0, n, J, grad, *_ = adj_case
    dirn = random_f(g.shape, seed=100 + seed) * f0.reshape(g.shape)
    e = 1e-6
    fd = (_J(orc, g, f0 + e * dirn, n) - _J(orc, g, f0 - e * dirn, n)) / (2 * e)
    an = np.sum(grad * dirn)
    assert abs(an - fd) < 1e-6 * abs(fd) + 1e-12, (an, fd)


@pytest.mark.parametrize("i", [0, 777, 4321, 9000])
def test_backward_single_dof_fd(orc, adj_case, i):
    g, f0, n, J, grad, *_ = adj_case
    e = 1e-6
    fp, fm = f0.copy().ravel(), f0.copy().ravel()
    fp[i] += e
    fm[i] -= e
    fd = (_J(orc, g, fp, n) - _J(orc, g, fm, n)) / (2 * e)
    assert abs(grad.ravel()[i] - fd) < 1e-6 * abs(fd) + 1e-11, (grad.ravel()[i], fd)


def test_backward_amplitude_fd(orc, adj_case):
    # dJ/deps = <dJ/df0, df0/deps>, df0/deps = (cos k x1 + cos k x2) M(v)
    g, f0, n, J, grad, W, eps, k = adj_case
    dfde = orc.init(g, orc.LANDAU, [1.0, k, k]) - orc.init(g, orc.LANDAU, [0.0, k, k])
    e = 1e-6
    fd = (_J(orc, g, orc.init(g, orc.LANDAU, [eps + e, k, k]), n) -
          _J(orc, g, orc.init(g, orc.LANDAU, [eps - e, k, k]), n)) / (2 * e)
    an = np.sum(grad * dfde)
    assert abs(an - fd) < 1e-6 * abs(fd), (an, fd)


def test_backward_independent_of_checkpoint_interval(orc, adj_case):
    g, f0, n, J, grad, *_ = adj_case
    for ck in (1, 2, 6):
        J2, grad2, _ = orc.backward(g, f0, n, ckpt=ck)
        assert J2 == J
        np.testing.assert_array_equal(grad2, grad)


def test_backward_weighted_energy_fd(orc, adj_case):
    # general weights c_m: J = sum_m c_m W(E^m)
    g, f0, n, *_ = adj_case
    c = np.linspace(0.3, -0.2, n)
    J, grad, W = orc.backward(g, f0, n, ckpt=3, cW=c)
    dirn = random_f(g.shape, seed=77) * f0.reshape(g.shape)
    e = 1e-6

    def Jc(f):
        _, W, _, _ = orc.step(g, f, n)
        return float(c @ W)

    fd = (Jc(f0 + e * dirn) - Jc(f0 - e * dirn)) / (2 * e)
    assert abs(np.sum(grad * dirn) - fd) < 1e-6 * abs(fd) + 1e-12


def test_backward_degree0_fd(orc):
    # Degree 0: each v-sweep is piecewise linear in E, with a kink where E at
    # an x-node crosses zero (the shift changes its integer part); the
    # symmetric Landau data has E = 0 at the node of the middle cell of an
    # odd cell count, so a seeded perturbation of f0 moves E off zero and a
    # small step (1e-7) keeps the central difference on one side of every
    # kink.
    g = orc.Grid(deg=0, nc=(5, 7, 6, 6), lo=LANDAU_LO, hi=LANDAU_HI, dt=0.1)
    f0 = orc.init(g, orc.LANDAU, [0.5, 0.5, 0.5])
    f0 = f0 + 1e-3 * random_f(f0.shape, seed=77).reshape(f0.shape)
    n = 7
    _, grad, _ = orc.backward(g, f0, n, ckpt=3)
    dirn = random_f(f0.shape, seed=78).reshape(f0.shape)
    e = 1e-7
    fd = (_J(orc, g, f0 + e * dirn, n) - _J(orc, g, f0 - e * dirn, n)) / (2 * e)
    assert abs(np.sum(grad * dirn) - fd) < 1e-7 * abs(fd)
