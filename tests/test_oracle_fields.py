"""Pins of the oracle's charge density, Poisson map and diagnostics.

rho(x) = int f dv and div E = rho - 1, curl E = 0 (Eq. (vlasov-poisson)).
The Poisson map is checked against closed-form fields of single Fourier
modes (signs, wavenumbers, component order, unequal box lengths) and by the
dot-product identity of its transpose; rho and the diagnostics against
Gaussian moments.
"""
import numpy as np
import pytest

from inputs import LANDAU_HI, LANDAU_LO, random_f, random_field


def _grid(orc, deg=2, nc=(12, 10, 8, 8), lo=LANDAU_LO, hi=LANDAU_HI, kmax=-1, dt=0.1):
    return orc.Grid(deg=deg, nc=nc, lo=lo, hi=hi, dt=dt, kmax=kmax)


@pytest.mark.parametrize("m", [(1, 0), (0, 1), (1, 2), (-2, 1), (3, -1)])
@pytest.mark.parametrize("deg", [1, 2, 3])
def test_poisson_single_mode_closed_form(orc, m, deg):
    # rho - 1 = eps cos(k.m.x) gives phi = eps cos/(|k m|^2), E = -grad phi:
    #   E_d = eps k_d m_d sin(k.m.x) / |k m|^2.
    # Unequal box lengths separate k1 from k2.  The composite Gauss-Legendre
    # rule integrates modes |m| < nc exactly, so with K = 4 (no aliasing) the
    # map reproduces the closed form to round-off.
    lo = (0.0, 0.0, -6.0, -6.0)
    hi = (4 * np.pi, 6 * np.pi, 6.0, 6.0)
    g = _grid(orc, deg=deg, nc=(12, 14, 2, 2), lo=lo, hi=hi, kmax=4)
    k = np.array([2 * np.pi / (hi[0] - lo[0]), 2 * np.pi / (hi[1] - lo[1])])
    X2, X1 = np.meshgrid(g.nodes(1), g.nodes(0), indexing="ij")
    eps = 0.3
    ph = k[0] * m[0] * X1 + k[1] * m[1] * X2
    rho = 1 + eps * np.cos(ph)
    E1, E2 = orc.poisson(g, rho)
    km2 = (k[0] * m[0]) ** 2 + (k[1] * m[1]) ** 2
    np.testing.assert_allclose(E1, eps * k[0] * m[0] * np.sin(ph) / km2, rtol=0, atol=1e-13)
    np.testing.assert_allclose(E2, eps * k[1] * m[1] * np.sin(ph) / km2, rtol=0, atol=1e-13)


@pytest.mark.parametrize("deg", [1, 2, 3])
@pytest.mark.parametrize("mp", [7, 9, 11])
@pytest.mark.parametrize("d", [0, 1])
def test_poisson_high_mode_aliasing_exact(orc, deg, mp, d):
    # With the default cap K = nc - 1 a high mode m' aliases onto nc - m'.
    # The node set repeats every cell, so the composite Gauss-Legendre sum of
    # exp(i kappa j x) over the box vanishes unless j is a multiple of nc, and
    # for j = +-nc it is L times a = -1/2 sum_n w_n cos(pi t_n) (the one-cell
    # rule's error on one period; nodes t_n, weights w_n from numpy).  For
    # rho - 1 = eps cos(kappa m' x_d) that gives rho_hat(+-m') = eps/2 and
    # rho_hat(+-(nc - m')) = a eps/2, hence exactly
    #   E_d = eps sin(kappa m' x)/(kappa m') + a eps sin(kappa m_a x)/(kappa m_a),
    # m_a = nc - m', and no field in the other component.
    lo = (0.0, 0.0, -6.0, -6.0)
    hi = (4 * np.pi, 6 * np.pi, 6.0, 6.0)
    nc = (12, 12, 2, 2)
    g = _grid(orc, deg=deg, nc=nc, lo=lo, hi=hi)
    kap = 2 * np.pi / (hi[d] - lo[d])
    X2, X1 = np.meshgrid(g.nodes(1), g.nodes(0), indexing="ij")
    X = X1 if d == 0 else X2
    eps = 0.3
    E = orc.poisson(g, 1 + eps * np.cos(kap * mp * X))
    t, w = np.polynomial.legendre.leggauss(deg + 1)
    a = -0.5 * np.sum(w * np.cos(np.pi * t))
    ma = nc[d] - mp
    pred = eps * (np.sin(kap * mp * X) / (kap * mp) + a * np.sin(kap * ma * X) / (kap * ma))
    np.testing.assert_allclose(E[d], pred, rtol=0, atol=1e-13)
    np.testing.assert_allclose(E[1 - d], 0, atol=1e-13)


def test_poisson_landau_field_default_modes(orc):
    # Landau density 1 + eps cos(k x1) at degree 3 with the default mode
    # count: E1 = (eps/k) sin(k x1), E2 = 0, up to the aliasing of the
    # Gauss-Legendre rule at mode nc (small for 4 nodes per cell).
    g = _grid(orc, deg=3, nc=(16, 16, 2, 2))
    X2, X1 = np.meshgrid(g.nodes(1), g.nodes(0), indexing="ij")
    eps, k = 0.01, 0.5
    E1, E2 = orc.poisson(g, 1 + eps * np.cos(k * X1))
    np.testing.assert_allclose(E1, eps / k * np.sin(k * X1), rtol=0, atol=1e-4 * eps / k)
    np.testing.assert_allclose(E2, 0, atol=1e-14)


def test_poisson_removes_mean_and_is_linear(orc):
    g = _grid(orc)
    r = random_field(g.xshape, seed=1)
    E1, E2 = orc.poisson(g, r)
    F1, F2 = orc.poisson(g, r + 7.5)
    np.testing.assert_allclose(F1, E1, atol=1e-12)
    np.testing.assert_allclose(F2, E2, atol=1e-12)
    s = random_field(g.xshape, seed=2)
    G1, G2 = orc.poisson(g, 2 * r - 3 * s)
    S1, S2 = orc.poisson(g, s)
    np.testing.assert_allclose(G1, 2 * E1 - 3 * S1, atol=1e-12)
    np.testing.assert_allclose(G2, 2 * E2 - 3 * S2, atol=1e-12)


@pytest.mark.parametrize("kmax", [-1, 3])
def test_poisson_adjoint_dot_product(orc, kmax):
    g = _grid(orc, deg=1, nc=(6, 9, 2, 2), kmax=kmax)
    r = random_field(g.xshape, seed=3)
    a = random_field(g.xshape, seed=4)
    b = random_field(g.xshape, seed=5)
    E1, E2 = orc.poisson(g, r)
    rb = orc.poisson_adj(g, a, b)
    lhs = np.sum(a * E1) + np.sum(b * E2)
    assert abs(lhs - np.sum(rb * r)) < 1e-13 * (abs(lhs) + 1)


def test_rho_of_maxwellian(orc):
    # int (1 + eps(cos k x1 + cos k x2)) exp(-|v|^2/2)/(2 pi) dv
    #   = (1 + eps(cos k x1 + cos k x2)) * m1 * m2, with m the 1D Gaussian
    # mass on [-6, 6] (erf(6/sqrt2)); GL per cell of width 1.5 at degree 3.
    from math import erf, sqrt

    g = _grid(orc, deg=3, nc=(5, 4, 8, 8))
    eps, k = 0.2, 0.5
    f = orc.init(g, orc.LANDAU, [eps, k, k])
    r = orc.rho(g, f)
    X2, X1 = np.meshgrid(g.nodes(1), g.nodes(0), indexing="ij")
    m = erf(6 / sqrt(2))
    np.testing.assert_allclose(r, (1 + eps * (np.cos(k * X1) + np.cos(k * X2))) * m * m,
                               rtol=2e-6)


def test_rho_adjoint_dot_product(orc):
    g = _grid(orc, deg=1, nc=(3, 4, 5, 2))
    f = random_f(g.shape, seed=6)
    rb = random_field(g.xshape, seed=7)
    lhs = np.sum(rb * orc.rho(g, f))
    rhs = np.sum(orc.rho_adj(g, rb) * f.reshape(g.shape))
    assert abs(lhs - rhs) < 1e-13 * (abs(lhs) + 1)


def test_diagnostics_gaussian_moments(orc):
    from math import erf, exp, pi, sqrt

    g = _grid(orc, deg=3, nc=(4, 4, 10, 10))
    eps, k = 0.3, 0.5
    f = orc.init(g, orc.LANDAU, [eps, k, k])
    L = 4 * pi
    m = erf(6 / sqrt(2))                        # int_-6^6 exp(-v^2/2)/sqrt(2pi)
    m2 = m - 2 * 6 * exp(-18) / sqrt(2 * pi)    # int v^2 exp(-v^2/2)/sqrt(2pi)
    E1 = random_field(g.xshape, seed=8)
    E2 = random_field(g.xshape, seed=9)
    d = orc.diagnostics(g, f, E1, E2)
    # the perturbation cos(k x) integrates to zero over the period
    assert abs(d["mass"] - L * L * m * m) < 1e-7 * L * L  # v-quadrature error
    assert abs(d["l1"] - d["mass"]) < 1e-12 * d["mass"]  # f > 0
    assert abs(d["kinetic"] - L * L * m * m2) < 1e-7 * L * L
    # int f^2 = (L^2 + eps^2 L^2) * (int M1^2)^2, int exp(-v^2)/(2pi) = erf(6)/(2 sqrt(pi))
    q = erf(6.0) / (2 * sqrt(pi))
    assert abs(d["l2sq"] - L * L * (1 + eps * eps) * q * q) < 1e-5 * d["l2sq"]  # exp(-v^2) is sharper
    wx = np.outer(g.weights(1), g.weights(0))
    assert abs(d["electric"] - 0.5 * np.sum(wx * (E1 ** 2 + E2 ** 2))) < 1e-12 * d["electric"]
    assert abs(d["total"] - d["kinetic"] - d["electric"]) < 1e-12


@pytest.mark.parametrize("deg", [1, 2, 3])
def test_uniform_density_has_no_field(orc, deg):
    # A uniform plasma carries no field: the default mode range stays below
    # the aliasing mode nc of the composite Gauss-Legendre rule.
    g = _grid(orc, deg=deg, nc=(7, 9, 2, 2))
    E1, E2 = orc.poisson(g, np.full(g.xshape, 1.7))
    assert np.abs(E1).max() < 1e-14 and np.abs(E2).max() < 1e-14
    # with modes beyond nc - 1 the background would alias into mode nc
    g2 = _grid(orc, deg=2, nc=(7, 9, 2, 2), kmax=10)
    F1, _ = orc.poisson(g2, np.full(g2.xshape, 1.7))
    assert np.abs(F1).max() > 1e-4


def _gauss_moments(a, lo, hi):
    """Integrals of v^0, v^1, v^2 against the unit Gaussian density centred
    at a over [lo, hi] (closed forms by the error function:
    int u phi = -phi, int u^2 phi = Phi - u phi)."""
    from math import erf, exp, pi, sqrt

    def Phi(u):
        return 0.5 * (1 + erf(u / sqrt(2)))

    def phi(u):
        return exp(-u * u / 2) / sqrt(2 * pi)

    l, r = lo - a, hi - a
    m0 = Phi(r) - Phi(l)
    m1 = -(phi(r) - phi(l)) + a * m0
    m2 = (Phi(r) - r * phi(r)) - (Phi(l) - l * phi(l)) - 2 * a * (phi(r) - phi(l)) + a * a * m0
    return m0, m1, m2


def _v_moments(g, f):
    """rho and the v1^2, v2^2 moments of f at every x-node by the grid's
    tensor Gauss-Legendre weights (nodes and weights pinned above)."""
    F = f.reshape(g.shape)
    w2, w3 = g.weights(2), g.weights(3)
    v1, v2 = g.nodes(2), g.nodes(3)
    W = np.outer(w3, w2)[:, :, None, None]
    rho = np.sum(W * F, axis=(0, 1))
    m11 = np.sum(W * (v1 ** 2)[None, :, None, None] * F, axis=(0, 1))
    m22 = np.sum(W * (v2 ** 2)[:, None, None, None] * F, axis=(0, 1))
    return rho, m11, m22


def test_two_stream_initial_value_moments(orc):
    # Additive two-stream initial value (kind 1) on [0, 10 pi]^2 x [-9, 9]^2:
    #   f0 = (e^{-(v1-v0)^2/2} + e^{-(v1+v0)^2/2}) e^{-v2^2/2} / (4 pi)
    #        * (1 + eps cos k x1 + eps cos k x2).
    # Its v-moments are closed forms of truncated Gaussians: the density is
    # (1 + eps cos k x1 + eps cos k x2) m0(v0) g0 with m0 the mean mass of
    # the two shifted unit Gaussians on [-9, 9] and g0 that of the centred
    # one; <v1^2> = 1 + v0^2 (the beams), <v2^2> = 1 (a Maxwellian).  A 4 pi
    # / 8 pi slip, a dropped v2 factor, beams put in v2, or a product in
    # place of the sum of the x-perturbations each fail one of these.
    from inputs import TSI_HI, TSI_LO

    g = orc.Grid(deg=3, nc=(5, 4, 24, 16), lo=TSI_LO, hi=TSI_HI, dt=0.1)
    eps, k, v0 = 0.3, 0.2, 3.0
    f = orc.init(g, orc.TWO_STREAM, [eps, k, v0])
    rho, m11, m22 = _v_moments(g, f)
    X2, X1 = np.meshgrid(g.nodes(1), g.nodes(0), indexing="ij")
    pert = 1 + eps * np.cos(k * X1) + eps * np.cos(k * X2)
    p, q = _gauss_moments(v0, -9, 9), _gauss_moments(-v0, -9, 9)
    c = _gauss_moments(0.0, -9, 9)
    beam0, beam2 = 0.5 * (p[0] + q[0]), 0.5 * (p[2] + q[2])
    np.testing.assert_allclose(rho, pert * beam0 * c[0], rtol=2e-6)
    np.testing.assert_allclose(m11, pert * beam2 * c[0], rtol=2e-6)
    np.testing.assert_allclose(m22, pert * beam0 * c[2], rtol=2e-6)
    # the oracle's own charge density agrees with this quadrature
    np.testing.assert_allclose(orc.rho(g, f), rho, rtol=1e-13)


def test_paper_two_stream_initial_value_moments(orc):
    # Sec. 5, Eq. (iv-tsi) (kind 2) on [0, 10 pi]^2 x [-6, 6]^2:
    #   f0 = (1 + eps cos k x1 cos k x2) / (8 pi) prod_d (e^{-(v_d-v0)^2/2} + e^{-(v_d+v0)^2/2}).
    # Density (1 + eps cos k x1 cos k x2) m0^2, <v_d^2> = m2/m0 in both
    # directions, with the truncation of the beams at |v| = 6 in m0, m2.
    from inputs import TSI_HI

    lo, hi = (0.0, 0.0, -6.0, -6.0), (TSI_HI[0], TSI_HI[1], 6.0, 6.0)
    g = orc.Grid(deg=3, nc=(4, 5, 20, 20), lo=lo, hi=hi, dt=0.1)
    eps, k, v0 = 0.25, 0.2, 2.4
    f = orc.init(g, orc.TWO_STREAM_PAPER, [eps, k, v0])
    rho, m11, m22 = _v_moments(g, f)
    X2, X1 = np.meshgrid(g.nodes(1), g.nodes(0), indexing="ij")
    pert = 1 + eps * np.cos(k * X1) * np.cos(k * X2)
    p, q = _gauss_moments(v0, -6, 6), _gauss_moments(-v0, -6, 6)
    b0, b2 = 0.5 * (p[0] + q[0]), 0.5 * (p[2] + q[2])
    np.testing.assert_allclose(rho, pert * b0 * b0, rtol=2e-6)
    np.testing.assert_allclose(m11, pert * b2 * b0, rtol=2e-6)
    np.testing.assert_allclose(m22, pert * b0 * b2, rtol=2e-6)


def test_rho_column_matches_rho(orc):
    # The single-node v-quadrature (the checker of the full-size charge
    # density) equals the whole-grid one at every x-node, on a grid whose
    # two velocity directions differ in cell count, box and node count, so
    # a swapped v1/v2 index or weight would show.
    g = orc.Grid(deg=2, nc=(3, 4, 5, 7), lo=(0.0, 0.0, -6.0, -2.0),
                 hi=(4 * np.pi, 2 * np.pi, 6.0, 9.0), dt=0.1)
    f = random_f(g.shape, seed=11)
    r = orc.rho(g, f)
    F = f.reshape(g.shape)
    for i1 in range(g.D(1)):
        for i0 in range(g.D(0)):
            c = orc.rho_column(g, F[:, :, i1, i0])
            assert abs(c - r[i1, i0]) <= 1e-14 * max(1.0, abs(r[i1, i0]))
    # and it weighs v1 and v2 by their own rules: a column varying in v1
    # only against its closed form
    v1 = g.nodes(2)
    col = np.tile(v1 ** 2, (g.D(3), 1))
    exact = (6.0 ** 3 - (-6.0) ** 3) / 3 * (9.0 - (-2.0))
    assert abs(orc.rho_column(g, col) - exact) < 1e-12 * exact
