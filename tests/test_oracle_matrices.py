"""Pins of the oracle's Gauss-Legendre nodes and projection matrices.

Each check uses something other than the oracle itself: numpy's Gauss-Legendre
routine, the closed-form nodes, exact polynomial integration (40-digit mpmath) of the
L2-projection integrals of Sec. 2 / Eq. (AB-sldg), the textbook donor-cell
scheme at degree 0, and identities any translate-then-project map satisfies.
"""
import numpy as np
import pytest
from conftest import golden_rows


@pytest.mark.parametrize("n", range(1, 9))
def test_gauss_legendre_matches_numpy(orc, n):
    xi, w = orc.gauss_legendre(n)
    x2, w2 = np.polynomial.legendre.leggauss(n)
    np.testing.assert_allclose(xi, (x2 + 1) / 2, rtol=0, atol=2e-16)
    np.testing.assert_allclose(w, w2 / 2, rtol=0, atol=1e-15)
    assert abs(w.sum() - 1.0) < 1e-15


def test_gauss_legendre_closed_forms(orc):
    import math

    def ev(expr):
        return eval(expr, {"__builtins__": {}}, {"sqrt": math.sqrt})

    rows = golden_rows("gauss_legendre_01.txt")
    assert [int(r[0]) for r in rows] == [1, 2, 3, 4]
    for n, nodes, weights in rows:
        xi, w = orc.gauss_legendre(int(n))
        np.testing.assert_allclose(xi, [ev(e) for e in nodes.split(",")], rtol=0, atol=2e-16)
        np.testing.assert_allclose(w, [ev(e) for e in weights.split(",")], rtol=0, atol=2e-16)


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_lagrange_basis(orc, n):
    xi, _ = orc.gauss_legendre(n)
    for j in range(n):
        for l in range(n):
            assert abs(orc.lagrange(n, j, xi[l]) - (1.0 if j == l else 0.0)) < 1e-14
    for t in (0.0, 0.13, 0.77, 1.0):
        assert abs(sum(orc.lagrange(n, j, t) for j in range(n)) - 1.0) < 1e-14
        assert abs(sum(orc.lagrange(n, j, t, True) for j in range(n))) < 1e-12
        for j in range(n):
            e = 1e-6
            fd = (orc.lagrange(n, j, t + e) - orc.lagrange(n, j, t - e)) / (2 * e)
            assert abs(fd - orc.lagrange(n, j, t, True)) < 1e-8


def _exact_matrices(deg, theta_rat):
    """A(theta), B(theta) by exact polynomial integration of the L2 projection.

    Nodes are the closed-form Gauss-Legendre roots mapped to [0,1], evaluated
    in 40-digit arithmetic (mpmath).  The integrands of Sec. 2 (translate by
    theta cells, project on degree deg) are expanded as polynomials in t and
    integrated through their antiderivatives, not by quadrature."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    th = mp.mpf(theta_rat[0]) / theta_rat[1]
    s35, s65 = mp.sqrt(mp.mpf(3) / 5), mp.sqrt(mp.mpf(6) / 5)
    roots = {
        1: [mp.mpf(0)],
        2: [-1 / mp.sqrt(3), 1 / mp.sqrt(3)],
        3: [-s35, mp.mpf(0), s35],
        4: [-mp.sqrt(mp.mpf(3) / 7 + mp.mpf(2) / 7 * s65), -mp.sqrt(mp.mpf(3) / 7 - mp.mpf(2) / 7 * s65),
            mp.sqrt(mp.mpf(3) / 7 - mp.mpf(2) / 7 * s65), mp.sqrt(mp.mpf(3) / 7 + mp.mpf(2) / 7 * s65)],
    }[deg + 1]
    xi = [(1 + r) / 2 for r in roots]
    n = deg + 1

    def pmul(p, q):  # coefficient lists, lowest degree first
        r = [mp.mpf(0)] * (len(p) + len(q) - 1)
        for i, a in enumerate(p):
            for k, b in enumerate(q):
                r[i + k] += a * b
        return r

    def phi(j, shift):  # phi_j(t + shift) as a polynomial in t
        p = [mp.mpf(1)]
        for m in range(n):
            if m != j:
                p = pmul(p, [(shift - xi[m]) / (xi[j] - xi[m]), 1 / (xi[j] - xi[m])])
        return p

    def integ(p, a, b):
        return sum(c * (b ** (i + 1) - a ** (i + 1)) / (i + 1) for i, c in enumerate(p))

    A = np.zeros((n, n))
    B = np.zeros((n, n))
    for j in range(n):
        wj = integ(pmul(phi(j, 0), phi(j, 0)), 0, 1)  # exact mass-matrix diagonal
        for l in range(n):
            A[j, l] = float(integ(pmul(phi(j, 0), phi(l, 1 - th)), 0, th) / wj)
            B[j, l] = float(integ(pmul(phi(j, 0), phi(l, -th)), th, 1) / wj)
    return A, B


@pytest.mark.parametrize("deg", [0, 1, 2, 3])
@pytest.mark.parametrize("theta", [(1, 3), (5, 8)])
def test_matrices_against_exact_integration(orc, deg, theta):
    Ae, Be = _exact_matrices(deg, theta)
    A, B = orc.matrices(deg, theta[0] / theta[1])
    np.testing.assert_allclose(A, Ae, rtol=0, atol=5e-14)
    np.testing.assert_allclose(B, Be, rtol=0, atol=5e-14)


@pytest.mark.parametrize("theta", [0.0, 0.1, 0.5, 0.93])
def test_degree0_is_donor_cell(orc, theta):
    # Degree 0: out[c] = theta u[c-s-1] + (1-theta) u[c-s], first-order upwind.
    A, B = orc.matrices(0, theta)
    assert abs(A[0, 0] - theta) < 1e-15 and abs(B[0, 0] - (1 - theta)) < 1e-15


@pytest.mark.parametrize("deg", [0, 1, 2, 3])
def test_matrices_endpoints_and_continuity(orc, deg):
    n = deg + 1
    A, B = orc.matrices(deg, 0.0)
    np.testing.assert_allclose(A, 0, atol=1e-15)
    np.testing.assert_allclose(B, np.eye(n), atol=1e-14)
    # theta -> 1 with cell s equals theta = 0 with cell s+1: A(1) = I, B(1) = 0
    A, B = orc.matrices(deg, 1.0 - 1e-13)
    np.testing.assert_allclose(A, np.eye(n), atol=1e-11)
    np.testing.assert_allclose(B, 0, atol=1e-11)


@pytest.mark.parametrize("deg", [0, 1, 2, 3])
@pytest.mark.parametrize("theta", [0.0, 0.21, 0.5, 0.87])
def test_column_mass_identity(orc, deg, theta):
    # Mass of a translated basis function is preserved: sum_j w_j (A+B)_jl = w_l
    _, w = orc.gauss_legendre(deg + 1)
    A, B = orc.matrices(deg, theta)
    np.testing.assert_allclose(w @ (A + B), w, rtol=0, atol=2e-15)


@pytest.mark.parametrize("deg", [1, 2, 3])
@pytest.mark.parametrize("theta", [0.2, 0.55, 0.8])
def test_matrix_theta_derivatives(orc, deg, theta):
    A, B, dA, dB = orc.matrices(deg, theta, deriv=True)
    e = 1e-6
    Ap, Bp = orc.matrices(deg, theta + e)
    Am, Bm = orc.matrices(deg, theta - e)
    np.testing.assert_allclose(dA, (Ap - Am) / (2 * e), rtol=0, atol=1e-8)
    np.testing.assert_allclose(dB, (Bp - Bm) / (2 * e), rtol=0, atol=1e-8)
    # total mass does not depend on theta
    _, w = orc.gauss_legendre(deg + 1)
    np.testing.assert_allclose(w @ (dA + dB), 0, atol=1e-13)


@pytest.mark.parametrize("deg", [1, 2, 3])
def test_matrices_are_polynomials_of_degree_2l_plus_1(orc, deg):
    # Each entry is a polynomial in theta of degree <= 2l+1 (integral of a
    # degree-2l integrand with theta-dependent limits and arguments).
    ths = np.linspace(0.0, 0.95, 3 * deg + 6)
    vals = np.array([np.concatenate([m.ravel() for m in orc.matrices(deg, t)]) for t in ths])
    V = np.vander(ths, 2 * deg + 2, increasing=True)
    coef, *_ = np.linalg.lstsq(V, vals, rcond=None)
    np.testing.assert_allclose(V @ coef, vals, atol=1e-12)
