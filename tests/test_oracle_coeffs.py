"""Pins of the oracle's coefficients and equilibrium (Eq. eq:rdr, Appendix, Tables 1-2).

Each test checks the oracle against a route that does not use its Gauss-Jordan
inverse: the closed form of the Appendix in exact rationals, the explicit
formulas of Eq. (eq:1d5v) and of the four-velocity model, the rows of
Table 1 and Table 2, and Gauss-Hermite quadrature of the Maxwellian.
"""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle as O

SETS = [
    (0, 1, -1, 3, -3),
    (0, 1, -1, 2, -2),
    (0, 2, -2, 3, -3),
    (0, 1, -1),
    (0, 2, -4),
    (1, -1, 3, -3),
    (0, 1, -1, 2, -2, 3, -3),
    (0, 1, -2, 3),
]


def closed_form_coeffs(v):
    """Appendix closed form, index set read as all n-subsets of {v_j : j != i}.

    r_i = sum_n (-1)^n mu_{q-1-n} e_n({v_j}_{j!=i}) / prod_{j!=i}(v_i - v_j),
    so the coefficient of mu_m (m = q-1-n) is (-1)^n e_n / prod.  Exact rationals.
    """
    q = len(v)
    C = [[Fraction(0)] * q for _ in range(q)]
    for i in range(q):
        others = [Fraction(v[j]) for j in range(q) if j != i]
        den = Fraction(1)
        for w in others:
            den *= Fraction(v[i]) - w
        for n in range(q):
            e_n = sum((math.prod(c) for c in itertools.combinations(others, n)), Fraction(0))
            C[i][q - 1 - n] = Fraction((-1) ** n) * e_n / den
    return C


@pytest.mark.parametrize("v", SETS)
def test_vandermonde_inverse_matches_closed_form(v):
    C = O.vandermonde_inverse(v)
    ref = closed_form_coeffs(v)
    q = len(v)
    for i in range(q):
        for n in range(q):
            assert abs(C[i, n] - float(ref[i][n])) <= 1e-14 * max(1.0, abs(float(ref[i][n])))


@pytest.mark.parametrize("v", SETS)
def test_lagrange_property(v):
    # sum_n C[i][n] v_k^n = delta_ik: row i is the Lagrange polynomial through (v_k, delta_ik).
    C = O.vandermonde_inverse(v)
    q = len(v)
    V = np.array([[float(vk) ** n for vk in v] for n in range(q)])
    assert np.max(np.abs(C @ V - np.eye(q))) < 1e-13


def test_singular_set_rejected():
    with pytest.raises(ValueError):
        O.vandermonde_inverse([0, 1, 1])


def test_mb_moments_table2_row():
    # Table 2, Maxwell-Boltzmann row: mu_2 = theta + u^2, mu_3 = 3 theta u + u^3,
    # mu_4 = 3 theta^2 + 6 theta u^2 + u^4.
    for u, t in [(0.0, 1.0), (0.1, 1.0), (-0.37, 0.6), (1.3, 2.1)]:
        mu = O.mb_moments(u, t, 4)
        assert mu[0] == 1.0 and mu[1] == u
        assert abs(mu[2] - (t + u * u)) < 1e-15
        assert abs(mu[3] - (3 * t * u + u ** 3)) < 1e-14
        assert abs(mu[4] - (3 * t * t + 6 * t * u * u + u ** 4)) < 1e-13


def test_mb_moments_against_quadrature():
    # mu_n = int v^n F(v) dv, F Gaussian (mean u, variance theta): probabilists'
    # Gauss-Hermite quadrature with 40 nodes is exact for these polynomial degrees.
    x, w = np.polynomial.hermite_e.hermegauss(40)
    w = w / np.sqrt(2 * np.pi)
    for u, t in [(0.2, 0.5), (-0.8, 1.7), (0.0, 1.0)]:
        mu = O.mb_moments(u, t, 9)
        v = u + np.sqrt(t) * x
        for n in range(10):
            ref = float(np.sum(w * v ** n))
            assert abs(mu[n] - ref) <= 1e-12 * max(1.0, abs(ref))


@pytest.mark.parametrize("v", SETS)
def test_moment_identity(v):
    # Eq. (eq:rdr): mu_hat_n = sum_i v_i^n r_i equals mu_n for n = 0..q-1.
    q = len(v)
    for u in np.linspace(-0.3, 0.3, 7):
        for t in (0.4, 0.9, 1.2):
            r = O.r1d(v, u, t)
            mu = O.mb_moments(u, t, q - 1)
            for n in range(q):
                muh = float(np.dot(np.array(v, float) ** n, r))
                assert abs(muh - mu[n]) <= 1e-13 * max(1.0, abs(mu[n]))


def test_fifth_moment_node_polynomial():
    # On {0,+-1,+-3} the node polynomial v(v^2-1)(v^2-9) = v^5 - 10 v^3 + 9 v vanishes,
    # so mu_hat_5 = 10 mu_3 - 9 mu_1 (the first moment the model does not match).
    v = (0, 1, -1, 3, -3)
    for u, t in [(0.1, 1.0), (-0.2, 0.7)]:
        r = O.r1d(v, u, t)
        mu = O.mb_moments(u, t, 5)
        muh5 = float(np.dot(np.array(v, float) ** 5, r))
        assert abs(muh5 - (10 * mu[3] - 9 * mu[1])) < 1e-13
        assert abs(muh5 - mu[5]) > 1e-3


def test_eq_1d5v_explicit_formula():
    # Eq. (eq:1d5v) for v = {0, +-a, +-b}: c = b for v = +-a and c = a for v = +-b.
    for a, b in [(1.0, 3.0), (1.0, 2.0), (1.4, 2.8), (0.7, 2.3)]:
        v = [0.0, a, -a, b, -b]
        C = np.ascontiguousarray(O.vandermonde_inverse(v))
        for u, t in [(0.05, 1.0), (-0.2, 0.6)]:
            mu = O.mb_moments(u, t, 4)
            r = O.r1d(v, u, t, C)
            r1 = (mu[0] * a * a * b * b - mu[2] * (a * a + b * b) + mu[4]) / (a * a * b * b)
            assert abs(r[0] - r1) < 1e-14
            for i, vi in enumerate(v[1:], start=1):
                c = b if i in (1, 2) else a
                ri = (-mu[1] * vi * c * c - mu[2] * c * c + mu[3] * vi + mu[4]) / (
                    2 * vi * vi * (vi * vi - c * c))
                assert abs(r[i] - ri) < 1e-14


def test_four_velocity_formula():
    # Sec. 2.3: v = {+-a, +-b}, r_i = (v_i c^2 mu_0 + c^2 mu_1 - v_i mu_2 - mu_3)
    #                                   / (2 (v_i c^2 - v_i^3)), c = b for +-a, a for +-b.
    for a, b in [(1.0, 3.0), (0.5, 1.5), (1.0, 2.0)]:
        v = [a, -a, b, -b]
        C = np.ascontiguousarray(O.vandermonde_inverse(v))
        for u, t in [(0.1, 0.4), (-0.3, 0.25)]:
            mu = O.mb_moments(u, t, 3)
            r = O.r1d(v, u, t, C)
            for i, vi in enumerate(v):
                c = b if i < 2 else a
                ri = (vi * c * c * mu[0] + c * c * mu[1] - vi * mu[2] - mu[3]) / (
                    2 * (vi * c * c - vi ** 3))
                assert abs(r[i] - ri) < 1e-14


@pytest.mark.parametrize("zeta", [3, 4])
def test_table1_rows(zeta):
    # Table 1: D1Q3 with v = {0, +-sqrt(zeta theta0)}, theta held at theta0.
    # Lattice velocities {0, +-1} give theta0 = 1/zeta; u_bar = u / sqrt(theta0).
    theta0 = 1.0 / zeta
    v = (0, 1, -1)
    for u in np.linspace(-0.4, 0.4, 9):
        r = O.r1d(v, u, theta0)
        ub2 = u * u / theta0
        ub = u / math.sqrt(theta0)
        if zeta == 3:
            ref = [2 / 3 * (1 - ub2 / 2), (1 + math.sqrt(3) * ub + ub2) / 6,
                   (1 - math.sqrt(3) * ub + ub2) / 6]
        else:
            ref = [3 / 4 * (1 - ub2 / 3), (1 + 2 * ub + ub2) / 8, (1 - 2 * ub + ub2) / 8]
        assert np.max(np.abs(r - np.array(ref))) < 1e-15
        # Eq. (eq:1d3v): r_i = w_i [1 + v_i u/theta0 + u^2 (v_i^2 - theta0)/((zeta-1) theta0^2)]
        w = [1 - 1 / zeta, 1 / (2 * zeta), 1 / (2 * zeta)]
        ref2 = [w[i] * (1 + v[i] * u / theta0 + u * u * (v[i] ** 2 - theta0) / ((zeta - 1) * theta0 ** 2))
                for i in range(3)]
        assert np.max(np.abs(r - np.array(ref2))) < 1e-15


@pytest.mark.parametrize("theta0", [1.0, 0.25])
def test_table1_asymmetric_example(theta0):
    # Table 1 caption: v = {0, 2 sqrt(theta0), -4 sqrt(theta0)} (the caption's second
    # "v_1" is read as v_2) gives r_1 = (7 - 2ub - ub^2)/8, r_2 = (1 + 4ub + ub^2)/12,
    # r_3 = (1 - 2ub + ub^2)/24 with ub = u/sqrt(theta0).
    s = math.sqrt(theta0)
    v = (0, 2, -4) if theta0 == 1.0 else (0, 1, -2)
    assert v[1] == 2 * s and v[2] == -4 * s
    for u in np.linspace(-0.3, 0.3, 7):
        r = O.r1d(v, u, theta0)
        ub = u / s
        ref = [(7 - 2 * ub - ub * ub) / 8, (1 + 4 * ub + ub * ub) / 12, (1 - 2 * ub + ub * ub) / 24]
        assert np.max(np.abs(r - np.array(ref))) < 1e-15


def test_table2_rows():
    # Table 2: third moment of the isothermal D1Q3 models and of the 4-velocity model,
    # and the 5-velocity model matching all moments up to 4th order.
    for u in (0.05, -0.2, 0.31):
        for zeta, coef in ((3, 3.0), (4, 4.0)):
            th0 = 1.0 / zeta
            r = O.r1d((0, 1, -1), u, th0)
            v = np.array([0.0, 1.0, -1.0])
            assert abs(np.dot(v ** 2, r) - (th0 + u * u)) < 1e-15       # 2nd order: theta0 + u^2
            assert abs(np.dot(v ** 3, r) - coef * th0 * u) < 1e-15      # 3rd order: zeta theta0 u
        th0 = 0.3
        a = math.sqrt(3 * th0) / 2
        v4 = np.array([a, -a, 3 * a, -3 * a])
        r = O.r1d(v4, u, th0)
        assert abs(np.dot(v4 ** 2, r) - (th0 + u * u)) < 1e-14
        assert abs(np.dot(v4 ** 3, r) - (3 * th0 * u + u ** 3)) < 1e-14
        for t in (0.7, 1.0):
            r = O.r1d((0, 1, -1, 3, -3), u, t)
            v5 = np.array([0.0, 1, -1, 3, -3])
            assert abs(np.dot(v5 ** 2, r) - (t + u * u)) < 1e-14
            assert abs(np.dot(v5 ** 3, r) - (3 * t * u + u ** 3)) < 1e-14
            assert abs(np.dot(v5 ** 4, r) - (3 * t * t + 6 * t * u * u + u ** 4)) < 1e-13


def test_feq_tensor_product_moments():
    # Sec. 2.1 / Appendix: the 2D equilibrium is the product of 1D rules, so
    # sum v_x^a v_y^b f^eq = rho mu_a(u_x) mu_b(u_y) for a, b <= q1 - 1.
    v = (0, 1, -1, 3, -3)
    rho, ux, uy, t = 1.07, 0.08, -0.05, 0.93
    f = O.feq(2, v, rho, ux, uy, t)
    vel = np.array([(a, b) for a in v for b in v], dtype=float)
    mx = O.mb_moments(ux, t, 4)
    my = O.mb_moments(uy, t, 4)
    for a in range(5):
        for b in range(5):
            m = float(np.sum(vel[:, 0] ** a * vel[:, 1] ** b * f))
            assert abs(m - rho * mx[a] * my[b]) < 1e-12 * max(1.0, abs(rho * mx[a] * my[b]))
