"""Pins of the oracle's exact Riemann solver and of the oracle's shock tubes.

Riemann solver (Sec. 4): all 72 entries of Table 3, the printed
Rankine-Hugoniot relations for the shock speed and post-shock velocity, the
isothermal/thermal ratios quoted in Sec. 4, and conservation of mass, momentum
and energy by the sampled solution.

Shock tubes run on the oracle:
* D1Q3 zeta = 4 isothermal, rho 6:1 (Fig. 2 caption, Sec. 3.2): post-shock
  velocity 0.91 and shock front at 826 after 418 iterations.
* D1Q5 {0,+-1,+-3} thermal (gamma = 3), rho 1.1:1 and 2:1 at theta = 0.5,
  omega = 1.5: L1 distance to the exact solution before any wave reaches an end.
* The literal 1 / 0.125, theta 0.5 / 0.4 tube leaves the positivity region
  and produces theta <= 0 within a few dozen steps.
"""
import math

import numpy as np
import pytest

import oracle as O
from oracle import riemann as R
from paper_1402_5487_gb300 import inputs as I

from conftest import golden, read_printed_values

GAMMAS = (1.0, 5.0 / 3.0, 2.0, 3.0)


def _table3():
    rows = []
    with open(golden("table3_riemann_pressure_ratio.txt")) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([float(t) for t in line.split()])
    return rows


def test_table3_all_entries():
    rows = _table3()
    assert len(rows) == 18
    for row in rows:
        P = row[0]
        ndig = 3 if P < 2 else 2
        for g, printed in zip(GAMMAS, row[1:]):
            val = R.pressure_ratio_post_pre(P, g)
            # printed to ndig decimals: within half a unit of the last digit (+ slack
            # of 1e-4 for values printed as x.xx5 boundaries)
            assert abs(val - printed) <= 0.5 * 10 ** (-ndig) + 1e-4, (P, g, val, printed)


@pytest.mark.parametrize("gamma", GAMMAS)
def test_rankine_hugoniot_relations(gamma):
    # right-moving shock into gas at rest with theta_pre = theta_R: solver's shock speed and
    # u* equal the printed relations in units of sqrt(theta_pre).
    for ratio in (1.1, 2.0, 6.0, 10.0):
        thR = 0.7
        left = R.State(ratio, 0.0, ratio * thR)
        right = R.State(1.0, 0.0, thR)
        w = R.wave_speeds(left, right, gamma)
        P = w["p_star"] / right.p
        assert w["right"][0] == "shock"
        assert abs(w["right"][1] / math.sqrt(thR) - R.rh_shock_speed(P, gamma)) < 1e-12
        assert abs(w["u_star"] / math.sqrt(thR) - R.rh_post_velocity(P, gamma)) < 1e-12


def test_isothermal_over_thermal_ratios():
    vals = read_printed_values()
    out = {}
    for g in GAMMAS:
        w = R.wave_speeds(R.State(1.1, 0.0, 1.1), R.State(1.0, 0.0, 1.0), g)
        out[g] = (w["u_star"], w["right"][1])
    r1 = out[1.0][0] / out[3.0][0]
    r3 = out[1.0][0] / out[5.0 / 3.0][0]
    s1 = out[3.0][1] / out[1.0][1]
    s3 = out[5.0 / 3.0][1] / out[1.0][1]
    assert abs(r1 - vals["iso_over_thermal_1d"]) < 0.015 and abs(s1 - vals["iso_over_thermal_1d"]) < 0.015
    assert abs(r3 - vals["iso_over_thermal_3d"]) < 0.015 and abs(s3 - vals["iso_over_thermal_3d"]) < 0.015


@pytest.mark.parametrize("gamma", GAMMAS)
def test_sampled_solution_conserves(gamma):
    # Integrals of rho, rho u and total energy over [-X, X] are unchanged at time t
    # (no wave reaches the ends): checks the fan and star-state formulas.
    left, right = R.State(2.5, 0.1, 2.5 * 0.6), R.State(1.0, -0.05, 0.6)
    t, X = 1.0, 10.0
    xi = np.linspace(-X, X, 400001)
    rho, u, p = R.sample(left, right, gamma, xi / t)
    dx = xi[1] - xi[0]

    def energy(r, uu, pp):
        eint = pp / (gamma - 1.0) if gamma != 1.0 else 0.0
        return 0.5 * r * uu * uu + eint

    mass = np.sum(rho) * dx
    mom = np.sum(rho * u) * dx
    m0 = X * (left.rho + right.rho)
    j0 = X * (left.rho * left.u + right.rho * right.u)
    # flux balance over [0, t]: d/dt int q = F(-X) - F(X)
    fm = left.rho * left.u - right.rho * right.u
    fj = (left.rho * left.u ** 2 + left.p) - (right.rho * right.u ** 2 + right.p)
    assert abs(mass - (m0 + t * fm)) < 1e-3
    assert abs(mom - (j0 + t * fj)) < 1e-3
    if gamma != 1.0:
        e = np.sum(energy(rho, u, p)) * dx
        eL, eR = energy(left.rho, left.u, left.p), energy(right.rho, right.u, right.p)
        fe = left.u * (eL + left.p) - right.u * (eR + right.p)
        assert abs(e - (X * (eL + eR) + t * fe)) < 1e-3


def _tube(v, omega, theta0, left, right, steps, isothermal=False, n=1000):
    lat = O.Lattice(1, v, omega, n, bc="fixed", theta0=theta0, isothermal=isothermal,
                    left_state=left, right_state=right)
    f = lat.init(*I.shock_tube_fields(n, left, right))
    f = lat.run(f, steps)
    return lat, lat.moments(f)


def test_isothermal_zeta4_shock_tube_printed_front():
    vals = read_printed_values()
    theta0 = 0.25  # lattice velocities {0, +-1} = {0, +-sqrt(4 theta0)}
    omega = 4 * math.sqrt(3) - 6
    steps = int(vals["shock6_iterations_param"])
    _, (rho, ux, _, _) = _tube((0, 1, -1), omega, theta0, (6.0, 0.0, theta0), (1.0, 0.0, theta0),
                               steps, isothermal=True)
    ub = ux[0] / math.sqrt(theta0)
    assert abs(np.mean(ub[650:750]) - vals["shock6_u_post"]) < 0.005
    r = rho[0]
    plateau = np.mean(r[650:750])
    half = 0.5 * (plateau + 1.0)
    i = int(np.nonzero(r > half)[0].max())
    front = (i + 1) + (r[i] - half) / (r[i] - r[i + 1])  # 1-based node coordinate
    assert abs(front - vals["shock6_front_x"]) < 2.5


def zeta4_vs_lbgk_small_ratio(tube=None, ratio=1.1):
    """Sec. 3.2 and the captions of Figs. 3-4: isothermal three-velocity shock tubes at
    rho_L/rho_R = 1.1 and theta = theta0, LBGK (zeta = 3, theta0 = 1/3, omega = 1, 362
    iterations) against the parametric zeta = 4 model (theta0 = 1/4, 418 iterations), once with
    the viscosity nu = (1/omega - 1/2) sqrt(theta0) dx / sqrt(zeta) matched (omega = 4 sqrt(3) - 6)
    and once with nu_hat = nu (zeta - 1) / 2 matched instead.  Returns the largest density and
    velocity (normalised by sqrt(theta0)) differences of both zeta = 4 runs against LBGK.
    `tube(v, omega, theta0, left, right, steps)` returns the moments (rho, ux, uy, theta)."""
    tube = tube or (lambda *a: _tube(*a, isothermal=True)[1])

    def run(zeta, omega, steps):
        th = 1.0 / zeta
        rho, ux, _, _ = tube((0, 1, -1), omega, th, (ratio, 0.0, th), (1.0, 0.0, th), steps)
        return np.asarray(rho).ravel(), np.asarray(ux).ravel() / math.sqrt(th)

    nu_lbgk = (1.0 / 1.0 - 0.5) / math.sqrt(3)
    omega_nu = 1.0 / (0.5 + nu_lbgk * math.sqrt(4))
    omega_nu_hat = 1.0 / (0.5 + nu_lbgk * math.sqrt(4) * 2 / (4 - 1))
    r3, u3 = run(3, 1.0, 362)
    out = {}
    for name, om in (("nu", omega_nu), ("nu_hat", omega_nu_hat)):
        r4, u4 = run(4, om, 418)
        out[name] = (float(np.max(np.abs(r4 - r3))), float(np.max(np.abs(u4 - u3))))
    return out, omega_nu, omega_nu_hat


def test_zeta4_differs_from_lbgk_by_about_three_tenths_of_a_percent():
    vals = read_printed_values()
    out, omega_nu, omega_nu_hat = zeta4_vs_lbgk_small_ratio()
    assert abs(omega_nu - vals["omega_zeta4_matched"]) < 1e-14
    # (zeta - 1)/2 (1/omega - 1/2)/sqrt(4) = (1 - 1/2)/sqrt(3)
    assert abs(1.5 * (1 / omega_nu_hat - 0.5) / 2 - 0.5 / math.sqrt(3)) < 1e-15
    printed = vals["shock11_max_diff_zeta4_lbgk"]
    drho, du = out["nu"]
    # "about 0.3 %" for both density and velocity (measured 0.29 % and 0.28 %)
    assert abs(drho - printed) < 0.0005 and abs(du - printed) < 0.0005, out
    # Fig. 4: matching nu_hat instead of nu reduces the difference markedly (measured 26x)
    drho_h, du_h = out["nu_hat"]
    assert drho_h < drho / 10 and du_h < du / 10, out


@pytest.mark.parametrize("ratio,t_cmp,bounds", [(1.1, 361, (0.002, 0.02, 0.002)),
                                                (2.0, 327, (0.01, 0.03, 0.01))])
def test_d1q5_thermal_shock_tube_vs_exact(ratio, t_cmp, bounds):
    theta = 0.5
    left, right = (ratio, 0.0, theta), (1.0, 0.0, theta)
    _, (rho, ux, _, th) = _tube((0, 1, -1, 3, -3), 1.5, theta, left, right, t_cmp)
    x = np.arange(1000) + 0.5
    re, ue, pe = R.sample(R.State(ratio, 0.0, ratio * theta), R.State(1.0, 0.0, theta), 3.0,
                          (x - 500.0) / t_cmp)
    te = pe / re
    e_rho = np.mean(np.abs(rho[0] - re)) / np.mean(re)
    e_u = np.mean(np.abs(ux[0] - ue)) / np.max(np.abs(ue))
    e_th = np.mean(np.abs(th[0] - te)) / np.mean(te)
    assert e_rho < bounds[0] and e_u < bounds[1] and e_th < bounds[2]


def test_literal_shock_tube_leaves_positivity_region():
    theta_l, theta_r = 0.5, 0.4
    lat = O.Lattice(1, (0, 1, -1, 3, -3), 1.5, 1000, bc="fixed", theta0=0.5,
                    left_state=(1.0, 0.0, theta_l), right_state=(0.125, 0.0, theta_r))
    f = lat.init(*I.shock_tube_fields(1000, (1.0, 0.0, theta_l), (0.125, 0.0, theta_r)))
    bad_at = None
    for s in range(1, 101):
        f = lat.step(f)
        rho, _, _, th = lat.moments(f)
        if not (np.all(np.isfinite(rho)) and np.all(np.isfinite(th)) and rho.min() > 0 and th.min() > 0):
            bad_at = s
            break
    assert bad_at is not None and bad_at < 100
    # exact star-left temperature is below the u = 0 positivity floor a^2/3 = 1/3
    w = R.wave_speeds(R.State(1.0, 0.0, theta_l), R.State(0.125, 0.0, 0.125 * theta_r), 3.0)
    th_star_left = w["p_star"] / w["left_rho_star"]
    assert th_star_left < 1.0 / 3.0
