"""Exact Riemann solver for the 1D Euler equations of an ideal gas, FP64.

TEST INFRASTRUCTURE ONLY (part of the oracle).

Sec. 4 of the paper compares the thermal shock tube with "the analytical
solution of the Riemann problem for the Euler equations", prints the
Rankine-Hugoniot shock relations

    u_shock = sqrt((gamma+1)/2 (P - 1) + gamma),   u_post = (P - 1) / u_shock,

(velocities in units of sqrt(theta_pre), P = p_post / p_pre) and tabulates
p_post / p_pre against p_L / p_R for gamma = 1, 5/3, 2, 3 (Table 3).

Equation of state p = rho theta (theta = kT/m, Sec. 1), sound speed
a = sqrt(gamma theta).  The solver is the textbook exact method: the star
pressure p* is the root of f_L(p) + f_R(p) + (u_R - u_L) = 0, where each f_K is
the velocity jump across a shock (p > p_K) or a rarefaction (p <= p_K), and the
solution is self-similar in xi = (x - x0) / t.  gamma = 1 (isothermal) uses the
limits of those jumps: a (P - 1)/sqrt(P) across a shock, a ln P across a
rarefaction.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
from scipy.optimize import brentq


@dataclass
class State:
    rho: float
    u: float
    p: float


def _a(gamma: float, s: State) -> float:
    return math.sqrt(gamma * s.p / s.rho)


def _f_side(p: float, s: State, gamma: float) -> float:
    """Velocity jump u_K -> u* across the wave of side K, as a function of p*."""
    a = _a(gamma, s)
    if p > s.p:  # shock
        A = 2.0 / ((gamma + 1.0) * s.rho)
        B = (gamma - 1.0) / (gamma + 1.0) * s.p
        return (p - s.p) * math.sqrt(A / (p + B))
    if gamma == 1.0:
        return a * math.log(p / s.p)
    return 2.0 * a / (gamma - 1.0) * ((p / s.p) ** ((gamma - 1.0) / (2.0 * gamma)) - 1.0)


def star_state(left: State, right: State, gamma: float):
    """(p*, u*) of the Riemann problem."""
    g = lambda p: _f_side(p, left, gamma) + _f_side(p, right, gamma) + (right.u - left.u)
    lo = 1e-12 * min(left.p, right.p)
    hi = 10.0 * max(left.p, right.p)
    while g(hi) < 0:
        hi *= 10.0
    ps = brentq(g, lo, hi, xtol=1e-15, rtol=1e-15, maxiter=500)
    us = 0.5 * (left.u + right.u) + 0.5 * (_f_side(ps, right, gamma) - _f_side(ps, left, gamma))
    return ps, us


def _shock_density(s: State, ps: float, gamma: float) -> float:
    P = ps / s.p
    if gamma == 1.0:
        return s.rho * P
    m = (gamma - 1.0) / (gamma + 1.0)
    return s.rho * (P + m) / (m * P + 1.0)


def wave_speeds(left: State, right: State, gamma: float) -> dict:
    """Speeds of the left wave (head, tail), contact and right wave (head, tail)."""
    ps, us = star_state(left, right, gamma)
    out = {"p_star": ps, "u_star": us}
    for side, s, sgn in (("left", left, -1.0), ("right", right, 1.0)):
        a = _a(gamma, s)
        if ps > s.p:
            P = ps / s.p
            S = s.u + sgn * a * math.sqrt((gamma + 1.0) / (2.0 * gamma) * P + (gamma - 1.0) / (2.0 * gamma))
            out[side] = ("shock", S, S)
            out[side + "_rho_star"] = _shock_density(s, ps, gamma)
        else:
            rho_s = s.rho * (ps / s.p) ** (1.0 / gamma)
            a_s = math.sqrt(gamma * ps / rho_s)
            head = s.u + sgn * a
            tail = us + sgn * a_s
            out[side] = ("rarefaction", head, tail)
            out[side + "_rho_star"] = rho_s
    return out


def sample(left: State, right: State, gamma: float, xi: np.ndarray):
    """Exact (rho, u, p) at similarity coordinates xi = (x - x0) / t."""
    w = wave_speeds(left, right, gamma)
    ps, us = w["p_star"], w["u_star"]
    xi = np.asarray(xi, dtype=np.float64)
    rho = np.empty_like(xi)
    u = np.empty_like(xi)
    p = np.empty_like(xi)
    for k, x in np.ndenumerate(xi):
        if x <= us:
            s, sgn, kind, side = left, -1.0, w["left"], "left"
        else:
            s, sgn, kind, side = right, 1.0, w["right"], "right"
        a = _a(gamma, s)
        # position measured from the unperturbed side outwards
        if kind[0] == "shock":
            S = kind[1]
            if (x - S) * sgn >= 0.0:
                rho[k], u[k], p[k] = s.rho, s.u, s.p
            else:
                rho[k], u[k], p[k] = w[side + "_rho_star"], us, ps
            continue
        head, tail = kind[1], kind[2]
        if (x - head) * sgn >= 0.0:
            rho[k], u[k], p[k] = s.rho, s.u, s.p
        elif (x - tail) * sgn <= 0.0:
            rho[k], u[k], p[k] = w[side + "_rho_star"], us, ps
        else:  # inside the fan
            if gamma == 1.0:
                uu = x - sgn * a
                rr = s.rho * math.exp(sgn * (uu - s.u) / a)
                rho[k], u[k], p[k] = rr, uu, rr * s.p / s.rho
            else:
                g1 = gamma - 1.0
                uu = 2.0 / (gamma + 1.0) * (-sgn * a + 0.5 * g1 * s.u + x)
                c = 2.0 / (gamma + 1.0) * (a - sgn * 0.5 * g1 * (s.u - x))
                rr = s.rho * (c / a) ** (2.0 / g1)
                rho[k], u[k], p[k] = rr, uu, s.p * (c / a) ** (2.0 * gamma / g1)
    return rho, u, p


def pressure_ratio_post_pre(pl_over_pr: float, gamma: float) -> float:
    """Table 3: p_post/p_pre (= p*/p_R) for an equal-temperature shock tube at rest."""
    ps, _ = star_state(State(pl_over_pr, 0.0, pl_over_pr), State(1.0, 0.0, 1.0), gamma)
    return ps


def rh_shock_speed(P: float, gamma: float) -> float:
    """Printed Rankine-Hugoniot relation (Sec. 4): u_shock / sqrt(theta_pre)."""
    return math.sqrt((gamma + 1.0) / 2.0 * (P - 1.0) + gamma)


def rh_post_velocity(P: float, gamma: float) -> float:
    """Printed Rankine-Hugoniot relation (Sec. 4): u_post / sqrt(theta_pre)."""
    return (P - 1.0) / rh_shock_speed(P, gamma)
