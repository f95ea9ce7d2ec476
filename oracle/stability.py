"""Linear analysis tools of the oracle (FP64, NumPy).

TEST INFRASTRUCTURE ONLY (part of the oracle).

* ``collision_jacobian``: J = d(collide)/d(f_in) at a uniform equilibrium,
  by central differences through the C oracle's BGK collision (Eq. eq:srt).
* ``step_operator``: the one-step map of a Fourier mode exp(i k.x),
  A(k) = J S(k) with S(k) = diag(exp(-i k.v_p)) for the pull of
  f_in,p(x) = f_p(x - v_p).
* ``hydro_modes``: eigenvalues of A(k) closest to 1 at a small k; their decay
  -ln|lambda| / k^2 is compared with nu = (1/omega - 1/2) theta (Sec. 2.1) and
  their phase speed with the adiabatic sound speed sqrt(gamma theta),
  gamma = (d+2)/d.  With kappa = (d+2)/2 nu rho the thermal diffusivity
  kappa / (rho c_p) equals nu, and the sound attenuation also equals nu, so
  every hydrodynamic mode decays at nu k^2.
* ``spectral_radius``: max |lambda(k)| over a k-grid (von Neumann stability).
* ``positivity_interval``: the interval of u around 0 with all r_i >= 0.
"""
from __future__ import annotations

import numpy as np

from . import Lattice, feq, r1d


def collision_jacobian(lat: Lattice, rho=1.0, ux=0.0, uy=0.0, theta=None, h=1e-6):
    theta = lat.theta0 if theta is None else theta
    f0 = feq(lat.dim, lat.v, rho, ux, uy, theta)
    J = np.zeros((lat.q, lat.q))
    for p in range(lat.q):
        e = np.zeros(lat.q)
        e[p] = h
        J[:, p] = (lat.collide_node(f0 + e) - lat.collide_node(f0 - e)) / (2.0 * h)
    return J


def step_operator(lat: Lattice, J: np.ndarray, kx: float, ky: float = 0.0) -> np.ndarray:
    vel = lat.velocities().astype(np.float64)
    phase = kx * vel[:, 0] + (ky * vel[:, 1] if lat.dim == 2 else 0.0)
    S = np.exp(-1j * phase)
    return J * S[np.newaxis, :]


def hydro_modes(lat: Lattice, k: float, rho=1.0, ux=0.0, uy=0.0, theta=None, J=None):
    """Eigenvalues of A(k along x), sorted by |lambda| descending (hydrodynamic first)."""
    if J is None:
        J = collision_jacobian(lat, rho, ux, uy, theta)
    lam = np.linalg.eigvals(step_operator(lat, J, k, 0.0))
    return lam[np.argsort(-np.abs(lam))]


def spectral_radius(lat: Lattice, n=32, rho=1.0, ux=0.0, uy=0.0, theta=None, axis_refine=1) -> float:
    """max |lambda| over the k-grid 2 pi (a, b) / n; with axis_refine > 1 the two k
    axes are also sampled at n * axis_refine points."""
    J = collision_jacobian(lat, rho, ux, uy, theta)
    ks = 2.0 * np.pi * np.arange(n) / n
    pts = [(kx, ky) for kx in ks for ky in (ks if lat.dim == 2 else [0.0])]
    if axis_refine > 1:
        fine = 2.0 * np.pi * np.arange(n * axis_refine) / (n * axis_refine)
        pts += [(k, 0.0) for k in fine]
        if lat.dim == 2:
            pts += [(0.0, k) for k in fine]
    best = 0.0
    for kx, ky in pts:
        lam = np.linalg.eigvals(step_operator(lat, J, kx, ky))
        best = max(best, float(np.max(np.abs(lam))))
    return best


def positivity_interval(v, theta: float, umax: float = 10.0, tol: float = 1e-13):
    """Largest interval [u_lo, u_hi] containing 0 with min_i r_i(u, theta) >= 0.

    Returns None if r_i(0, theta) already has a negative entry.  Ends found by
    bisection on min_i r_i (continuous in u).
    """
    from . import vandermonde_inverse
    C = vandermonde_inverse(v)
    g = lambda u: float(np.min(r1d(v, u, theta, C)))
    if g(0.0) < 0.0:
        return None
    ends = []
    for sgn in (1.0, -1.0):
        a, b = 0.0, sgn * umax
        if g(b) >= 0.0:
            ends.append(b)
            continue
        while abs(b - a) > tol:
            m = 0.5 * (a + b)
            if g(m) >= 0.0:
                a = m
            else:
                b = m
        ends.append(a)
    return ends[1], ends[0]


def positivity_theta_window(v, tol: float = 1e-13, tmax: float = 100.0):
    """Interval of theta with all r_i(0, theta) >= 0, by bisection from its midpoint scan."""
    from . import vandermonde_inverse
    C = vandermonde_inverse(v)
    g = lambda t: float(np.min(r1d(v, 0.0, t, C)))
    ts = np.linspace(1e-6, tmax, 200001)
    ok = np.array([g(t) >= 0 for t in ts[::100]])
    if not ok.any():
        return None
    idx = np.nonzero(ok)[0]
    lo_i, hi_i = idx[0] * 100, idx[-1] * 100
    t_in = ts[(lo_i + hi_i) // 2]

    def edge(a, b):
        while abs(b - a) > tol:
            m = 0.5 * (a + b)
            if g(m) >= 0.0:
                a = m
            else:
                b = m
        return a

    lo = edge(t_in, 1e-9)
    hi = edge(t_in, tmax)
    return lo, hi
