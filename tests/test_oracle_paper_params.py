"""The paper's own parameters (Sec. 4): the 25-velocity shear layer and the
five-velocity shock tube on the lattice set {0, +-1, +-2} = {0, +-a, +-2a} sqrt(theta0)
with theta0 = 1 / a^2 (a = 1.6 and 1.4), omega = 1.9.

* The shear-layer parameters are linearly stable (spectral radius of the
  linearised one-step operator <= 1) and keep every r_i >= 0 up to the initial
  velocity amplitude, as the paper's run at omega = 1.9 ("close to the upper
  limit") needs.
* The shear layer at omega = 1.9 is stable in FP64 to the paper's last printed
  step (3695) but carries a mode that grows from a perturbation of relative size
  1e-7 (FP32 rounding level) and ruins the flow before step 3695.
* The shock tube rho_L / rho_R = 1.1 at a = 1.4: the post-shock plateau values of
  u, rho and theta (the quantities the paper compares with the exact Riemann
  solution) agree with the exact gamma = 3 solution.
"""
import math

import numpy as np
import pytest

import oracle as O
from oracle import riemann as R
from oracle import stability as S
from paper_1402_5487_gb300 import inputs as I

SET_012 = (0, 1, -1, 2, -2)


def test_paper_shear_layer_parameters_are_stable_and_positive():
    fields, theta0 = I.paper_kh_fields()
    assert abs(theta0 - 1 / 2.56) < 1e-15
    u_max = float(np.max(np.abs(fields[1])))
    assert abs(u_max - 0.069 / 1.6) < 1e-3
    lat = O.Lattice(2, SET_012, 1.9, 4, 4, theta0=theta0)
    for ux in (0.0, u_max):
        assert S.spectral_radius(lat, 24, 1.0, ux, 0.0, theta0, axis_refine=4) <= 1 + 1e-9
    lo, hi = S.positivity_interval(SET_012, theta0)
    assert lo < -u_max and hi > u_max


@pytest.mark.slow
def test_paper_shear_layer_grows_a_seeded_mode():
    fields, theta0 = I.paper_kh_fields()
    rng = np.random.default_rng(1)
    u0 = float(np.max(np.abs(fields[1])))
    seeded = (fields[0], fields[1] + 1e-7 * u0 * rng.uniform(-1, 1, fields[1].shape), fields[2], fields[3])
    lat = O.Lattice(2, SET_012, 1.9, 128, 128, theta0=theta0)
    th_min = {}
    for name, f0 in (("plain", fields), ("seeded", seeded)):
        f = lat.run(lat.init(*f0), 3500)
        th_min[name] = float(lat.moments(f)[3].min() / theta0)
    assert th_min["plain"] > 0.995, th_min
    assert th_min["seeded"] < 0.95, th_min


def test_paper_d1q5_shock_tube_plateau_values():
    theta = 1 / 1.96
    left, right = (1.1, 0.0, theta), (1.0, 0.0, theta)
    lat = O.Lattice(1, SET_012, 1.9, 1000, bc="fixed", theta0=theta, left_state=left, right_state=right)
    t = 346
    rho, ux, _, th = lat.moments(lat.run(lat.init(*I.shock_tube_fields(1000, left, right)), t))
    x = np.arange(1000) + 0.5
    re, ue, pe = R.sample(R.State(1.1, 0.0, 1.1 * theta), R.State(1.0, 0.0, theta), 3.0, (x - 500.0) / t)
    te = pe / re
    plateau = np.nonzero(np.abs(ue - ue.max()) < 1e-12)[0]
    core = plateau[(plateau > plateau.min() + 30) & (plateau < plateau.max() - 30)]
    assert core.size > 100
    for sim, ex in ((ux[0], ue), (rho[0], re), (th[0], te)):
        assert abs(sim[core].mean() / ex[core].mean() - 1) < 5e-3
