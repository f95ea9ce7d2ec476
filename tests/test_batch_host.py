"""Host-side gates of the batched sweep against the oracle (CPU only).

The library screens parameter draws with its own positivity test (Sec. 3.1) and
von Neumann analysis (complex-step Jacobian + its own eigenvalue routine); the
oracle does the same with NumPy (central differences + numpy.linalg.eigvals).
"""
import numpy as np
import pytest

import oracle as O
from oracle import stability as S
from paper_1402_5487_gb300 import batch as B, build, inputs as I, plbm


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    plbm.lib()


@pytest.mark.parametrize("v,omega,theta,ux,iso", [
    (I.SET_013, 1.3, 1.0, 0.0, False), (I.SET_013, 1.8, 1.0, 0.0, False), (I.SET_013, 1.3, 1.0, 0.1, False),
    (I.SET_012, 1.9, 0.6, 0.1, False), (I.SET_012, 1.5, 0.95, 0.1, False), (I.SET_012, 1.0, 0.7, 0.05, False),
    (I.SET_013, 1.7, 0.6, 0.1, False), ((0, 1, -1), 1.2, 0.25, 0.05, True), ((0, 1, -1), 1.99, 1 / 3, 0.1, True),
    ((1, -1, 3, -3), 1.1, 4 / 3, 0.0, True)])
def test_library_spectral_radius_matches_oracle(v, omega, theta, ux, iso):
    got = plbm.linear_stability(2, v, omega, theta, ux, nk=12, isothermal=iso)
    lat = O.Lattice(2, v, omega, 4, 4, theta0=theta, isothermal=iso)
    ref = S.spectral_radius(lat, n=12, ux=ux, axis_refine=8)
    # the oracle's central-difference Jacobian is good to ~1e-10
    assert abs(got - ref) < 1e-8, (got, ref)


@pytest.mark.parametrize("v", [I.SET_013, I.SET_012, I.SET_023, (0, 1, -1), (0, 2, -4)])
@pytest.mark.parametrize("theta", [0.25, 0.6, 1.0, 1.7])
def test_library_positivity_matches_oracle(v, theta):
    iv = S.positivity_interval(v, theta)
    for u_max in (0.0, 0.05, 0.1, 0.3):
        got = plbm.positivity(2, v, theta, u_max)
        oracle_ok = iv is not None and iv[0] <= -u_max and iv[1] >= u_max
        # sampling at 401 points can miss a violation only within a grid step of the edge
        if iv is not None and min(abs(iv[0] + u_max), abs(iv[1] - u_max)) < 2e-3 * max(u_max, 1e-3):
            continue
        assert (got >= 0.0) == oracle_ok, (v, theta, u_max, got, iv)


def test_draws_are_admissible_and_deterministic():
    inst, stats = B.draw_instances(24, seed=77)
    inst2, _ = B.draw_instances(24, seed=77)
    assert [(a.L, a.v, a.omega, a.theta0) for a in inst] == [(a.L, a.v, a.omega, a.theta0) for a in inst2]
    assert all(64 <= a.L <= 1024 for a in inst)
    assert any(a.L % 2 for a in inst) and any(a.L % 2 == 0 for a in inst)   # R10: every integer side
    assert all(a.v != I.SET_023 for a in inst)  # its u = 0 window is 4/3 < theta < 3
    for a in inst[:6]:
        lat = O.Lattice(2, a.v, a.omega, 4, 4, theta0=a.theta0)
        u_max = 0.1 if a.kind == "kh" else 1e-3
        assert S.spectral_radius(lat, n=12, ux=u_max) <= 1 + 1e-8
        assert S.spectral_radius(lat, n=12) <= 1 + 1e-8
    assert 0 < stats["acceptance"] <= 1
