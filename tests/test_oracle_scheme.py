"""Pins of the oracle's collision and streaming (Eq. eq:srt) against invariants.

* The BGK collision with n* = q-1 >= 2 conserves rho, rho u and the energy
  per node (thermal models); isothermal models conserve rho and rho u only.
* f^eq is a fixed point of the collision.
* With omega = 0 the step is a pure pull-stream: one population at one node
  moves by exactly its velocity (direction and population index pin).
* Periodic streaming permutes values, so global sums are invariant.
* A uniform equilibrium state is an exact fixed point of the whole step.
* Fixed ends feed the frozen f^eq(C_L), f^eq(C_R) ghost populations in.
"""
import numpy as np
import pytest

import oracle as O

V5 = (0, 1, -1, 3, -3)


def _random_state(lat, rng, scale=0.05):
    rho = 1.0 + scale * rng.uniform(-1, 1)
    ux, uy = scale * rng.uniform(-1, 1, 2)
    th = lat.theta0 * (1.0 + scale * rng.uniform(-1, 1))
    f = O.feq(lat.dim, lat.v, rho, ux, uy, th)
    return f * (1.0 + 0.2 * rng.uniform(-1, 1, f.size))


def _node_sums(lat, f):
    vel = lat.velocities().astype(float)
    vx = vel[:, 0]
    vy = vel[:, 1] if lat.dim == 2 else np.zeros_like(vx)
    return np.array([f.sum(), (vx * f).sum(), (vy * f).sum(), ((vx * vx + vy * vy) * f).sum()])


@pytest.mark.parametrize("dim,v,omega,theta0", [
    (1, V5, 1.5, 0.5), (2, V5, 1.3, 1.0), (2, (0, 1, -1, 2, -2), 1.9, 0.39), (1, (0, 2, -4, 1), 1.1, 0.8)])
def test_collision_conserves_mass_momentum_energy(dim, v, omega, theta0):
    lat = O.Lattice(dim, v, omega, 4, 4, theta0=theta0)
    rng = np.random.default_rng(7)
    for _ in range(20):
        f = _random_state(lat, rng)
        g = lat.collide_node(f)
        s0, s1 = _node_sums(lat, f), _node_sums(lat, g)
        assert np.max(np.abs(s1 - s0)) <= 1e-13 * max(1.0, np.max(np.abs(s0)))
        assert np.max(np.abs(g - f)) > 1e-4  # not the identity


def test_isothermal_collision_conserves_mass_momentum_only():
    lat = O.Lattice(2, (0, 1, -1), 1.0, 4, 4, theta0=0.25, isothermal=True)
    rng = np.random.default_rng(3)
    f = _random_state(lat, rng, scale=0.1)
    g = lat.collide_node(f)
    s0, s1 = _node_sums(lat, f), _node_sums(lat, g)
    assert np.max(np.abs(s1[:3] - s0[:3])) < 1e-14
    assert abs(s1[3] - s0[3]) > 1e-5


@pytest.mark.parametrize("dim", [1, 2])
def test_equilibrium_is_collision_fixed_point(dim):
    lat = O.Lattice(dim, V5, 1.7, 4, 4, theta0=0.8)
    for rho, ux, uy, th in [(1.0, 0.0, 0.0, 0.8), (0.9, 0.12, -0.07, 0.95), (1.3, -0.2, 0.1, 0.6)]:
        f = O.feq(dim, V5, rho, ux, uy, th)
        assert np.max(np.abs(lat.collide_node(f) - f)) < 2e-15
        r, a, b, t = lat.node_moments(f)
        assert abs(r - rho) < 1e-15 and abs(a - ux) < 1e-15 and abs(t - th) < 1e-14
        if dim == 2:
            assert abs(b - uy) < 1e-15


def test_pure_stream_moves_each_population_by_its_velocity():
    nx, ny = 11, 9
    lat = O.Lattice(2, V5, 0.0, nx, ny, theta0=1.0)  # omega = 0: streaming only
    vel = lat.velocities()
    rng = np.random.default_rng(1)
    f = rng.uniform(0.5, 1.5, lat.shape)
    g = lat.step(f)
    for p in range(lat.q):
        vx, vy = vel[p]
        assert np.array_equal(g[p], np.roll(np.roll(f[p], vx, axis=1), vy, axis=0)), p
    # population index p = ix*q1 + iy carries velocity (v[ix], v[iy])
    assert tuple(vel[1 * 5 + 3]) == (1, 3) and tuple(vel[4 * 5 + 2]) == (-3, -1)


def test_pure_stream_1d_fixed_ends():
    n = 20
    left, right = (1.2, 0.1, 0.5), (0.9, -0.05, 0.45)
    lat = O.Lattice(1, V5, 0.0, n, bc="fixed", theta0=0.5, left_state=left, right_state=right)
    rng = np.random.default_rng(2)
    f = rng.uniform(0.5, 1.5, lat.shape)
    g = lat.step(f)
    gl = O.feq(1, V5, left[0], left[1], 0.0, left[2])
    gr = O.feq(1, V5, right[0], right[1], 0.0, right[2])
    for p, vp in enumerate(V5):
        for x in range(n):
            s = x - vp
            ref = gl[p] if s < 0 else (gr[p] if s >= n else f[p, 0, s])
            assert g[p, 0, x] == ref


@pytest.mark.parametrize("dim,shape,steps", [(2, (33, 17), 40), (2, (7, 5), 10000), (2, (1, 1), 10000),
                                              (1, (50, 1), 10000)])
def test_periodic_global_sums_invariant(dim, shape, steps):
    nx, ny = shape
    lat = O.Lattice(dim, V5, 1.3, nx, ny, theta0=1.0)
    rng = np.random.default_rng(5)
    rho = 1 + 0.01 * rng.uniform(-1, 1, (lat.ny, nx))
    ux = 0.05 * rng.uniform(-1, 1, (lat.ny, nx))
    uy = 0.05 * rng.uniform(-1, 1, (lat.ny, nx))
    th = 1 + 0.01 * rng.uniform(-1, 1, (lat.ny, nx))
    f = lat.init(rho, ux, uy, th)
    c0 = lat.conserved(f)
    f = lat.run(f, steps)
    c1 = lat.conserved(f)
    assert np.all(np.isfinite(f))
    assert np.max(np.abs(c1 - c0)) <= 1e-12 * np.max(np.abs(c0))


def test_uniform_state_is_fixed_point_of_step():
    lat = O.Lattice(2, V5, 1.3, 12, 10, theta0=1.0)
    f = lat.init(1.05, 0.07, -0.04, 0.97)
    g = lat.run(f, 10)
    assert np.max(np.abs(g - f)) < 1e-15


def test_init_reproduces_fields():
    lat = O.Lattice(2, V5, 1.3, 16, 8, theta0=1.0)
    rng = np.random.default_rng(9)
    rho = 1 + 0.02 * rng.uniform(-1, 1, (8, 16))
    ux = 0.1 * rng.uniform(-1, 1, (8, 16))
    uy = 0.1 * rng.uniform(-1, 1, (8, 16))
    th = 1 + 0.02 * rng.uniform(-1, 1, (8, 16))
    f = lat.init(rho, ux, uy, th)
    r, a, b, t = lat.moments(f)
    for x, y in ((r, rho), (a, ux), (b, uy), (t, th)):
        assert np.max(np.abs(x - y)) < 1e-14


@pytest.mark.parametrize("dim,nx,ny", [(2, 11, 7), (1, 23, 1)])
def test_conserved_sums_equal_sums_of_the_node_moments(dim, nx, ny):
    """orc_conserved against the fields of orc_moments (reading R3:
    rho = sum f, rho u = sum v f, d rho theta = sum |v - u|^2 f, so that
    sum |v|^2 f = rho (|u|^2 + d theta)) on a random, far-from-equilibrium
    state whose momentum components differ: a swapped or rescaled component or
    a dropped energy term cannot match."""
    lat = O.Lattice(dim, V5, 1.3, nx, ny, theta0=1.0)
    rng = np.random.default_rng(31)
    f = rng.uniform(0.2, 1.8, lat.shape) * (1.0 + 0.5 * rng.uniform(0, 1, (lat.q, 1, 1)))
    rho, ux, uy, th = lat.moments(f)
    ref = np.array([rho.sum(), (rho * ux).sum(), (rho * uy).sum(),
                    (rho * (ux * ux + uy * uy + dim * th)).sum()])
    got = lat.conserved(f)
    assert abs(ref[1]) > 1e-2 * ref[0]
    if dim == 2:
        assert abs(ref[1] - ref[2]) > 1e-2 * ref[0]
    assert np.max(np.abs(got - ref)) <= 1e-12 * ref[0], (got, ref)


def test_conserved_sums_of_an_equilibrium_are_the_field_integrals():
    """For f = f^eq(rho, u, theta) the moment identity of Eq. (eq:rdr) (mu_0..mu_2
    reproduced) makes the sums exactly sum rho, sum rho u and
    sum rho (|u|^2 + 2 theta) of the fields that built it."""
    lat = O.Lattice(2, V5, 1.3, 13, 9, theta0=1.0)
    rng = np.random.default_rng(32)
    rho = 1 + 0.1 * rng.uniform(-1, 1, (9, 13))
    ux = 0.08 * rng.uniform(-0.2, 1, (9, 13))
    uy = 0.08 * rng.uniform(-1, 0.3, (9, 13))
    th = 1 + 0.1 * rng.uniform(-1, 1, (9, 13))
    got = lat.conserved(lat.init(rho, ux, uy, th))
    ref = np.array([rho.sum(), (rho * ux).sum(), (rho * uy).sum(), (rho * (ux * ux + uy * uy + 2 * th)).sum()])
    assert np.max(np.abs(got - ref)) <= 1e-12 * ref[0], (got, ref)
