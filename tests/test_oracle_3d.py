"""Pins of the three-dimensional oracle (Sec. 2.1: D3 models are the tensor
product of three 1D rules).

* Isothermal runs with fields uniform along one axis reduce exactly to the 2D
  oracle on the other two axes (the marginal over that axis's velocity index):
  pins the population index, the three stream directions and the tensor
  product, against the independently pinned 2D code.
* Collision conserves mass, momentum and energy per node; f^eq is a fixed point.
* omega = 0 moves every population by exactly its velocity.
* A shear wave decays at nu k^2, nu = (1/omega - 1/2) theta (Sec. 2.1).
* An adiabatic sound wave travels at sqrt(gamma theta), gamma = (d + 2)/d = 5/3.
* Plausible one-spot mistakes in the 3D code are rejected by these pins.
"""
import math
import os
import tempfile

import numpy as np
import pytest

import oracle as O

V5 = (0, 1, -1, 3, -3)


def _smooth(n, rng, amp):
    """A smooth periodic random field on n points."""
    x = np.arange(n)
    return sum(amp * rng.uniform(-1, 1) * np.cos(2 * np.pi * m * x / n + rng.uniform(0, 6.3)) for m in (1, 2))


@pytest.mark.parametrize("axis", ["z", "y", "x"])
def test_isothermal_3d_uniform_along_one_axis_is_the_2d_model(axis):
    rng = np.random.default_rng(11)
    n1, n2, n3 = 7, 6, 5                     # sizes of the two varying axes and the uniform one
    theta0, omega, steps = 1.0, 1.2, 15
    a = _smooth(n1, rng, 0.02)[None, :] + _smooth(n2, rng, 0.02)[:, None]   # [n2][n1]
    b = _smooth(n1, rng, 0.02)[None, :] * _smooth(n2, rng, 1.0)[:, None]
    rho = 1.0 + 0.01 * np.cos(2 * np.pi * np.arange(n1) / n1)[None, :] * np.ones((n2, 1))
    lat2 = O.Lattice(2, V5, omega, n1, n2, theta0=theta0, isothermal=True)
    f2 = lat2.run(lat2.init(rho, a, b), steps)
    q1 = len(V5)
    if axis == "z":   # 2D (x, y) = 3D (x, y)
        lat3 = O.Lattice3(V5, omega, n1, n2, n3, theta0=theta0, isothermal=True)
        F = lambda g: np.broadcast_to(g[None], (n3, n2, n1))
        f3 = lat3.run(lat3.init(F(rho), F(a), F(b), 0.0), steps).reshape(q1, q1, q1, n3, n2, n1)
        marg = f3.sum(axis=2)[:, :, 0]                         # sum over iz, any z
    elif axis == "y":  # 2D (x, y) = 3D (x, z)
        lat3 = O.Lattice3(V5, omega, n1, n3, n2, theta0=theta0, isothermal=True)
        F = lambda g: np.broadcast_to(g[:, None, :], (n2, n3, n1))
        f3 = lat3.run(lat3.init(F(rho), F(a), 0.0, F(b)), steps).reshape(q1, q1, q1, n2, n3, n1)
        marg = f3.sum(axis=1)[:, :, :, 0, :]                   # sum over iy, any y
    else:              # 2D (x, y) = 3D (y, z)
        lat3 = O.Lattice3(V5, omega, n3, n1, n2, theta0=theta0, isothermal=True)
        F = lambda g: np.broadcast_to(g[:, :, None], (n2, n1, n3))
        f3 = lat3.run(lat3.init(F(rho), 0.0, F(a), F(b)), steps).reshape(q1, q1, q1, n2, n1, n3)
        marg = f3.sum(axis=0)[:, :, :, :, 0]                   # sum over ix, any x
    ref = f2.reshape(q1, q1, n2, n1)
    assert np.max(np.abs(marg - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_collision_conserves_and_equilibrium_is_fixed_point():
    lat = O.Lattice3(V5, 1.4, 2, 2, 2, theta0=0.9)
    feq = lat.feq(1.05, 0.03, -0.02, 0.04, 0.95)
    m = lat.node_moments(feq)
    assert abs(m[0] - 1.05) < 1e-14 and abs(m[1] - 0.03) < 1e-14 and abs(m[4] - 0.95) < 1e-13
    assert np.max(np.abs(lat.collide_node(feq) - feq)) < 1e-15
    rng = np.random.default_rng(3)
    fin = feq * (1 + 0.05 * rng.uniform(-1, 1, feq.size))
    out = lat.collide_node(fin)
    vel = lat.velocities()
    for w in (np.ones(len(vel)), vel[:, 0], vel[:, 1], vel[:, 2], (vel ** 2).sum(1)):
        assert abs(np.dot(w, out) - np.dot(w, fin)) < 1e-13 * max(1.0, abs(np.dot(w, fin)))


def test_pure_streaming_moves_each_population_by_its_velocity():
    lat = O.Lattice3(V5, 0.0, 9, 8, 7)
    rng = np.random.default_rng(5)
    f = rng.uniform(0.0, 1.0, lat.shape)
    g = lat.step(f)
    for p, (cx, cy, cz) in enumerate(lat.velocities()):
        expect = np.roll(np.roll(np.roll(f[p], cz, axis=0), cy, axis=1), cx, axis=2)
        assert np.array_equal(g[p], expect), p


def test_shear_wave_decays_at_nu_k2():
    L, theta0, omega = 48, 1.0, 1.3
    lat = O.Lattice3(V5, omega, 2, 2, L, theta0=theta0)
    z = np.arange(L)
    k = 2 * np.pi / L
    ux = 1e-3 * np.sin(k * z)[:, None, None] * np.ones((L, 2, 2))
    f = lat.init(1.0, ux)
    nu = (1 / omega - 0.5) * theta0
    amps = []
    for _ in range(3):
        f = lat.run(f, 80)
        u = lat.moments(f)[1]
        amps.append(np.sum(u[:, 0, 0] * np.sin(k * z)) * 2 / L)
    rate = -math.log(amps[2] / amps[0]) / (k * k * 160)
    assert abs(rate / nu - 1) < 0.01


def test_adiabatic_sound_wave_travels_at_sqrt_gamma_theta():
    L, theta0, omega, eps = 64, 1.0, 1.5, 1e-4
    gamma = 5.0 / 3.0
    c = math.sqrt(gamma * theta0)
    lat = O.Lattice3(V5, omega, 1, 1, L, theta0=theta0)
    z = np.arange(L)
    k = 2 * np.pi / L
    s = np.cos(k * z)[:, None, None]
    f = lat.init(1 + eps * s, 0.0, 0.0, eps * c * s, theta0 * (1 + (gamma - 1) * eps * s))
    phases = []
    for _ in range(4):
        f = lat.run(f, 10)
        rho = lat.moments(f)[0][:, 0, 0]
        phases.append(np.angle(np.sum((rho - rho.mean()) * np.exp(-1j * k * z))))
    speed = -np.mean(np.diff(np.unwrap(phases))) / (10 * k)
    assert abs(speed / c - 1) < 0.01


def test_conserved_sums_equal_sums_of_the_node_moments():
    """orc3_conserved against the fields of orc3_moments on a random state
    (sum |v|^2 f = rho (|u|^2 + 3 theta), reading R3 with d = 3)."""
    lat = O.Lattice3(V5, 1.3, 5, 4, 3, theta0=1.0)
    rng = np.random.default_rng(33)
    q = len(V5) ** 3
    f = rng.uniform(0.2, 1.8, (q, 3, 4, 5)) * (1.0 + 0.5 * rng.uniform(0, 1, (q, 1, 1, 1)))
    rho, ux, uy, uz, th = lat.moments(f)
    ref = np.array([rho.sum(), (rho * ux).sum(), (rho * uy).sum(), (rho * uz).sum(),
                    (rho * (ux * ux + uy * uy + uz * uz + 3 * th)).sum()])
    assert min(abs(ref[1] - ref[2]), abs(ref[2] - ref[3]), abs(ref[1] - ref[3])) > 1e-2 * ref[0]
    got = lat.conserved(f)
    assert np.max(np.abs(got - ref)) <= 1e-12 * ref[0], (got, ref)


# --------------------------------------------------------------------------
# Mutants of the 3D code: each must fail at least one pin above.
# --------------------------------------------------------------------------
MUTANTS_3D = [
    ("stream z direction", "const int pz = orc3_wrap(z - L->v[c], nz);", "const int pz = orc3_wrap(z + L->v[c], nz);"),
    ("stream x uses z velocity", "const int px = orc3_wrap(x - L->v[a], nx);", "const int px = orc3_wrap(x - L->v[c], nx);"),
    ("z factor uses u_y", "orc_r1d(q1, C, uz, theta, rc);", "orc_r1d(q1, C, uy, theta, rc);"),
    ("theta divides by 2", "m_out[4] = (en / m0 - (wx * wx + wy * wy + wz * wz)) / 3.0;",
     "m_out[4] = (en / m0 - (wx * wx + wy * wy + wz * wz)) / 2.0;"),
    ("energy drops c_z^2", "en = en + (cx * cx + cy * cy + cz * cz) * fv;", "en = en + (cx * cx + cy * cy) * fv;"),
    ("population index transposed", "fi[p] = fsrc[p * vol + ((long)pz * ny + py) * nx + px];",
     "fi[p] = fsrc[((c * q1 + b) * q1 + a) * vol + ((long)pz * ny + py) * nx + px];"),
    ("conserved y and z momentum swapped", "neu_add(&s[2], &c[2], cy * fv);\n                    neu_add(&s[3], &c[3], cz * fv);",
     "neu_add(&s[2], &c[2], cz * fv);\n                    neu_add(&s[3], &c[3], cy * fv);"),
    ("conserved energy drops c_z^2", "neu_add(&s[4], &c[4], (cx * cx + cy * cy + cz * cz) * fv);",
     "neu_add(&s[4], &c[4], (cx * cx + cy * cy) * fv);"),
]


def _battery3():
    fails = []
    for name, fn in (("reduction z", lambda: test_isothermal_3d_uniform_along_one_axis_is_the_2d_model("z")),
                     ("reduction y", lambda: test_isothermal_3d_uniform_along_one_axis_is_the_2d_model("y")),
                     ("reduction x", lambda: test_isothermal_3d_uniform_along_one_axis_is_the_2d_model("x")),
                     ("conservation", test_collision_conserves_and_equilibrium_is_fixed_point),
                     ("streaming", test_pure_streaming_moves_each_population_by_its_velocity),
                     ("sound", test_adiabatic_sound_wave_travels_at_sqrt_gamma_theta),
                     ("conserved sums", test_conserved_sums_equal_sums_of_the_node_moments)):
        try:
            fn()
        except Exception:
            fails.append(name)
    return fails


@pytest.mark.parametrize("name,orig,repl", MUTANTS_3D, ids=[m[0] for m in MUTANTS_3D])
def test_3d_pins_reject_mutant(name, orig, repl):
    src = O.source_text()
    assert src.count(orig) == 1, name
    with tempfile.TemporaryDirectory() as d:
        path = O.compile_variant(src.replace(orig, repl), os.path.join(d, "mutant3.so"))
        with O.using_library(path):
            fails = _battery3()
    assert fails, name
