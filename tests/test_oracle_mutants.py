"""The oracle's pins reject plausible mistakes.

Each case edits one spot of the oracle's C source (a dropped term, a flipped
sign, a swapped index or operand), compiles that copy with the oracle's flags
and reruns a battery of the pins from the other oracle tests through it.  The
battery must fail for every mutant and pass for the unmodified source.
"""
import math
import os
import tempfile

import numpy as np
import pytest

import oracle as O
from oracle import stability as S
from paper_1402_5487_gb300 import inputs as I

V5 = (0, 1, -1, 3, -3)

# (name, original text, replacement); each original must occur exactly once.
MUTANTS = [
    ("stream direction", "int sx = x - L->v[ix];", "int sx = x + L->v[ix];"),
    ("stream y direction", "int sy = (L->dim == 1) ? 0 : y - L->v[iy];",
     "int sy = (L->dim == 1) ? 0 : y + L->v[iy];"),
    ("stream population transpose", "int ix = (L->dim == 1) ? p : p / q1;\n                int iy = (L->dim == 1) ? 0 : p % q1;",
     "int ix = (L->dim == 1) ? p : p % q1;\n                int iy = (L->dim == 1) ? 0 : p / q1;"),
    ("wrap y with nx", "sy = ((sy % ny) + ny) % ny;", "sy = ((sy % nx) + nx) % nx;"),
    ("recurrence factor", "mu[n + 1] = u * mu[n] + n * theta * mu[n - 1];",
     "mu[n + 1] = u * mu[n] + (n + 1) * theta * mu[n - 1];"),
    ("recurrence dropped term", "mu[n + 1] = u * mu[n] + n * theta * mu[n - 1];",
     "mu[n + 1] = u * mu[n];"),
    ("coefficient transpose", "C[i * q + n] = A[i][q + n];", "C[i * q + n] = A[n][q + i];"),
    ("rdr index", "s = s + C[i * q1 + n] * mu[n];", "s = s + C[n * q1 + i] * mu[n];"),
    ("tensor product uses ux twice", "orc_r1d(q1, C, uy, theta, ry);", "orc_r1d(q1, C, ux, theta, ry);"),
    ("bgk weight", "fout[p] = (1.0 - L->omega) * fin[p] + L->omega * feq[p];",
     "fout[p] = (1.0 - L->omega) * fin[p] + feq[p];"),
    ("bgk sign", "fout[p] = (1.0 - L->omega) * fin[p] + L->omega * feq[p];",
     "fout[p] = (1.0 + L->omega) * fin[p] - L->omega * feq[p];"),
    ("theta without 1/d", "double theta = (e / rho - (ux * ux + uy * uy)) / L->dim;",
     "double theta = (e / rho - (ux * ux + uy * uy));"),
    ("theta drops u^2", "double theta = (e / rho - (ux * ux + uy * uy)) / L->dim;",
     "double theta = (e / rho) / L->dim;"),
    ("energy drops vy^2", "e = e + (vx * vx + vy * vy) * f[p];", "e = e + (vx * vx) * f[p];"),
    ("momentum y uses vx", "jy = jy + vy * f[p];", "jy = jy + vx * f[p];"),
    ("ghosts swapped", "if (sx < 0) { fin[p] = L->ghost_left[p]; continue; }",
     "if (sx < 0) { fin[p] = L->ghost_right[p]; continue; }"),
    ("vandermonde power off by one", "for (int e = 0; e < n; ++e) p = p * v[k];",
     "for (int e = 0; e <= n; ++e) p = p * v[k];"),
    ("elimination skips a row", "if (r == col) continue;", "if (r <= col) continue;"),
    ("conserved momentum components swapped",
     "neu_add(&s[1], &c[1], vx * fv);\n            neu_add(&s[2], &c[2], vy * fv);",
     "neu_add(&s[1], &c[1], vy * fv);\n            neu_add(&s[2], &c[2], vx * fv);"),
    ("conserved energy drops vy^2", "neu_add(&s[3], &c[3], (vx * vx + vy * vy) * fv);",
     "neu_add(&s[3], &c[3], (vx * vx) * fv);"),
]


def _battery():
    """Returns the list of failing pin names (empty = all pins hold)."""
    fails = []

    def check(name, cond):
        if not cond:
            fails.append(name)

    # coefficients: Lagrange property and the explicit formula of Eq. (eq:1d5v)
    for v in (V5, (0, 2, -4), (1, -1, 3, -3)):
        C = O.vandermonde_inverse(v)
        Vm = np.array([[float(vk) ** n for vk in v] for n in range(len(v))])
        check("lagrange", np.max(np.abs(C @ Vm - np.eye(len(v)))) < 1e-12)
    u, t = 0.1, 0.8
    mu = [1.0, u, t + u * u, 3 * t * u + u ** 3, 3 * t * t + 6 * t * u * u + u ** 4]
    check("table2 mb row", np.max(np.abs(O.mb_moments(u, t, 4) - mu)) < 1e-13)
    r = O.r1d(V5, u, t)
    check("moment identity", max(abs(np.dot(np.array(V5, float) ** n, r) - mu[n]) for n in range(5)) < 1e-13)
    # collision: conservation and fixed point (2D)
    lat = O.Lattice(2, V5, 1.3, 9, 7, theta0=1.0)
    rng = np.random.default_rng(0)
    f0 = O.feq(2, V5, 1.02, 0.05, -0.03, 0.98) * (1 + 0.1 * rng.uniform(-1, 1, 25))
    g0 = lat.collide_node(f0)
    vel = lat.velocities().astype(float)
    sums = lambda f: np.array([f.sum(), (vel[:, 0] * f).sum(), (vel[:, 1] * f).sum(),
                               ((vel ** 2).sum(1) * f).sum()])
    check("collision conservation", np.max(np.abs(sums(g0) - sums(f0))) < 1e-13)
    fe = O.feq(2, V5, 1.1, 0.07, -0.04, 0.9)
    check("fixed point", np.max(np.abs(lat.collide_node(fe) - fe)) < 1e-14)
    rr, a, b, th = lat.node_moments(fe)
    check("node moments", abs(rr - 1.1) + abs(a - 0.07) + abs(b + 0.04) + abs(th - 0.9) < 1e-13)
    # pure streaming moves populations by their velocity
    lat0 = O.Lattice(2, V5, 0.0, 9, 7, theta0=1.0)
    f = rng.uniform(0.5, 1.5, lat0.shape)
    g = lat0.step(f)
    ok = all(np.array_equal(g[p], np.roll(np.roll(f[p], vel[p, 0].astype(int), 1), vel[p, 1].astype(int), 0))
             for p in range(25))
    check("pure stream", ok)
    # fixed ends feed the correct ghost states
    l1 = O.Lattice(1, V5, 0.0, 12, bc="fixed", theta0=0.5, left_state=(1.2, 0.0, 0.5),
                   right_state=(0.9, 0.0, 0.45))
    f1 = rng.uniform(0.5, 1.5, l1.shape)
    g1 = l1.step(f1)
    gl = O.feq(1, V5, 1.2, 0.0, 0.0, 0.5)
    check("fixed ends", abs(g1[1, 0, 0] - gl[1]) < 1e-15 and abs(g1[3, 0, 2] - gl[3]) < 1e-15)
    # hydrodynamics: shear-wave decay rate on a non-square grid
    L = 32
    lat2 = O.Lattice(2, V5, 1.3, 5, L, theta0=1.0)
    fw = lat2.init(*I.shear_wave_fields(5, 1.0, amp=1e-3, ny=L))
    k = 2 * np.pi / L
    amps = []
    for _ in range(2):
        fw = lat2.run(fw, 40)
        _, ux, _, _ = lat2.moments(fw)
        amps.append(np.sum(ux[:, 0] * np.sin(k * np.arange(L))) * 2 / L)
    nu = (1 / 1.3 - 0.5)
    ok = amps[0] > 0 and amps[1] > 0 and abs(-math.log(amps[1] / amps[0]) / (k * k * 40) / nu - 1) < 0.02
    check("shear decay", ok)
    # global sums against the fields of the node moments (reading R3)
    fr = rng.uniform(0.2, 1.8, lat.shape) * (1.0 + 0.5 * rng.uniform(0, 1, (lat.q, 1, 1)))
    rho, ux, uy, th = lat.moments(fr)
    ref = np.array([rho.sum(), (rho * ux).sum(), (rho * uy).sum(), (rho * (ux * ux + uy * uy + 2 * th)).sum()])
    check("conserved sums", np.max(np.abs(lat.conserved(fr) - ref)) <= 1e-12 * ref[0])
    return fails


def test_battery_passes_on_oracle():
    assert _battery() == []


@pytest.mark.parametrize("name,orig,repl", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_rejected(name, orig, repl):
    src = O.source_text()
    assert src.count(orig) == 1, name
    with tempfile.TemporaryDirectory() as d:
        path = O.compile_variant(src.replace(orig, repl), os.path.join(d, "mutant.so"))
        with O.using_library(path):
            try:
                fails = _battery()
            except Exception:  # a crash in numpy/ctypes on garbage also counts as rejection
                fails = ["exception"]
    assert fails, "mutant '%s' passed every pin" % name
