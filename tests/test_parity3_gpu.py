"""GPU parity of three-dimensional lattices (D3Q125, D3Q27) against the 3D oracle.

The CUDA path runs through the C ABI (plbm_init3 / plbm_step / plbm_moments3 /
plbm_get_populations / plbm_conserved3) on the same seeded host fields as the
FP64 oracle (oracle.Lattice3).  Grids are ragged (nx not a multiple of the
128-thread block, odd ny and nz) and span several blocks.
"""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

V5 = (0, 1, -1, 3, -3)
TOL64 = 1e-12


def fields3(nx, ny, nz, seed, amp_u=0.03, amp_r=0.01, theta0=1.0):
    """Smooth periodic seeded fields [nz][ny][nx]."""
    rng = np.random.default_rng(seed)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")

    def wave():
        kx, ky, kz = rng.integers(1, 3, 3)
        ph = rng.uniform(0, 2 * np.pi)
        return np.cos(2 * np.pi * (kx * x / nx + ky * y / ny + kz * z / nz) + ph)

    rho = 1.0 + amp_r * wave()
    ux, uy, uz = (amp_u * wave() for _ in range(3))
    th = theta0 * (1.0 + amp_r * wave())
    return tuple(np.ascontiguousarray(a) for a in (rho, ux, uy, uz, th))


def run_pair(v, omega, shape, steps, prec, theta0=1.0, isothermal=False, seed=3, amp_u=0.03):
    from paper_1402_5487_gb300 import plbm
    nx, ny, nz = shape
    f = fields3(nx, ny, nz, seed, amp_u=amp_u, theta0=theta0)
    lat = O.Lattice3(v, omega, nx, ny, nz, theta0=theta0, isothermal=isothermal)
    fo = lat.run(lat.init(*f), steps)
    s = plbm.Solver(3, v, omega, nx, ny, nz=nz, theta0=theta0, prec=prec, isothermal=isothermal)
    s.init(f[0], f[1], f[2], None if isothermal else f[4], uz=f[3])
    s.step(steps)
    out = s.moments(), s.get_populations(), s.conserved()
    s.close()
    return lat, fo, out, f


@pytest.mark.parametrize("shape", [(130, 7, 5), (16, 9, 11)])
def test_d3q125_f64_matches_oracle(shape):
    lat, fo, (mg, fg, cg), _ = run_pair(V5, 1.3, shape, 30, "f64")
    assert O.rel_err(fg, fo) <= TOL64
    mo = lat.moments(fo)
    for a, b in zip(mg, mo):
        assert np.max(np.abs(a - b)) <= TOL64 * max(np.max(np.abs(b)), 0.03)
    assert np.max(np.abs(cg - lat.conserved(fo)) / np.maximum(1.0, np.abs(lat.conserved(fo)))) <= TOL64


def test_d3q27_isothermal_f64_matches_oracle():
    lat, fo, (mg, fg, cg), _ = run_pair((0, 1, -1), 1.2, (20, 6, 7), 40, "f64", theta0=1.0 / 3.0,
                                        isothermal=True)
    assert O.rel_err(fg, fo) <= TOL64


# Odd nz: one node per thread.  Even nz with 16-bit storage: the z-paired layout
# and the two-nodes-per-thread kernel (nz = 6 puts every pair row within
# max|v| = 3 of the wrap, so each pull of z crosses it in one lane or the other).
@pytest.mark.parametrize("prec,tol,shape", [("f32", 2e-6, (130, 7, 5)), ("f16dev", 2e-3, (130, 7, 5)),
                                            ("bf16dev", 2e-2, (130, 7, 5)), ("f16dev", 2e-3, (130, 7, 6)),
                                            ("bf16dev", 2e-2, (130, 7, 6)), ("f16dev", 2e-3, (20, 5, 14))])
def test_d3q125_reduced_storage_matches_oracle(prec, tol, shape):
    lat, fo, (mg, fg, cg), f = run_pair(V5, 1.3, shape, 30, prec)
    mo = lat.moments(fo)
    u0 = np.max(np.sqrt(f[1] ** 2 + f[2] ** 2 + f[3] ** 2))
    du = np.sqrt((mg[1] - mo[1]) ** 2 + (mg[2] - mo[2]) ** 2 + (mg[3] - mo[3]) ** 2)
    assert np.max(du) <= tol * u0
    assert O.rel_err(mg[0], mo[0]) <= tol * 0.1 and O.rel_err(mg[4], mo[4]) <= tol * 0.1
    assert np.max(np.abs(fg - fo)) <= tol * 0.1 * np.max(np.abs(fo))


def kh3(nx, ny, nz):
    from paper_1402_5487_gb300 import inputs as I
    return I.kh3_fields(nx, ny, nz)


def _f32_run_1000(fields, shape):
    from paper_1402_5487_gb300 import plbm
    nx, ny, nz = shape
    rho, ux, uy, uz, th = fields
    lat = O.Lattice3(V5, 1.3, nx, ny, nz)
    mo = lat.moments(lat.run(lat.init(rho, ux, uy, uz, th), 1000))
    s = plbm.Solver(3, V5, 1.3, nx, ny, nz=nz, prec="f32")
    s.init(rho, ux, uy, th, uz=uz)
    s.step(1000)
    mg = s.moments()
    s.close()
    den = np.max(np.sqrt(mo[1] ** 2 + mo[2] ** 2 + mo[3] ** 2))
    du = np.sqrt((mg[1] - mo[1]) ** 2 + (mg[2] - mo[2]) ** 2 + (mg[3] - mo[3]) ** 2)
    return np.max(du) / den, O.rel_err(mg[0], mo[0]), O.rel_err(mg[4], mo[4]), den


def test_d3q125_f32_1000_steps_shear_layer_within_1e5():
    # The FP32 bar of the parity contract (relative error <= 1e-5 after 1000
    # steps) on the 3D double shear layer.  The box is long across the layers
    # (nz = 256, so nu k^2 t ~ 0.16 and the flow persists for 1000 steps) and
    # short in x and y to keep the oracle fast.
    eu, er, et, den = _f32_run_1000(kh3(8, 4, 256), (8, 4, 256))
    assert den > 0.05
    assert eu <= 1e-5 and er <= 1e-5 and et <= 1e-5, (eu, er, et)


def test_d3q125_f32_1000_steps_uniform_flow_bound():
    # Worst case for FP32 storage: a uniform flow (which viscosity cannot damp)
    # carrying small perturbations; every node holds nearly the same values, so
    # the rounding of the stored deviations is the same everywhere and the mean
    # velocity drifts by ~1e-9 per step.  A regression bound, not the contract.
    rho, ux, uy, uz, th = fields3(32, 16, 12, 21, amp_u=0.02)
    eu, er, et, den = _f32_run_1000((rho, ux + 0.04, uy - 0.03, uz + 0.02, th), (32, 16, 12))
    assert den > 0.04
    assert eu <= 5e-5 and er <= 1e-5 and et <= 1e-5, (eu, er, et)


@pytest.mark.parametrize("prec,nz", [("f64", 5), ("f32", 5), ("f16dev", 6), ("bf16dev", 6), ("f16dev", 10)])
def test_d3q125_pure_streaming_is_exact(prec, nz):
    from paper_1402_5487_gb300 import plbm
    nx, ny = 131, 6
    lat = O.Lattice3(V5, 0.0, nx, ny, nz)
    f0 = lat.init(*fields3(nx, ny, nz, 9))
    s = plbm.Solver(3, V5, 0.0, nx, ny, nz=nz, prec=prec, skip_admissibility=True)
    s.set_populations(f0)
    start = s.get_populations()        # the stored (rounded) state
    s.step(1)
    g = s.get_populations()
    s.close()
    for p, (cx, cy, cz) in enumerate(lat.velocities()):
        expect = np.roll(np.roll(np.roll(start[p], cz, axis=0), cy, axis=1), cx, axis=2)
        assert np.array_equal(g[p], expect), p


def test_d3q125_conserves_to_rounding():
    from paper_1402_5487_gb300 import plbm
    nx, ny, nz = 40, 12, 9
    f = fields3(nx, ny, nz, 4)
    s = plbm.Solver(3, V5, 1.3, nx, ny, nz=nz, prec="f32")
    s.init(f[0], f[1], f[2], f[4], uz=f[3])
    c0 = s.conserved()
    s.step(200)
    c1 = s.conserved()
    s.close()
    scale = np.array([c0[0], c0[0], c0[0], c0[0], c0[4]])
    assert np.max(np.abs(c1 - c0) / scale) < 2e-6


@pytest.mark.parametrize("prec,nz", [("f16dev", 6), ("bf16dev", 8), ("f32", 6)])
def test_d3q125_checkpoint_resume_is_bit_identical(prec, nz):
    # get/set_populations on the 3D layouts (z-paired for 16-bit storage and even nz)
    from paper_1402_5487_gb300 import plbm
    nx, ny = 40, 6
    f = fields3(nx, ny, nz, 12)
    a = plbm.Solver(3, V5, 1.3, nx, ny, nz=nz, prec=prec)
    a.init(f[0], f[1], f[2], f[4], uz=f[3])
    a.step(7)
    f7 = a.get_populations()
    a.step(9)
    ref = a.get_populations()
    b = plbm.Solver(3, V5, 1.3, nx, ny, nz=nz, prec=prec)
    b.set_populations(f7, step=7)
    b.step(9)
    assert np.array_equal(b.get_populations(), ref)
    a.close()
    b.close()


@pytest.mark.parametrize("prec,nz", [("f32", 5), ("f16dev", 6), ("bf16dev", 5)])
def test_d3q125_diagnostics_equal_fp64_sums_of_the_stored_state(prec, nz):
    # The 16/32-bit 3D reduction sums in float-float on the FP32 pipe; its record must
    # equal FP64 sums (numpy) of the stored populations, and its minima the FP64
    # minima of the nodes' rho and theta.
    from paper_1402_5487_gb300 import plbm
    nx, ny = 40, 6
    f = fields3(nx, ny, nz, 13)
    s = plbm.Solver(3, V5, 1.3, nx, ny, nz=nz, prec=prec)
    s.init(f[0], f[1], f[2], f[4], uz=f[3])
    s.step(9)
    pops = s.get_populations()
    lat = O.Lattice3(V5, 1.3, nx, ny, nz)
    vel = lat.velocities().astype(np.float64)
    flat = pops.reshape(pops.shape[0], -1)
    mass = flat.sum(axis=0)
    j = vel.T @ flat
    e = (vel ** 2).sum(axis=1) @ flat
    ref = np.array([mass.sum(), j[0].sum(), j[1].sum(), j[2].sum(), e.sum()])   # conserved3 order
    got = s.conserved()
    assert np.max(np.abs(got - ref)) <= 1e-12 * abs(ref[0]), (got, ref)
    u = j / mass
    th = (e / mass - (u ** 2).sum(axis=0)) / 3.0
    d = s.diagnostics()
    assert abs(d["rho_min"] - mass.min()) <= 1e-13 and abs(d["theta_min"] - th.min()) <= 1e-12
    s.close()


@pytest.mark.parametrize("prec,tol", [("f32", 2e-6), ("f16dev", 2e-3), ("bf16dev", 2e-2)])
def test_d3q125_bench_size_sampled_nodes(prec, tol):
    # The bench's 3D workload (256^3 double shear layer; FP32 on the split kernel,
    # 16-bit storage on the z-paired one): after k steps a node depends only on
    # nodes within 3k, so the oracle advances a (6k+1)^3 periodic window around
    # each sampled node and its centre must match the GPU.
    from paper_1402_5487_gb300 import inputs as I, plbm
    n, k, half = 256, 2, 6
    f = I.kh3_fields(n, n, n)
    s = plbm.Solver(3, V5, 1.3, n, n, nz=n, theta0=1.0, prec=prec)
    s.init(f[0], f[1], f[2], f[4], uz=f[3])
    s.step(k)
    mg = s.moments()                       # rho, ux, uy, uz, theta, each [nz][ny][nx]
    s.close()
    rng = np.random.default_rng(31)
    pts = [(0, 0, 0), (n - 1, n - 1, n - 1), (5, 250, 128)] + [tuple(int(a) for a in rng.integers(0, n, 3))
                                                                for _ in range(5)]
    w = 2 * half + 1
    for cx, cy, cz in pts:
        zs, ys, xs = (np.arange(c - half, c + half + 1) % n for c in (cz, cy, cx))
        patch = [np.ascontiguousarray(a[np.ix_(zs, ys, xs)]) for a in f]
        lat = O.Lattice3(V5, 1.3, w, w, w, theta0=1.0)
        mo = lat.moments(lat.run(lat.init(*patch), k))
        for g, o, scale in zip(mg, mo, (1.0, 0.1, 0.1, 0.1, 1.0)):
            assert abs(g[cz, cy, cx] - o[half, half, half]) <= tol * scale, (prec, cx, cy, cz)
