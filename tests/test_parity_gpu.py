"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (max|a-b|/max|b| per field, vector norm for u, and the same over
all populations):
  FP64 storage  <= 1e-12 relative,
  FP32 storage  <= 1e-5 relative over 1000 steps.
Integer-like work (pure streaming with omega = 0, checkpoint round trips)
is compared bit for bit.
"""
import math

import numpy as np
import pytest

import oracle as O
from oracle import riemann as R
from paper_1402_5487_gb300 import build, inputs as I, plbm

from parity_util import field_errors, gpu_run, oracle_run, patch_fields, rel

pytestmark = pytest.mark.gpu

V5 = I.SET_013
TOL64 = 1e-12
TOL32 = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    plbm.lib()


def smooth_fields(nx, ny, seed, amp_u=0.05, amp_r=0.02, theta0=1.0):
    rng = np.random.default_rng(seed)
    x = np.arange(nx)[None, :] * 2 * np.pi / nx
    y = np.arange(ny)[:, None] * 2 * np.pi / ny
    ph = rng.uniform(0, 2 * np.pi, 4)
    rho = 1 + amp_r * np.sin(x + ph[0]) * np.cos(y + ph[1]) + 0.001 * rng.uniform(-1, 1, (ny, nx))
    ux = amp_u * np.sin(y + ph[2]) + 0.002 * rng.uniform(-1, 1, (ny, nx))
    uy = amp_u * np.cos(x + ph[3]) + 0.002 * rng.uniform(-1, 1, (ny, nx))
    th = theta0 * (1 + amp_r * np.cos(x + y + ph[0])) + 0 * rho
    return (np.ascontiguousarray(rho), np.ascontiguousarray(ux), np.ascontiguousarray(uy),
            np.ascontiguousarray(th))


@pytest.mark.parametrize("nx,ny", [(33, 17), (7, 5), (1, 1), (130, 3), (256, 2)])
def test_pure_stream_bit_exact(nx, ny):
    # omega = 0 leaves only the pull: identical FP64 inputs must give identical outputs.
    lat = O.Lattice(2, V5, 0.0, nx, ny, theta0=1.0)
    f0 = lat.init(*smooth_fields(nx, ny, 1))
    s = plbm.Solver(2, V5, 0.0, nx, ny, theta0=1.0, prec="f64")
    s.set_populations(f0)
    s.step(3)
    assert np.array_equal(s.get_populations(), lat.run(f0, 3))
    s.close()


@pytest.mark.parametrize("nx,ny", [(33, 17), (130, 3)])
def test_pure_stream_fixed_ends_bit_exact(nx, ny):
    left, right = (1.2, 0.05, 0.9), (0.8, -0.02, 1.1)
    lat = O.Lattice(2, V5, 0.0, nx, ny, bc="fixed", theta0=1.0, left_state=left, right_state=right)
    f0 = lat.init(*smooth_fields(nx, ny, 5))
    s = plbm.Solver(2, V5, 0.0, nx, ny, theta0=1.0, prec="f64", bc="fixed", left_state=left,
                    right_state=right)
    s.set_populations(f0)
    s.step(4)
    got, ref = s.get_populations(), lat.run(f0, 4)
    # ghost populations come from the library's own FP64 f^eq: equal to rounding
    assert np.max(np.abs(got - ref)) <= 1e-15
    s.close()


@pytest.mark.parametrize("nx,ny", [(33, 17), (7, 5), (1, 1), (200, 9), (34, 18), (1, 2)])
def test_parity_d2q25_f64(nx, ny):
    fields = smooth_fields(nx, ny, 2)
    (mg, fg, _) = gpu_run(2, V5, 1.3, nx, ny, fields, 100, prec="f64")
    _, fo, mo = oracle_run(2, V5, 1.3, nx, ny, fields, 100)
    assert rel(fg, fo) <= TOL64
    # tiny periodic grids damp u to a small fraction of its start within 100 steps: scale
    # the velocity error by its initial amplitude
    u0 = np.max(np.hypot(fields[1], fields[2]))
    assert np.max(np.hypot(mg[1] - mo[1], mg[2] - mo[2])) <= TOL64 * u0
    assert O.rel_err(mg[0], mo[0]) <= TOL64 and O.rel_err(mg[3], mo[3]) <= TOL64


# Even ny takes the row-paired two-nodes-per-thread kernel, odd ny the one-node kernel.
@pytest.mark.parametrize("nx,ny", [(33, 17), (7, 5), (1, 1), (130, 3), (34, 18), (8, 6), (1, 2),
                                   (130, 4), (257, 10)])
@pytest.mark.parametrize("prec,tol", [("f32", 2e-6), ("f16dev", 2e-3), ("bf16dev", 2e-2)])
def test_parity_d2q25_reduced_storage_small_grids(nx, ny, prec, tol):
    fields = smooth_fields(nx, ny, 7)
    steps = 50
    (mg, fg, _) = gpu_run(2, V5, 1.3, nx, ny, fields, steps, prec=prec)
    _, fo, mo = oracle_run(2, V5, 1.3, nx, ny, fields, steps)
    u0 = np.max(np.hypot(fields[1], fields[2]))
    assert np.max(np.hypot(mg[1] - mo[1], mg[2] - mo[2])) <= tol * u0
    assert O.rel_err(mg[0], mo[0]) <= tol * 0.1 and O.rel_err(mg[3], mo[3]) <= tol * 0.1
    assert np.max(np.abs(fg - fo)) <= tol * 0.1 * np.max(np.abs(fo))


@pytest.mark.parametrize("prec,tol", [("f64", TOL64), ("f32", 2e-6)])
@pytest.mark.parametrize("v,theta0,omega,iso", [((0, 1, -1), 0.25, 1.2, True),
                                                ((0, 1, -1), 1.0 / 3.0, 1.5, True),
                                                ((1, -1, 3, -3), 4.0 / 3.0, 1.1, True),
                                                ((0, 1, -1, 2, -2), 1 / 1.6 ** 2, 1.6, False),
                                                ((0, 2, -2, 3, -3), 1.6, 1.2, False),
                                                ((0, 2, -4), 1.0, 1.0, True),
                                                ((0, 1, -1, 2, -2, 3), 0.8, 1.3, False),
                                                ((0, 1, -1, 2, -2, 3, -3), 1.0, 1.3, False),
                                                ((0, 1, -1, 2, -2, 3, -3, 4), 1.0, 1.3, False)])
def test_parity_other_sets(v, theta0, omega, iso, prec, tol):
    nx, ny = 70, 19
    fields = smooth_fields(nx, ny, 3, amp_u=0.03, amp_r=0.01, theta0=theta0)
    (mg, fg, _) = gpu_run(2, v, omega, nx, ny, fields, 60, prec=prec, theta0=theta0, isothermal=iso)
    _, fo, mo = oracle_run(2, v, omega, nx, ny, fields, 60, theta0=theta0, isothermal=iso)
    assert rel(fg, fo) <= tol
    assert O.rel_err(mg[0], mo[0]) <= tol and O.rel_err(mg[3], mo[3]) <= tol


@pytest.mark.parametrize("prec,tol", [("f64", TOL64), ("f32", TOL32)])
def test_parity_d1q5_shock_tube(prec, tol):
    left, right = (1.1, 0.0, 0.5), (1.0, 0.0, 0.5)
    fields = I.shock_tube_fields(1000, left, right)
    (mg, fg, _) = gpu_run(1, V5, 1.5, 1000, 1, fields, 500, prec=prec, theta0=0.5, bc="fixed",
                          left=left, right=right)
    _, fo, mo = oracle_run(1, V5, 1.5, 1000, 1, fields, 500, theta0=0.5, bc="fixed", left=left,
                           right=right)
    errs = field_errors(mg, mo)
    assert max(errs.values()) <= tol, errs
    if prec == "f64":
        assert rel(fg, fo) <= tol


def test_shock_tube_gpu_vs_exact_riemann():
    left, right = (1.1, 0.0, 0.5), (1.0, 0.0, 0.5)
    fields = I.shock_tube_fields(1000, left, right)
    (mg, _, _) = gpu_run(1, V5, 1.5, 1000, 1, fields, 361, prec="f64", theta0=0.5, bc="fixed",
                         left=left, right=right)
    rho, ux, _, th = (a[0] for a in mg)
    x = np.arange(1000) + 0.5
    re, ue, pe = R.sample(R.State(1.1, 0.0, 0.55), R.State(1.0, 0.0, 0.5), 3.0, (x - 500) / 361)
    assert np.mean(np.abs(rho - re)) / np.mean(re) < 0.002
    assert np.mean(np.abs(ux - ue)) / np.max(np.abs(ue)) < 0.02
    assert np.mean(np.abs(th - pe / re)) / np.mean(pe / re) < 0.002


@pytest.mark.parametrize("L", [128])
def test_parity_kh_1000_steps(L):
    fields = I.kh_fields(L)
    _, fo, mo = oracle_run(2, V5, 1.3, L, L, fields, 1000)
    (m64, f64, _) = gpu_run(2, V5, 1.3, L, L, fields, 1000, prec="f64")
    (m32, f32, _) = gpu_run(2, V5, 1.3, L, L, fields, 1000, prec="f32")
    e64 = field_errors(m64, mo)
    e32 = field_errors(m32, mo)
    assert max(e64.values()) <= TOL64 and rel(f64, fo) <= TOL64, e64
    assert max(e32.values()) <= TOL32 and rel(f32, fo) <= TOL32, e32


@pytest.mark.slow
def test_parity_kh_512_config_1000_steps():
    # Kelvin-Helmholtz double shear layer, 512^2, D2Q25 {0,+-1,+-3}^2, theta0 = 1, omega = 1.3.
    L = 512
    fields = I.kh_fields(L)
    _, fo, mo = oracle_run(2, V5, 1.3, L, L, fields, 1000)
    (m64, f64, _) = gpu_run(2, V5, 1.3, L, L, fields, 1000, prec="f64")
    (m32, f32, _) = gpu_run(2, V5, 1.3, L, L, fields, 1000, prec="f32")
    e64 = field_errors(m64, mo)
    e32 = field_errors(m32, mo)
    assert max(e64.values()) <= TOL64 and rel(f64, fo) <= TOL64, e64
    assert max(e32.values()) <= TOL32 and rel(f32, fo) <= TOL32, e32


@pytest.mark.parametrize("L,prec,tol", [(2048, "f32", 1e-6), (2047, "f32", 1e-6), (2048, "f16dev", 2e-3),
                                         (2048, "bf16dev", 2e-2)])
def test_fullsize_2048_sampled_nodes(L, prec, tol):
    # Bench workloads (2048^2 KH in FP32 and 16-bit storage on row pairs; 2047^2, the
    # plain layout of odd sides): after k steps a node depends only on nodes within 3k
    # in each direction, so the oracle advances a (6k+1)^2 periodic window around each
    # sampled node and its centre must match the GPU.
    k, half = 4, 12
    fields = I.kh_fields(L)
    s = plbm.Solver(2, V5, 1.3, L, L, theta0=1.0, prec=prec)
    s.init(*fields)
    s.step(k)
    mg = s.moments()
    rng = np.random.default_rng(11)
    pts = [(0, 0), (L - 1, L - 1), (L // 2, L // 4), (3, L - 2)] + [
        tuple(int(a) for a in rng.integers(0, L, 2)) for _ in range(28)]
    errs = []
    for cx, cy in pts:
        pf = patch_fields(fields, cx, cy, half, L, L)
        lat, f, mo = oracle_run(2, V5, 1.3, 2 * half + 1, 2 * half + 1, pf, k)
        for gi, oi in zip(mg, mo):
            errs.append(abs(gi[cy, cx] - oi[half, half]) / max(1e-30, np.max(np.abs(fields[0]))))
    rho_g, ux_g, uy_g, _ = mg
    assert max(errs[0::4]) < tol      # rho
    assert max(errs[3::4]) < tol      # theta
    assert max(max(errs[1::4]), max(errs[2::4])) < tol  # velocity components (scale ~0.1)
    d = s.diagnostics()
    assert abs(d["mass"] - L * L) / (L * L) < max(tol, 1e-6)
    s.close()


def test_conservation_periodic_f64():
    L = 64
    fields = I.kh_fields(L)
    s = plbm.Solver(2, V5, 1.3, L, L, theta0=1.0, prec="f64")
    s.init(*fields)
    c0 = s.conserved()
    s.step(10000)
    c1 = s.conserved()
    assert np.max(np.abs(c1 - c0)) <= 1e-12 * np.max(np.abs(c0))
    lat = O.Lattice(2, V5, 1.3, L, L, theta0=1.0)
    f = lat.init(*fields)
    assert np.max(np.abs(c0 - lat.conserved(f))) <= 1e-13 * np.max(np.abs(c0))
    s.close()


def test_diagnostics_match_oracle():
    L = 48
    fields = I.kh_fields(L, seed=5)
    (mg, fg, s) = gpu_run(2, V5, 1.3, L, L, fields, 37, prec="f64")
    lat, fo, mo = oracle_run(2, V5, 1.3, L, L, fields, 37)
    d = s.diagnostics()
    co = lat.conserved(fo)
    for a, b in zip((d["mass"], d["jx"], d["jy"], d["energy"]), co):
        assert abs(a - b) <= 1e-12 * max(1.0, abs(co[0]))
    assert abs(d["rho_min"] - mo[0].min()) < 1e-13
    assert abs(d["theta_min"] - mo[3].min()) < 1e-13
    assert d["status"] == 0 and d["steps"] == 37
    s.close()


@pytest.mark.parametrize("prec", ["f64", "f32", "f16dev", "bf16dev"])
def test_checkpoint_resume_is_bit_identical(prec):
    L = 40
    fields = I.kh_fields(L, seed=3)
    a = plbm.Solver(2, V5, 1.3, L, L, theta0=1.0, prec=prec)
    a.init(*fields)
    a.step(20)
    f20 = a.get_populations()
    a.step(20)
    ref = a.get_populations()
    b = plbm.Solver(2, V5, 1.3, L, L, theta0=1.0, prec=prec)
    b.set_populations(f20, step=20)
    b.step(20)
    assert np.array_equal(b.get_populations(), ref)
    assert b.diagnostics()["steps"] == 40
    a.close()
    b.close()


def test_device_pointers_and_streams():
    import torch
    L = 64
    fields = I.kh_fields(L, seed=4)
    st = torch.cuda.Stream()
    s = plbm.Solver(2, V5, 1.3, L, L, theta0=1.0, prec="f32", stream=st)
    dev = [torch.from_numpy(a).to("cuda") for a in fields]
    torch.cuda.synchronize()
    s.init(*dev)
    s.step(10)
    md = s.moments(on_device=True)
    st.synchronize()
    mh = s.moments()
    for a, b in zip(md, mh):
        assert np.array_equal(a.cpu().numpy(), b)
    (mg, _, _) = gpu_run(2, V5, 1.3, L, L, fields, 10, prec="f32")
    for a, b in zip(mg, mh):
        assert np.array_equal(a, b)
    s.close()


@pytest.mark.parametrize("prec,tol", [("f16dev", 2e-2), ("bf16dev", 1e-1)])
def test_reduced_precision_error_is_bounded(prec, tol):
    L = 128
    fields = I.kh_fields(L)
    _, _, mo = oracle_run(2, V5, 1.3, L, L, fields, 1000)
    (mg, _, s) = gpu_run(2, V5, 1.3, L, L, fields, 1000, prec=prec)
    errs = field_errors(mg, mo)
    assert errs["u"] <= tol and errs["rho"] <= tol * 0.1 and errs["theta"] <= tol * 0.1, errs
    assert s.check() == plbm.PLBM_OK


def test_literal_shock_tube_reports_divergence():
    # rho 1 / 0.125, theta 0.5 / 0.4 on {0,+-1,+-3}: leaves the positivity region (theta <= 0).
    left, right = (1.0, 0.0, 0.5), (0.125, 0.0, 0.4)
    s = plbm.Solver(1, V5, 1.5, 1000, 1, theta0=0.5, prec="f64", bc="fixed", left_state=left,
                    right_state=right, check_every=5)
    s.init(*I.shock_tube_fields(1000, left, right))
    st = s.step_status(500)
    assert st == plbm.PLBM_E_DIVERGED
    assert "diverged" in plbm.last_error(s.h)
    # sticky: further steps are refused, diagnostics still readable
    assert s.step_status(1) == plbm.PLBM_E_DIVERGED
    assert s.diagnostics()["status"] != 0
    s.close()


def test_literal_kh_omega_reports_divergence():
    L = 64
    s = plbm.Solver(2, V5, 1.8, L, L, theta0=1.0, prec="f32", check_every=50)
    s.init(*I.kh_fields(L))
    assert s.step_status(3000) == plbm.PLBM_E_DIVERGED
    s.close()


def test_stable_kh_stays_healthy():
    L = 64
    s = plbm.Solver(2, V5, 1.3, L, L, theta0=1.0, prec="f32", check_every=100)
    s.init(*I.kh_fields(L))
    assert s.step_status(3000) == plbm.PLBM_OK
    rho, ux, uy, th = s.moments()
    assert abs(rho - 1).max() < 0.01 and abs(th - 1).max() < 0.01
    assert np.hypot(ux, uy).max() < 0.12
    s.close()


# --------------------------------------------------------------------------
# The paper's own parameters (Sec. 4): {0, +-1, +-2} = {0, +-a, +-2a} sqrt(theta0),
# theta0 = 1 / a^2, omega = 1.9.
# --------------------------------------------------------------------------
SET_012 = (0, 1, -1, 2, -2)


def _exact_rounded_coefficients(v):
    """V^{-1} in exact rational arithmetic, each entry rounded once to FP64."""
    from fractions import Fraction
    q = len(v)
    A = [[Fraction(vk) ** n for vk in v] + [Fraction(int(n == k)) for k in range(q)] for n in range(q)]
    for c in range(q):
        p = next(r for r in range(c, q) if A[r][c] != 0)
        A[c], A[p] = A[p], A[c]
        d = A[c][c]
        A[c] = [x / d for x in A[c]]
        for r in range(q):
            if r != c and A[r][c] != 0:
                m = A[r][c]
                A[r] = [a_ - m * b_ for a_, b_ in zip(A[r], A[c])]
    return np.array([[float(A[i][q + n]) for n in range(q)] for i in range(q)])


def coefficient_sensitivity(dim, v, omega, nx, ny, fields, steps, **kw):
    """Oracle fields after `steps` and the oracle's own drift against a copy of
    itself whose c_ij are the exact rationals rounded once (a few ulps of each
    row's scale from its Gauss-Jordan values): the part of an FP64 difference
    that the last bits of the coefficients explain."""
    lat = O.Lattice(dim, v, omega, nx, ny, **kw)
    alt = O.Lattice(dim, v, omega, nx, ny, **kw)
    cex = _exact_rounded_coefficients(v)
    row = np.max(np.abs(cex), axis=1, keepdims=True)
    assert np.max(np.abs(cex - lat.C) / (np.finfo(float).eps * row)) <= 8.0
    for i, c in enumerate(cex.ravel()):
        alt.struct.C[i] = c
    m0 = lat.moments(lat.run(lat.init(*fields), steps))
    m1 = alt.moments(alt.run(alt.init(*fields), steps))
    return m0, field_errors(m1, m0)


def test_paper_shear_layer_f64_within_the_coefficient_rounding_sensitivity():
    # At omega = 1.9 the BGK step hardly damps the momentum error that a one-ulp
    # difference in the c_ij injects every step, so two correct FP64
    # implementations whose coefficients differ in the last bit drift apart
    # linearly (the library builds c_ij by Lagrange expansion, the oracle by
    # Gauss-Jordan elimination).  The bound is the oracle's own drift against a
    # copy of itself with correctly rounded coefficients (at most one ulp away).
    fields, theta0 = I.paper_kh_fields()
    steps = 1000
    lat = O.Lattice(2, SET_012, 1.9, 128, 128, theta0=theta0)
    alt = O.Lattice(2, SET_012, 1.9, 128, 128, theta0=theta0)
    cex = _exact_rounded_coefficients(SET_012)
    assert np.max(np.abs(cex - lat.C) / np.spacing(np.abs(cex) + 1e-300)) <= 1.0
    for i, c in enumerate(cex.ravel()):
        alt.struct.C[i] = c
    m0 = lat.moments(lat.run(lat.init(*fields), steps))
    m1 = alt.moments(alt.run(alt.init(*fields), steps))
    (mg, _, _) = gpu_run(2, SET_012, 1.9, 128, 128, fields, steps, prec="f64", theta0=theta0)
    sens = field_errors(m1, m0)
    errs = field_errors(mg, m0)
    assert errs["rho"] <= TOL64 and errs["theta"] <= TOL64, errs
    assert errs["u"] <= max(TOL64, 2.0 * sens["u"]), (errs, sens)


@pytest.mark.parametrize("steps,tol", [(100, TOL32), (1000, 1e-4)])
def test_paper_shear_layer_f32_matches_oracle(steps, tol):
    # The FP32 bar (1e-5) at 100 steps.  With the paper's slow flow (u0 = 0.043)
    # and omega = 1.9, which hardly damps the momentum error of the FP32 storage
    # rounding (a few 1e-9 per population per step), the relative u error walks to
    # 1.05e-5 at 200 steps and 4.4e-5 at 1000 steps (a regression bound there).
    fields, theta0 = I.paper_kh_fields()
    (mg, fg, _) = gpu_run(2, SET_012, 1.9, 128, 128, fields, steps, prec="f32", theta0=theta0)
    _, fo, mo = oracle_run(2, SET_012, 1.9, 128, 128, fields, steps, theta0=theta0)
    errs = field_errors(mg, mo)
    assert max(errs.values()) <= tol, errs


def test_paper_shear_layer_stays_stable_to_the_last_printed_step_in_f64():
    # The paper shows the 25-velocity shear layer up to step 3695 at omega = 1.9.
    from paper_1402_5487_gb300 import plbm
    fields, theta0 = I.paper_kh_fields()
    s = plbm.Solver(2, SET_012, 1.9, 128, 128, theta0=theta0, prec="f64")
    s.init(*fields)
    s.step(3695)
    assert s.check() == plbm.PLBM_OK
    rho, ux, uy, th = s.moments()
    s.close()
    assert 0.995 < rho.min() and rho.max() < 1.005
    assert 0.995 < th.min() / theta0 and th.max() / theta0 < 1.005
    assert np.max(np.hypot(ux, uy)) < 0.06


def test_paper_shear_layer_in_f32_follows_f64_then_diverges_and_is_reported():
    # FP32 rounding (~1e-7) seeds the mode that the oracle shows growing from a
    # 1e-7 perturbation of the FP64 initial state (tests/test_oracle_paper_params.py):
    # the FP32 run follows FP64 for 1500 steps, then departs and the status word
    # reports the divergence before the paper's last printed step.
    from paper_1402_5487_gb300 import plbm
    fields, theta0 = I.paper_kh_fields()
    a = plbm.Solver(2, SET_012, 1.9, 128, 128, theta0=theta0, prec="f32")
    b = plbm.Solver(2, SET_012, 1.9, 128, 128, theta0=theta0, prec="f64")
    for s in (a, b):
        s.init(*fields)
        s.step(1500)
    ea = field_errors(a.moments(), b.moments())
    assert max(ea.values()) < 1e-3, ea
    statuses = []
    for _ in range(9):                       # up to step 3750
        a.step(250)
        statuses.append(a.check())
        if statuses[-1] != plbm.PLBM_OK:
            break
    a.close()
    b.close()
    assert statuses[-1] == plbm.PLBM_E_DIVERGED, statuses


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_d1q7_thermal_shock_tube_matches_oracle(prec):
    # The conventional seven-velocity on-lattice thermal set {0, +-1, +-2, +-3}
    # (q1 = 7, n* = 6) through the general-q1 kernels.  FP64: rho, theta within
    # 1e-12 and u within twice the oracle's own sensitivity to the last bit of
    # its c_ij (denominators up to 720 here); FP32 within 1e-5.
    v = (0, 1, -1, 2, -2, 3, -3)
    left, right = (1.1, 0.0, 1.0), (1.0, 0.0, 1.0)
    fields = I.shock_tube_fields(1000, left, right)
    (mg, fg, _) = gpu_run(1, v, 1.5, 1000, 1, fields, 300, prec=prec, theta0=1.0, bc="fixed", left=left,
                          right=right)
    m0, sens = coefficient_sensitivity(1, v, 1.5, 1000, 1, fields, 300, bc="fixed", theta0=1.0,
                                       left_state=left, right_state=right)
    errs = field_errors(mg, m0)
    if prec == "f64":
        assert errs["rho"] <= TOL64 and errs["theta"] <= TOL64, errs
        assert errs["u"] <= max(TOL64, 2.0 * sens["u"]), (errs, sens)
    else:
        assert max(errs.values()) <= TOL32, errs


def test_paper_d1q5_shock_tube_f64_within_the_coefficient_rounding_sensitivity():
    # Same bound as the shear layer: at omega = 1.9 the one-ulp differences of the
    # c_ij between the library and the oracle drift the slow post-shock flow apart.
    theta = 1 / 1.96
    left, right = (1.1, 0.0, theta), (1.0, 0.0, theta)
    fields = I.shock_tube_fields(1000, left, right)
    m0, sens = coefficient_sensitivity(1, SET_012, 1.9, 1000, 1, fields, 346, bc="fixed", theta0=theta,
                                       left_state=left, right_state=right)
    (mg, _, _) = gpu_run(1, SET_012, 1.9, 1000, 1, fields, 346, prec="f64", theta0=theta, bc="fixed",
                         left=left, right=right)
    errs = field_errors(mg, m0)
    assert errs["rho"] <= TOL64 and errs["theta"] <= TOL64, errs
    assert errs["u"] <= max(TOL64, 2.0 * sens["u"]), (errs, sens)


def test_paper_d1q5_shock_tube_f32_matches_oracle():
    # A regression bound: at omega = 1.9 the shock leaves acoustic oscillations of
    # a third of the post-shock velocity that the collision barely damps, and the
    # FP32 rounding of the stored populations walks the slow flow (u ~ 0.02) away
    # from FP64 by ~2.5e-5 in u after 346 steps (the 1e-5 bar holds for the
    # omega = 1.5 shock tube, test_parity_d1q5_shock_tube).
    theta = 1 / 1.96
    left, right = (1.1, 0.0, theta), (1.0, 0.0, theta)
    fields = I.shock_tube_fields(1000, left, right)
    (mg, fg, _) = gpu_run(1, SET_012, 1.9, 1000, 1, fields, 346, prec="f32", theta0=theta, bc="fixed",
                          left=left, right=right)
    _, fo, mo = oracle_run(1, SET_012, 1.9, 1000, 1, fields, 346, theta0=theta, bc="fixed", left=left,
                           right=right)
    errs = field_errors(mg, mo)
    assert errs["u"] <= 5e-5 and errs["rho"] <= 5e-6 and errs["theta"] <= 5e-6, errs


# --------------------------------------------------------------------------
# The three-velocity models of Sec. 4 (isothermal, D2Q9 tensor products):
# LBGK (zeta = 3) and the parametric zeta = 4 model on the paper's shear layer,
# and second-order convergence on the GPU path.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("zeta", [3, 4])
def test_zeta_shear_layer_matches_oracle_and_the_papers_stability_pattern(zeta):
    from paper_1402_5487_gb300 import plbm
    theta0 = 1.0 / zeta
    omega = {3: 1.99880, 4: 1.99862}[zeta]
    fields, _ = I.paper_kh_fields(theta0=theta0)
    early, late = {3: (500, 1800), 4: (577, 2078)}[zeta]
    (mg, fg, s) = gpu_run(2, (0, 1, -1), omega, 128, 128, fields, early, prec="f64", theta0=theta0,
                          isothermal=True)
    _, fo, mo = oracle_run(2, (0, 1, -1), omega, 128, 128, fields, early, theta0=theta0, isothermal=True)
    assert max(field_errors(mg, mo).values()) <= TOL64
    s.step(late - early)
    status = s.check()
    s.close()
    # LBGK is gone before its step 1800; zeta = 4 is still running at 2078
    assert status == (plbm.PLBM_E_DIVERGED if zeta == 3 else plbm.PLBM_OK), status


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("v,theta0,iso,omega", [((0, 1, -1), 0.25, True, 1.2),
                                                ((0, 1, -1, 3, -3), 1.0, False, 1.3)],
                         ids=["zeta4", "d2q25"])
def test_taylor_green_converges_at_second_order_on_gpu(v, theta0, iso, omega, prec):
    from test_oracle_paper_params import taylor_green_errors

    def runner(v, theta0, iso, omega, N, fields, steps):
        (m, _, s) = gpu_run(2, v, omega, N, N, fields, steps, prec=prec, theta0=theta0, isothermal=iso)
        s.close()
        return m

    errs = taylor_green_errors(v, theta0, iso, omega, runner=runner)
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert all(o > 1.8 for o in orders), (errs, orders)


@pytest.mark.parametrize("prec,dim", [("f64", 1), ("f32", 2), ("f16dev", 2)])
def test_graph_replayed_steps_equal_single_launches(prec, dim):
    # Small lattices advance by replays of a captured 32-step graph; the result must
    # equal the same steps launched one call at a time, bit for bit.
    nx, ny = (1000, 1) if dim == 1 else (64, 48)
    fields = I.kh_fields(nx, ny=ny) if dim == 2 else I.shock_tube_fields(nx)
    out = []
    for chunks in ([150], [1] * 150):
        if dim == 1:
            s = plbm.Solver(1, I.SET_013, 1.5, nx, 1, theta0=0.5, prec=prec, bc="fixed",
                            left_state=(1.1, 0.0, 0.5), right_state=(1.0, 0.0, 0.5))
            s.init(fields[0], fields[1], None, fields[3])
        else:
            s = plbm.Solver(2, I.SET_013, 1.3, nx, ny, theta0=1.0, prec=prec)
            s.init(*fields)
        for c in chunks:
            s.step(c)
        out.append(s.get_populations())
        assert s.check() == 0
        s.close()
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("prec", ["f32", "bf16dev", "f64"])
def test_banded_host_transfers_equal_device_pointers(prec):
    # Lattices of 2^18 nodes or more move host fields in eight row bands on a copy
    # stream overlapped with the kernels; the result must equal the device-pointer
    # calls bit for bit (640 x 512 = 327,680 nodes in bands of 64 rows; 520 x 517
    # in uneven bands).
    import torch
    for nx, ny in ((640, 512), (520, 517)):
        fields = I.kh_fields(nx, ny=ny, seed=6)
        st = torch.cuda.Stream()
        a = plbm.Solver(2, V5, 1.3, nx, ny, theta0=1.0, prec=prec, stream=st)
        b = plbm.Solver(2, V5, 1.3, nx, ny, theta0=1.0, prec=prec, stream=st)
        a.init(*fields)                                          # host pointers, banded
        b.init(*[torch.from_numpy(f).to("cuda") for f in fields])  # device pointers
        st.synchronize()
        assert np.array_equal(a.get_populations(), b.get_populations())
        a.step(3)
        b.step(3)
        mh = a.moments()                                         # host pointers, banded
        md = b.moments(on_device=True)
        st.synchronize()
        for x, y in zip(mh, md):
            assert np.array_equal(x, y.cpu().numpy())
        a.close()
        b.close()


@pytest.mark.parametrize("prec,dim", [("f64", 2), ("f32", 2), ("f16dev", 2), ("f64", 1), ("f32", 1)])
def test_fused_step_diagnostics_match_separate_reduction(prec, dim):
    # The last step of plbm_step_diagnostics forms the FP64 sums in the step kernel;
    # they must equal plbm_diagnostics of the same state (FP64: to rounding; 16/32-bit:
    # the fused sums use the kernel's FP32 moments, so to FP32 rounding), and the
    # populations must be those of plain stepping.
    if dim == 2:
        nx, ny = 96, 64
        fields = I.kh_fields(nx, ny=ny, seed=8)
        make = lambda: plbm.Solver(2, V5, 1.3, nx, ny, theta0=1.0, prec=prec)
        init = lambda s: s.init(*fields)
    else:
        nx, ny = 1000, 1
        left, right = (1.1, 0.0, 0.5), (1.0, 0.0, 0.5)
        fields = I.shock_tube_fields(nx, left, right)
        make = lambda: plbm.Solver(1, V5, 1.5, nx, 1, theta0=0.5, prec=prec, bc="fixed", left_state=left,
                                   right_state=right)
        init = lambda s: s.init(fields[0], fields[1], None, fields[3])
    a, b = make(), make()
    init(a)
    init(b)
    da = a.step_diagnostics(37)
    b.step(37)
    db = b.diagnostics()
    assert np.array_equal(a.get_populations(), b.get_populations())
    assert da["steps"] == db["steps"] == 37 and da["status"] == db["status"] == 0
    # 16-bit: the stored state carries the storage rounding of the deviations (~5e-6 each)
    tol = {"f64": 1e-12, "f32": 2e-6, "f16dev": 3e-5}[prec]
    scale = max(abs(db["mass"]), 1.0)
    for k in ("mass", "jx", "jy", "energy"):
        assert abs(da[k] - db[k]) <= tol * max(scale, abs(db["energy"])), (k, da[k], db[k])
    for k in ("rho_min", "theta_min"):
        assert abs(da[k] - db[k]) <= tol * abs(db[k]), (k, da[k], db[k])
    a.close()
    b.close()


# --------------------------------------------------------------------------
# The isothermal three-velocity shock tubes of Sec. 3.2 on the GPU path: the
# 6:1 tube's printed front and post-shock velocity, and the 1.1:1 comparison of
# the zeta = 4 model with LBGK under nu and nu_hat viscosity matching.
# --------------------------------------------------------------------------
def _gpu_tube(prec):
    def tube(v, omega, theta0, left, right, steps):
        fields = I.shock_tube_fields(1000, left, right)
        (m, _, s) = gpu_run(1, v, omega, 1000, 1, fields, steps, prec=prec, theta0=theta0, bc="fixed",
                            left=left, right=right, isothermal=True)
        s.close()
        return m
    return tube


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 2e-6)])
def test_zeta4_vs_lbgk_small_ratio_on_gpu(prec, tol):
    from test_oracle_riemann import zeta4_vs_lbgk_small_ratio
    ref, _, _ = zeta4_vs_lbgk_small_ratio()
    got, _, _ = zeta4_vs_lbgk_small_ratio(tube=_gpu_tube(prec))
    for k in ref:
        for a, b in zip(got[k], ref[k]):
            assert abs(a - b) <= tol, (k, got, ref)
    assert got["nu_hat"][0] < got["nu"][0] / 10


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_zeta4_shock_tube_printed_front_on_gpu(prec):
    from conftest import read_printed_values
    vals = read_printed_values()
    theta0 = 0.25
    omega = 4 * math.sqrt(3) - 6
    steps = int(vals["shock6_iterations_param"])
    left, right = (6.0, 0.0, theta0), (1.0, 0.0, theta0)
    mg = _gpu_tube(prec)((0, 1, -1), omega, theta0, left, right, steps)
    _, _, mo = oracle_run(1, (0, 1, -1), omega, 1000, 1, I.shock_tube_fields(1000, left, right), steps,
                          theta0=theta0, bc="fixed", left=left, right=right, isothermal=True)
    errs = field_errors(mg, mo)
    assert max(errs.values()) <= (TOL64 if prec == "f64" else TOL32), errs
    rho, ux = mg[0][0], mg[1][0] / math.sqrt(theta0)
    assert abs(np.mean(ux[650:750]) - vals["shock6_u_post"]) < 0.005
    plateau = np.mean(rho[650:750])
    half = 0.5 * (plateau + 1.0)
    i = int(np.nonzero(rho > half)[0].max())
    front = (i + 1) + (rho[i] - half) / (rho[i] - rho[i + 1])
    assert abs(front - vals["shock6_front_x"]) < 2.5


# --------------------------------------------------------------------------
# Degenerate calls and states: no steps, a negative count, the rest state.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("prec", ["f64", "f32", "f16dev", "bf16dev"])
def test_zero_steps_change_nothing_and_negative_counts_are_refused(prec):
    s = plbm.Solver(2, V5, 1.3, 34, 18, theta0=1.0, prec=prec)
    s.init(*smooth_fields(34, 18, 3))
    s.step(5)
    f0 = s.get_populations()
    n0 = s.diagnostics()["steps"]
    s.step(0)
    assert np.array_equal(s.get_populations(), f0) and s.diagnostics()["steps"] == n0 == 5
    assert s.step_status(-1) == plbm.PLBM_E_ARG
    assert np.array_equal(s.get_populations(), f0) and s.diagnostics()["steps"] == n0
    s.close()


@pytest.mark.parametrize("prec", ["f64", "f32", "f16dev", "bf16dev"])
@pytest.mark.parametrize("dim", [1, 2])
def test_rest_state_is_a_fixed_point(prec, dim):
    # rho = 1, u = 0, theta = theta0: f = w0, which streaming and the collision
    # (Eq. eq:srt with f^eq = w0) leave in place; the 16/32-bit kernels store the
    # deviation from w0, which stays exactly zero.  FP64 stores f itself and
    # recomputes f^eq from the rounded moments each step: the state stays uniform
    # bit for bit (every node does the same arithmetic) and moves by at most a few
    # roundings per step.
    nx, ny = 130, (18 if dim == 2 else 1)
    one, zero = np.ones((ny, nx)), np.zeros((ny, nx))
    s = plbm.Solver(dim, V5, 1.3, nx, ny, theta0=1.0, prec=prec)
    s.init(one, zero, zero if dim == 2 else None, one)
    f0 = s.get_populations()
    s.step(200)
    f = s.get_populations()
    assert s.check() == plbm.PLBM_OK
    if prec == "f64":
        assert np.all(f == f[:, :1, :1])
        assert np.max(np.abs(f - f0)) <= 200 * 16 * np.finfo(float).eps * np.max(f0)
    else:
        assert np.array_equal(f, f0)
    s.close()


@pytest.mark.parametrize("prec,ny,nx", [("f32", 48, 70), ("f16dev", 48, 70), ("bf16dev", 48, 70), ("f16dev", 12, 70),
                                        ("bf16dev", 16, 70), ("f16dev", 20, 70), ("f16dev", 14, 50),
                                        ("f16dev", 22, 200), ("f16dev", 2, 1)])
def test_plain_and_row_paired_layouts_give_the_same_state(prec, ny, nx):
    # The plain-layout kernel (one node per thread: odd ny, PLBM_FLAG_PLAIN_LAYOUT)
    # runs the single-lane forms of the row-paired kernel's packed operations,
    # each correctly rounded, so both layouts give every node the same bits.
    # ny = 12, 16, 20: most pair rows pull across the pair boundary (swapped lanes).
    # FP16 steps take two node pairs per thread (tiles of 64 pairs): nx = 50, ny = 14
    # gives an odd tile count (the last thread block has one tile), nx = 200 a ragged
    # last tile, and 1 x 2 a single node pair.
    fields = I.kh_fields(nx, ny=ny)
    out = []
    for plain in (False, True):
        s = plbm.Solver(2, V5, 1.3, nx, ny, theta0=1.0, prec=prec, plain_layout=plain)
        s.init(*fields)
        s.step(25)
        d = s.step_diagnostics(1)
        out.append((s.get_populations(), d))
        s.close()
    for o in out[1:]:
        assert np.array_equal(out[0][0], o[0])
        for k in ("mass", "jx", "jy", "energy", "rho_min", "theta_min"):
            assert abs(out[0][1][k] - o[1][k]) <= 1e-12 * max(1.0, abs(out[0][1][k])), k
