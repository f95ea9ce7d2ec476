"""Failure detection and checkpoint/resume on the GPU, with faults made on the host.

* Checkpoints: resuming from a checkpoint continues bit for bit as the
  uninterrupted run (2D row-paired FP32 and FP16, 2D FP64, 1D fixed ends, 3D
  z-paired BF16); a checkpoint with one corrupted byte (payload or header), a
  truncated one, or one of another lattice is rejected with PLBM_E_CHECKSUM and
  leaves the handle's state as it was.
* Initial fields with NaN, rho <= 0 or theta <= 0 are refused: host pointers by
  plbm_init itself (PLBM_E_ARG, handle left uninitialised), device pointers by
  the next status read (PLBM_E_DIVERGED).
The bounded tensor-core waits are exercised in test_surrogate_gpu.py.
"""
import numpy as np
import pytest

from paper_1402_5487_gb300 import build, inputs as I, plbm

pytestmark = pytest.mark.gpu

V5 = I.SET_013


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    plbm.lib()


def _kh(dim, prec, L=64, nz=1):
    if dim == 3:
        s = plbm.Solver(3, V5, 1.3, L, L, theta0=1.0, prec=prec, nz=nz)
        rho, ux, uy, uz, th = I.kh3_fields(L, L, nz)
        s.init(rho, ux, uy, th, uz=uz)
        return s
    if dim == 1:
        left, right = (1.1, 0.0, 0.5), (1.0, 0.0, 0.5)
        s = plbm.Solver(1, V5, 1.5, 200, 1, theta0=0.5, prec=prec, bc="fixed", left_state=left,
                        right_state=right)
        s.init(*I.shock_tube_fields(200, left, right))
        return s
    s = plbm.Solver(2, V5, 1.3, L, L - 2, theta0=1.0, prec=prec)
    s.init(*I.kh_fields(L, ny=L - 2))
    return s


CASES = [(2, "f32", 1), (2, "f16dev", 1), (2, "f64", 1), (1, "f64", 1), (3, "bf16dev", 6)]


@pytest.mark.parametrize("dim,prec,nz", CASES, ids=["%dd-%s" % (d, p) for d, p, _ in CASES])
def test_resume_from_a_checkpoint_is_bit_identical(dim, prec, nz):
    a = _kh(dim, prec, L=32 if dim == 3 else 64, nz=nz)
    a.step(17)                      # odd: the current array is the second one
    ck = a.checkpoint()
    a.step(23)
    ref = a.get_populations()
    b = _kh(dim, prec, L=32 if dim == 3 else 64, nz=nz)
    b.step(3)                       # some other state, to be replaced
    assert b.restore(ck) == plbm.PLBM_OK
    assert b.diagnostics()["steps"] == 17
    b.step(23)
    assert np.array_equal(b.get_populations(), ref)
    assert b.diagnostics()["steps"] == 40
    a.close()
    b.close()


def test_corrupted_or_foreign_checkpoints_are_rejected():
    a = _kh(2, "f32")
    a.step(5)
    ck = a.checkpoint()
    before = a.get_populations()
    for where in (len(ck) - 1, len(ck) // 2, 100, 40, 9):   # payload, header fields, magic
        bad = ck.copy()
        bad[where] ^= 0x10
        assert a.restore(bad) == plbm.PLBM_E_CHECKSUM, where
    assert a.restore(ck[:-8]) == plbm.PLBM_E_CHECKSUM
    assert a.restore(ck[:64]) == plbm.PLBM_E_CHECKSUM
    other = plbm.Solver(2, V5, 1.25, 64, 62, theta0=1.0, prec="f32")   # another omega
    other.init(*I.kh_fields(64, ny=62))
    assert other.restore(ck) == plbm.PLBM_E_CHECKSUM
    assert "another lattice" in plbm.last_error(other.h)
    other.close()
    assert np.array_equal(a.get_populations(), before)      # nothing was changed
    assert a.diagnostics()["steps"] == 5
    assert a.restore(ck) == plbm.PLBM_OK
    a.close()


@pytest.mark.parametrize("what", ["nan_ux", "inf_theta", "rho_zero", "theta_negative"])
def test_bad_initial_fields_from_host_memory_are_refused(what):
    L = 48
    rho, ux, uy, th = (np.array(a, dtype=np.float64) for a in I.kh_fields(L))
    if what == "nan_ux":
        ux[7, 11] = np.nan
    elif what == "inf_theta":
        th[0, 0] = np.inf
    elif what == "rho_zero":
        rho[L - 1, L - 1] = 0.0
    else:
        th[20, 3] = -0.5
    s = plbm.Solver(2, V5, 1.3, L, L, theta0=1.0, prec="f32")
    with pytest.raises(plbm.PlbmError) as e:
        s.init(rho, ux, uy, th)
    assert e.value.status == plbm.PLBM_E_ARG
    assert s.step_status(1) == plbm.PLBM_E_STATE          # left uninitialised
    s.init(*I.kh_fields(L))                               # good fields are accepted again
    s.step(2)
    assert s.check() == plbm.PLBM_OK
    s.close()


def test_bad_initial_fields_from_device_memory_are_reported_by_the_status_read():
    import torch
    L = 48
    fields = [torch.tensor(np.array(a, dtype=np.float64), device="cuda") for a in I.kh_fields(L)]
    fields[1][5, 5] = float("nan")
    s = plbm.Solver(2, V5, 1.3, L, L, theta0=1.0, prec="f64")
    s.init(*fields)
    assert s.check() == plbm.PLBM_E_DIVERGED
    s.close()


def test_bad_initial_fields_of_a_3d_lattice_are_refused():
    n = 8
    rho, ux, uy, uz, th = (np.array(a, dtype=np.float64) for a in I.kh3_fields(n, n, n))
    uz[3, 2, 1] = np.nan
    s = plbm.Solver(3, V5, 1.3, n, n, theta0=1.0, prec="f32", nz=n)
    with pytest.raises(plbm.PlbmError) as e:
        s.init(rho, ux, uy, th, uz=uz)
    assert e.value.status == plbm.PLBM_E_ARG
    s.close()
