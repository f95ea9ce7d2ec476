"""The C ABI library builds, loads and exports every symbol of include/plbm.h.

CPU-only checks of host logic: descriptor validation, the FP64 coefficients
computed by the library's host code (against the oracle), the positivity gate
of Sec. 3.1, and that creating a solver without a GPU fails loudly.
"""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle as O
from paper_1402_5487_gb300 import build, plbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build.build()
    return plbm.lib()


def header_functions():
    with open(os.path.join(ROOT, "include", "plbm.h")) as fh:
        text = fh.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(plbm_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_expected_calls():
    names = header_functions()
    for core in ("plbm_create", "plbm_init", "plbm_step", "plbm_moments", "plbm_destroy"):
        assert core in names


def test_every_declared_symbol_is_exported(L):
    for name in header_functions():
        assert hasattr(L, name), name
    assert set(header_functions()) == set(plbm.SIGNATURES)


def test_abi_version(L):
    assert L.plbm_abi_version() == 2


@pytest.mark.parametrize("v", [(0, 1, -1, 3, -3), (0, 1, -1, 2, -2), (0, 2, -4), (1, -1, 3, -3),
                               (0, 1, -1, 2, -2, 3, -3), (0, 1, -1)])
def test_library_coefficients_match_oracle(L, v):
    C = plbm.coefficients(v)
    ref = O.vandermonde_inverse(v)
    assert np.max(np.abs(C - ref)) <= 1e-14 * max(1.0, np.max(np.abs(ref)))


def test_coefficients_reject_repeated_velocity(L):
    with pytest.raises(plbm.PlbmError):
        plbm.coefficients((0, 1, 1))


def _create(desc):
    h = ctypes.c_void_p()
    st = plbm.lib().plbm_create(ctypes.byref(desc), ctypes.byref(h))
    return st, h


@pytest.mark.parametrize("field,value", [("omega", 2.0), ("omega", -0.1), ("omega", float("nan")),
                                         ("theta0", 0.0), ("nx", 0), ("dim", 4), ("q1", 9),
                                         ("prec", 7), ("bc", 5), ("check_every", -1)])
def test_descriptor_validation(L, field, value):
    desc, keep = plbm.make_desc(2, (0, 1, -1, 3, -3), 1.3, 16, 16)
    setattr(desc, field, value)
    st, h = _create(desc)
    assert st == plbm.PLBM_E_ARG and not h.value
    assert plbm.last_error(None)
    assert plbm.workspace_bytes(desc) == 0


@pytest.mark.parametrize("kw", [dict(v=(0, 1, -1, 3, -3), bc="fixed", left_state=(1, 0, 1), right_state=(1, 0, 1)),
                                dict(v=(0, 1, -1, 2, -3)),            # not a symmetric pair set
                                dict(v=(0, 1, -1)),                   # q1 = 3 needs FP64 in 3D
                                dict(v=(0, 1, -1, 3, -3), isothermal=True),
                                dict(v=(0, 1, -1, 3, -3), nz=0)],
                         ids=["fixed-ends", "asymmetric", "q1-3", "isothermal", "nz-0"])
def test_3d_descriptor_validation(L, kw):
    kw = dict(kw)
    v = kw.pop("v")
    nz = kw.pop("nz", 8)
    desc, keep = plbm.make_desc(3, v, 1.3, 16, 8, prec="f32", nz=nz, skip_admissibility=True, **kw)
    st, h = _create(desc)
    assert st == plbm.PLBM_E_ARG and not h.value, plbm.last_error(None)


def test_3d_workspace_counts_q1_cubed(L):
    desc, keep = plbm.make_desc(3, (0, 1, -1, 3, -3), 1.3, 64, 8, prec="f32", nz=4)
    # two population arrays of 125 x 4 x 8 rows x 64 floats, plus scratch
    assert plbm.workspace_bytes(desc) >= 2 * 125 * 4 * 8 * 64 * 4
    desc, keep = plbm.make_desc(3, (0, 1, -1), 1.2, 64, 8, prec="f64", nz=4, isothermal=True, theta0=1 / 3)
    assert plbm.workspace_bytes(desc) >= 2 * 27 * 4 * 8 * 64 * 8


def test_repeated_velocity_rejected(L):
    desc, keep = plbm.make_desc(1, (0, 1, 1, 3, -3), 1.3, 16)
    st, _ = _create(desc)
    assert st == plbm.PLBM_E_ARG


def test_one_d_needs_ny_one(L):
    desc, keep = plbm.make_desc(1, (0, 1, -1, 3, -3), 1.3, 16)
    desc.ny = 4
    assert _create(desc)[0] == plbm.PLBM_E_ARG


def test_fixed_ends_need_states(L):
    desc, keep = plbm.make_desc(1, (0, 1, -1, 3, -3), 1.5, 100, bc="fixed")
    assert _create(desc)[0] == plbm.PLBM_E_ARG
    desc, keep = plbm.make_desc(1, (0, 1, -1, 3, -3), 1.5, 100, bc="fixed",
                                left_state=(1.0, 0.0, -0.5), right_state=(1.0, 0.0, 0.5))
    assert _create(desc)[0] == plbm.PLBM_E_ARG


def test_positivity_gate_matches_oracle(L):
    # {0,+-2,+-3} has the u = 0 window 4/3 < theta < 3 (Eq. eq:1d5v): theta0 = 1 is rejected
    # at create; {0,+-1,+-3} at theta0 = 1 is admissible up to the oracle's positivity edge.
    from oracle import stability as S
    desc, keep = plbm.make_desc(2, (0, 2, -2, 3, -3), 1.3, 16, 16, theta0=1.0)
    assert _create(desc)[0] == plbm.PLBM_E_INADMISSIBLE
    assert "inadmissible" in plbm.last_error(None)
    lo, hi = S.positivity_interval((0, 1, -1, 3, -3), 1.0)
    for u_max, expect_ok in ((0.98 * hi, True), (1.02 * hi, False)):
        desc, keep = plbm.make_desc(2, (0, 1, -1, 3, -3), 1.3, 16, 16, theta0=1.0, u_max=u_max)
        st, h = _create(desc)
        if expect_ok:
            assert st != plbm.PLBM_E_INADMISSIBLE
            if st == plbm.PLBM_OK:
                plbm.lib().plbm_destroy(h)
        else:
            assert st == plbm.PLBM_E_INADMISSIBLE


def _gpu_present():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.mark.skipif(_gpu_present(), reason="checks the no-GPU failure path")
def test_create_without_gpu_fails_loudly(L):
    desc, keep = plbm.make_desc(2, (0, 1, -1, 3, -3), 1.3, 16, 16)
    st, h = _create(desc)
    assert st == plbm.PLBM_E_CUDA and not h.value
    assert "CUDA" in plbm.last_error(None) or "device" in plbm.last_error(None)


def test_status_strings(L):
    assert plbm.status_name(plbm.PLBM_E_DIVERGED) == "PLBM_E_DIVERGED"
    assert plbm.status_name(123) == "PLBM_E_UNKNOWN"
