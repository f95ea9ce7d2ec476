"""plbm_diagnostics_noalloc against plbm_diagnostics (GPU).

Some callers cannot allocate device memory (graph capture, host-owned memory,
no-allocation embedded set-ups).  plbm_diagnostics_noalloc serves them with a
static scratch array instead of a workspace.  This test calls it through the C
ABI on caller-held device populations and checks its six outputs against the
handle-based plbm_diagnostics on the same state, twice in a row with different
states (the shared scratch keeps the previous call's contents).  The file name
makes pytest collect it last.
"""
import ctypes

import numpy as np
import pytest

from paper_1402_5487_gb300 import build, inputs as I, plbm

pytestmark = pytest.mark.gpu

V5 = I.SET_013


def _noalloc(s, f_dev, out_dev, torch):
    va = (ctypes.c_int * len(s.v))(*s.v)
    st = plbm.lib().plbm_diagnostics_noalloc(s.dim, len(s.v), va, s.nx, s.ny, f_dev.data_ptr(),
                                             out_dev.data_ptr(), s.stream.cuda_stream)
    assert st == plbm.PLBM_OK, plbm.last_error(None)
    s.stream.synchronize()
    return out_dev.cpu().numpy().copy()


@pytest.mark.parametrize("dim,nx,ny,prec", [(2, 96, 80, "f64"), (2, 130, 33, "f32"), (1, 1000, 1, "f64")])
def test_noalloc_matches_handle_diagnostics(dim, nx, ny, prec):
    import torch
    build.build()
    if dim == 2:
        fields = I.kh_fields(nx, ny=ny)
        s = plbm.Solver(2, V5, 1.3, nx, ny, theta0=1.0, prec=prec)
    else:
        left, right = (1.1, 0.0, 0.5), (1.0, 0.0, 0.5)
        fields = I.shock_tube_fields(nx, left, right)
        s = plbm.Solver(1, V5, 1.5, nx, 1, theta0=0.5, prec=prec, bc="fixed", left_state=left,
                        right_state=right)
    s.init(*fields)
    out_dev = torch.empty(6, dtype=torch.float64, device=s.device)
    for steps in (7, 13):  # two calls in a row, on different states
        s.step(steps)
        f_dev = s.get_populations(on_device=True)
        got = _noalloc(s, f_dev, out_dev, torch)
        d = s.diagnostics()
        ref = np.array([d["mass"], d["jx"], d["jy"], d["energy"], d["rho_min"], d["theta_min"]])
        scale = np.array([abs(d["mass"])] * 4 + [1.0, 1.0])
        assert np.all(np.abs(got - ref) <= 1e-12 * scale), (got, ref)
    s.close()


def test_noalloc_rejects_oversized_lattice():
    import torch
    build.build()
    va = (ctypes.c_int * 5)(*V5)
    dummy = torch.empty(8, dtype=torch.float64, device="cuda")
    st = plbm.lib().plbm_diagnostics_noalloc(2, 5, va, 4096, 2048, dummy.data_ptr(), dummy.data_ptr(), None)
    assert st == plbm.PLBM_E_ARG
    assert "limit" in plbm.last_error(None)
