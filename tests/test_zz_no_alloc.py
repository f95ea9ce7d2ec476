"""plbm_diagnostics_noalloc against plbm_diagnostics (GPU).

Some callers cannot allocate device memory (host-owned memory, no-allocation
embedded set-ups).  plbm_diagnostics_noalloc serves them with a
static scratch array instead of a workspace.  This test calls it through the C
ABI on caller-held device populations and checks its six outputs against the
handle-based plbm_diagnostics on the same state, twice in a row with different
states (the shared scratch keeps the previous call's contents); that it
leaves the device's free memory and torch's allocator untouched; and that it
works in a context the caller created with the driver API, where the static
array sits at another address than in the runtime's primary context.  The file
name makes pytest collect it last.
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


def test_noalloc_allocates_nothing():
    """After a first call (which loads the kernels), calls change neither the
    device's free memory nor torch's allocator."""
    import torch
    build.build()
    nx, ny = 64, 48
    s = plbm.Solver(2, V5, 1.3, nx, ny, theta0=1.0, prec="f64")
    s.init(*I.kh_fields(nx, ny=ny))
    f_dev = s.get_populations(on_device=True)
    out_dev = torch.empty(6, dtype=torch.float64, device=s.device)
    _noalloc(s, f_dev, out_dev, torch)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info(s.device)
    alloc0 = torch.cuda.memory_allocated(s.device)
    for _ in range(3):
        _noalloc(s, f_dev, out_dev, torch)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info(s.device)[0] == free0
    assert torch.cuda.memory_allocated(s.device) == alloc0
    s.close()


def _driver():
    cu = ctypes.CDLL("libcuda.so.1")
    c_u64p = ctypes.POINTER(ctypes.c_uint64)
    sig = {
        "cuCtxGetCurrent": [ctypes.POINTER(ctypes.c_void_p)],
        "cuCtxSetCurrent": [ctypes.c_void_p],
        "cuCtxGetDevice": [ctypes.POINTER(ctypes.c_int)],
        "cuCtxCreate_v2": [ctypes.POINTER(ctypes.c_void_p), ctypes.c_uint, ctypes.c_int],
        "cuCtxDestroy_v2": [ctypes.c_void_p],
        "cuCtxSynchronize": [],
        "cuMemAlloc_v2": [c_u64p, ctypes.c_size_t],
        "cuMemFree_v2": [ctypes.c_uint64],
        "cuMemcpyHtoD_v2": [ctypes.c_uint64, ctypes.c_void_p, ctypes.c_size_t],
        "cuMemcpyDtoH_v2": [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_size_t],
    }
    for name, args in sig.items():
        fn = getattr(cu, name)
        fn.argtypes, fn.restype = args, ctypes.c_int
    return cu


def test_noalloc_in_a_driver_created_context():
    """A plug-in host may run the library in a context it created itself.  The
    static array has a different address there; the call must find it and give
    the same sums as in the primary context, twice in a row."""
    import torch
    build.build()
    nx, ny = 96, 40
    s = plbm.Solver(2, V5, 1.3, nx, ny, theta0=1.0, prec="f64")
    s.init(*I.kh_fields(nx, ny=ny))
    states = []
    for steps in (5, 11):
        s.step(steps)
        d = s.diagnostics()
        states.append((np.ascontiguousarray(s.get_populations(), dtype=np.float64),
                       np.array([d["mass"], d["jx"], d["jy"], d["energy"], d["rho_min"], d["theta_min"]])))
    out_dev = torch.empty(6, dtype=torch.float64, device=s.device)
    _noalloc(s, s.get_populations(on_device=True), out_dev, torch)  # primary context first
    torch.cuda.synchronize()

    cu = _driver()
    primary, ctx = ctypes.c_void_p(), ctypes.c_void_p()
    dev = ctypes.c_int()
    assert cu.cuCtxGetCurrent(ctypes.byref(primary)) == 0 and primary.value
    assert cu.cuCtxGetDevice(ctypes.byref(dev)) == 0
    assert cu.cuCtxCreate_v2(ctypes.byref(ctx), 0, dev.value) == 0
    va = (ctypes.c_int * len(V5))(*V5)
    d_f, d_out = ctypes.c_uint64(0), ctypes.c_uint64(0)
    results = []
    try:
        nbytes = states[0][0].nbytes
        assert cu.cuMemAlloc_v2(ctypes.byref(d_f), nbytes) == 0
        assert cu.cuMemAlloc_v2(ctypes.byref(d_out), 48) == 0
        for f_host, _ in states:
            assert cu.cuMemcpyHtoD_v2(d_f.value, f_host.ctypes.data, nbytes) == 0
            st = plbm.lib().plbm_diagnostics_noalloc(2, len(V5), va, nx, ny, d_f.value, d_out.value, None)
            assert st == plbm.PLBM_OK, plbm.last_error(None)
            assert cu.cuCtxSynchronize() == 0
            got = np.zeros(6)
            assert cu.cuMemcpyDtoH_v2(got.ctypes.data, d_out.value, 48) == 0
            results.append(got)
    finally:
        if d_f.value:
            cu.cuMemFree_v2(d_f.value)
        if d_out.value:
            cu.cuMemFree_v2(d_out.value)
        cu.cuCtxDestroy_v2(ctx)
        cu.cuCtxSetCurrent(primary)
    for got, (_, ref) in zip(results, states):
        scale = np.array([abs(ref[0])] * 4 + [1.0, 1.0])
        assert np.all(np.abs(got - ref) <= 1e-12 * scale), (got, ref)
    # the primary context's cached address is still the right one
    got = _noalloc(s, s.get_populations(on_device=True), out_dev, torch)
    scale = np.array([abs(states[1][1][0])] * 4 + [1.0, 1.0])
    assert np.all(np.abs(got - states[1][1]) <= 1e-12 * scale)
    s.close()
