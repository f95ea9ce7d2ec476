"""ctypes binding of libplbm (include/plbm.h): argument marshalling only.

Every step of the method runs in the CUDA kernels of ``libplbm.so``.  PyTorch
supplies device memory (the handle's workspace) and the CUDA stream; NumPy
arrays are accepted for host-side inputs and outputs.  There is no CPU path:
if the shared library is missing or no GPU is present the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libplbm.so")

PLBM_OK = 0
PLBM_E_ARG = -1
PLBM_E_CUDA = -2
PLBM_E_INADMISSIBLE = -3
PLBM_E_DIVERGED = -4
PLBM_E_TIMEOUT = -5
PLBM_E_STATE = -6
PLBM_E_CHECKSUM = -7
PLBM_E_NOMEM = -8

PREC = {"f64": 0, "f32": 1, "f16dev": 2, "bf16dev": 3}
BC = {"periodic": 0, "fixed": 1}
FLAG_ISOTHERMAL = 0x1
FLAG_SKIP_ADMISSIBILITY = 0x2
FLAG_PLAIN_LAYOUT = 0x4


class PlbmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (status_name(status) if _lib else status, msg))
        self.status = status


class PlbmDesc(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int),
        ("q1", ctypes.c_int),
        ("v", ctypes.POINTER(ctypes.c_int)),
        ("omega", ctypes.c_double),
        ("theta0", ctypes.c_double),
        ("nx", ctypes.c_int),
        ("ny", ctypes.c_int),
        ("prec", ctypes.c_int),
        ("bc", ctypes.c_int),
        ("left_state", ctypes.POINTER(ctypes.c_double)),
        ("right_state", ctypes.POINTER(ctypes.c_double)),
        ("stream", ctypes.c_void_p),
        ("flags", ctypes.c_uint),
        ("check_every", ctypes.c_int),
        ("u_max", ctypes.c_double),
        ("workspace", ctypes.c_void_p),
        ("workspace_bytes", ctypes.c_size_t),
        ("device", ctypes.c_int),
        ("nz", ctypes.c_int),
    ]


class PlbmDiag(ctypes.Structure):
    _fields_ = [
        ("mass", ctypes.c_double),
        ("jx", ctypes.c_double),
        ("jy", ctypes.c_double),
        ("energy", ctypes.c_double),
        ("rho_min", ctypes.c_double),
        ("theta_min", ctypes.c_double),
        ("status", ctypes.c_uint32),
        ("steps", ctypes.c_int64),
    ]


_D = ctypes.POINTER(ctypes.c_double)
_H = ctypes.c_void_p
_lock = threading.Lock()
_lib = None

# name -> (restype, argtypes) for every function declared in include/plbm.h
SIGNATURES = {
    "plbm_abi_version": (ctypes.c_int, []),
    "plbm_coefficients": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_int), _D]),
    "plbm_workspace_bytes": (ctypes.c_size_t, [ctypes.POINTER(PlbmDesc)]),
    "plbm_linear_stability": (ctypes.c_int, [ctypes.POINTER(PlbmDesc), ctypes.c_double, ctypes.c_int,
                                             ctypes.c_double, _D]),
    "plbm_positivity": (ctypes.c_int, [ctypes.POINTER(PlbmDesc), ctypes.c_double, _D]),
    "plbm_batch_create": (ctypes.c_int, [ctypes.POINTER(PlbmDesc), ctypes.c_int, ctypes.c_void_p,
                                         ctypes.POINTER(ctypes.c_void_p)]),
    "plbm_batch_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "plbm_batch_instance": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(_H)]),
    "plbm_batch_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_long, ctypes.c_int]),
    "plbm_batch_check": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]),
    "plbm_batch_set_config": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    "plbm_batch_set_order": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "plbm_batch_get_order": (ctypes.c_int, [ctypes.c_void_p]),
    "plbm_batch_info": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.POINTER(ctypes.c_int)] * 5),
    "plbm_batch_tune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                       ctypes.POINTER(ctypes.c_int), _D]),
    "plbm_batch_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "plbm_batch_groups": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.POINTER(ctypes.c_int)] * 3),
    "plbm_create": (ctypes.c_int, [ctypes.POINTER(PlbmDesc), ctypes.POINTER(_H)]),
    "plbm_destroy": (ctypes.c_int, [_H]),
    "plbm_init": (ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                 ctypes.c_void_p, ctypes.c_int]),
    "plbm_step": (ctypes.c_int, [_H, ctypes.c_long]),
    "plbm_check": (ctypes.c_int, [_H]),
    "plbm_moments": (ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_int]),
    "plbm_diagnostics": (ctypes.c_int, [_H, ctypes.POINTER(PlbmDiag)]),
    "plbm_step_diagnostics": (ctypes.c_int, [_H, ctypes.c_long, ctypes.POINTER(PlbmDiag)]),
    "plbm_conserved": (ctypes.c_int, [_H, _D]),
    "plbm_init3": (ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                  ctypes.c_void_p, ctypes.c_int]),
    "plbm_moments3": (ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_int]),
    "plbm_conserved3": (ctypes.c_int, [_H, _D]),
    "plbm_get_populations": (ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_int]),
    "plbm_set_populations": (ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_int, ctypes.c_int64]),
    "plbm_get_info": (ctypes.c_int, [_H, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.c_size_t)]),
    "plbm_device_populations": (ctypes.c_int, [_H, ctypes.POINTER(ctypes.c_void_p)]),
    "plbm_slab_rows": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(ctypes.c_int)]),
    "plbm_halo_width": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "plbm_halo_plan": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                      ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "plbm_slabs_create": (ctypes.c_int, [ctypes.POINTER(PlbmDesc), ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]),
    "plbm_slabs_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "plbm_slabs_slab": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(_H),
                                       ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "plbm_slabs_init": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_void_p] * 4),
    "plbm_slabs_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_long]),
    "plbm_slabs_moments": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_void_p] * 4),
    "plbm_slabs_get_populations": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "plbm_slabs_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "plbm_checkpoint_bytes": (ctypes.c_size_t, [_H]),
    "plbm_checkpoint_save": (ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_size_t]),
    "plbm_checkpoint_load": (ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_size_t]),
    "plbm_diagnostics_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                                 ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                                 ctypes.c_void_p, ctypes.c_void_p]),
    "plbm_sur_num_params": (ctypes.c_int, []),
    "plbm_sur_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_ulonglong,
                                       ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "plbm_sur_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "plbm_sur_set_params": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "plbm_sur_set_option": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    "plbm_sur_set_mean_penalty": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_float]),
    "plbm_sur_check": (ctypes.c_int, [ctypes.c_void_p]),
    "plbm_sur_get_params": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "plbm_sur_set_norm": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.POINTER(ctypes.c_float)] * 4),
    "plbm_sur_forward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]),
    "plbm_sur_backward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]),
    "plbm_sur_copy": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]),
    "plbm_sur_train_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_float, ctypes.POINTER(ctypes.c_float)]),
    "plbm_sur_pack_fields": (ctypes.c_int, [ctypes.c_void_p] * 4 + [ctypes.c_longlong, ctypes.c_void_p,
                                                                     ctypes.c_void_p]),
    "plbm_sur_assemble": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_longlong, ctypes.c_void_p,
                                         ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]),
    "plbm_sur_assemble_noise": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_longlong, ctypes.c_void_p,
                                               ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_float,
                                               ctypes.c_ulonglong]),
    "plbm_sur_advance": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p), ctypes.c_int,
                                        ctypes.c_int, ctypes.c_double, ctypes.POINTER(ctypes.c_int)]),
    "plbm_sur_last_drift": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "plbm_sur_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "plbm_last_error": (ctypes.c_char_p, [_H]),
    "plbm_status_string": (ctypes.c_char_p, [ctypes.c_int]),
}


def lib():
    """Load libplbm.so (built by ``paper_1402_5487_gb300.build``); raise if absent."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    "libplbm.so not built (%s); run paper_1402_5487_gb300.build.build() "
                    "(the CUDA library is required: there is no CPU path)" % LIB_PATH)
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
        return _lib


def status_name(st: int) -> str:
    return lib().plbm_status_string(int(st)).decode()


def last_error(h=None) -> str:
    return lib().plbm_last_error(h).decode(errors="replace")


def _ok(st: int, h=None):
    if st != PLBM_OK:
        raise PlbmError(st, last_error(h))


def coefficients(v) -> np.ndarray:
    """c_ij of Eq. (eq:rdr) computed by the library's host code (FP64)."""
    q1 = len(v)
    va = (ctypes.c_int * q1)(*[int(a) for a in v])
    C = np.zeros(q1 * q1)
    _ok(lib().plbm_coefficients(q1, va, C.ctypes.data_as(_D)))
    return C.reshape(q1, q1)


def make_desc(dim, v, omega, nx, ny=1, theta0=1.0, prec="f32", bc="periodic", left_state=None,
              right_state=None, isothermal=False, check_every=0, u_max=0.0, stream=None,
              device=0, skip_admissibility=False, nz=1, plain_layout=False):
    """Build a PlbmDesc; the returned tuple keeps the ctypes buffers alive."""
    q1 = len(v)
    va = (ctypes.c_int * q1)(*[int(a) for a in v])
    d = PlbmDesc()
    d.dim, d.q1, d.v = int(dim), q1, va
    d.omega, d.theta0 = float(omega), float(theta0)
    d.nx, d.ny = int(nx), int(ny)
    d.prec = PREC[prec] if isinstance(prec, str) else int(prec)
    d.bc = BC[bc] if isinstance(bc, str) else int(bc)
    keep = [va]
    if left_state is not None:
        ls = (ctypes.c_double * 3)(*[float(a) for a in left_state])
        rs = (ctypes.c_double * 3)(*[float(a) for a in right_state])
        d.left_state = ctypes.cast(ls, _D)
        d.right_state = ctypes.cast(rs, _D)
        keep += [ls, rs]
    d.stream = stream
    d.flags = ((FLAG_ISOTHERMAL if isothermal else 0) | (FLAG_SKIP_ADMISSIBILITY if skip_admissibility else 0) |
               (FLAG_PLAIN_LAYOUT if plain_layout else 0))
    d.check_every = int(check_every)
    d.u_max = float(u_max)
    d.device = int(device)
    d.nz = int(nz) if int(dim) == 3 else 1
    return d, keep


def linear_stability(dim, v, omega, theta0=1.0, ux=0.0, nk=48, isothermal=False, stop_above=0.0) -> float:
    """max |lambda| of the library's linearised one-step operator (host computation)."""
    desc, keep = make_desc(dim, v, omega, 4, 4 if dim == 2 else 1, theta0=theta0, isothermal=isothermal,
                           skip_admissibility=True)
    out = ctypes.c_double()
    _ok(lib().plbm_linear_stability(ctypes.byref(desc), float(ux), int(nk), float(stop_above),
                                    ctypes.byref(out)))
    return out.value


def positivity(dim, v, theta0=1.0, u_max=0.0) -> float:
    """min_i min_{|u| <= u_max} r_i(u, theta0) from the library's host code."""
    desc, keep = make_desc(dim, v, 1.0, 4, 4 if dim == 2 else 1, theta0=theta0, skip_admissibility=True)
    out = ctypes.c_double()
    _ok(lib().plbm_positivity(ctypes.byref(desc), float(u_max), ctypes.byref(out)))
    return out.value


def workspace_bytes(desc: PlbmDesc) -> int:
    return int(lib().plbm_workspace_bytes(ctypes.byref(desc)))


def _ptr(a) -> int | None:
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()  # torch tensor


class Solver:
    """One lattice on one GPU (a handle of the C ABI).

    Device memory for populations and scratch comes from a PyTorch uint8 tensor
    passed as the handle's workspace; launches go to PyTorch's current stream of
    the device unless ``stream`` is given (a ``torch.cuda.Stream``).
    """

    def __init__(self, dim, v, omega, nx, ny=1, theta0=1.0, prec="f32", bc="periodic",
                 left_state=None, right_state=None, isothermal=False, check_every=0, u_max=0.0,
                 device=0, stream=None, skip_admissibility=False, torch_workspace=True, nz=1,
                 plain_layout=False):
        import torch  # device memory and streams only

        self.torch = torch
        self.device = torch.device("cuda", device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.dim, self.v, self.q1 = dim, tuple(int(a) for a in v), len(v)
        self.q = self.q1 ** dim
        self.nx, self.ny = int(nx), (int(ny) if dim >= 2 else 1)
        self.nz = int(nz) if dim == 3 else 1
        self.prec = prec
        desc, self._keep = make_desc(dim, v, omega, nx, self.ny, theta0, prec, bc, left_state,
                                     right_state, isothermal, check_every, u_max,
                                     self.stream.cuda_stream, device, skip_admissibility, self.nz,
                                     plain_layout)
        self._ws = None
        if torch_workspace:
            nbytes = workspace_bytes(desc)
            if nbytes == 0:
                # invalid descriptor: let create report the reason
                pass
            else:
                self._ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
                base = self._ws.data_ptr()
                desc.workspace = (base + 255) // 256 * 256
                desc.workspace_bytes = nbytes
        h = _H()
        st = lib().plbm_create(ctypes.byref(desc), ctypes.byref(h))
        if st != PLBM_OK:
            raise PlbmError(st, last_error(None))
        self.h = h
        self.desc = desc

    # -- lifetime ----------------------------------------------------------
    def close(self):
        if getattr(self, "_borrowed", False):
            self.h = None
            return
        if getattr(self, "h", None):
            lib().plbm_destroy(self.h)
            self.h = None
        self._ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- calls ---------------------------------------------------------------
    def _field_args(self, arrs):
        on_dev = None
        ptrs = []
        keep = []
        for a in arrs:
            if a is None:
                ptrs.append(None)
                continue
            if isinstance(a, np.ndarray):
                a = np.ascontiguousarray(a, dtype=np.float64)
                assert a.size == self.nx * self.ny * self.nz
                dev = 0
            else:
                assert a.dtype == self.torch.float64 and a.is_contiguous() and a.numel() == self.nx * self.ny * self.nz
                dev = 1
            if on_dev is None:
                on_dev = dev
            elif on_dev != dev:
                raise ValueError("mix of host and device arrays")
            keep.append(a)
            ptrs.append(_ptr(a))
        return ptrs, on_dev or 0, keep

    def init(self, rho, ux, uy=None, theta=None, uz=None):
        """Equilibrium initial state; 3D handles take uz as well (fields [nz][ny][nx])."""
        if self.dim == 3:
            ptrs, on_dev, keep = self._field_args([rho, ux, uy, uz, theta])
            _ok(lib().plbm_init3(self.h, *ptrs, on_dev), self.h)
            return
        ptrs, on_dev, keep = self._field_args([rho, ux, uy, theta])
        _ok(lib().plbm_init(self.h, *ptrs, on_dev), self.h)

    def step(self, n: int = 1):
        _ok(lib().plbm_step(self.h, int(n)), self.h)

    def step_status(self, n: int = 1) -> int:
        """Like step() but returns the status code instead of raising."""
        return int(lib().plbm_step(self.h, int(n)))

    def check(self) -> int:
        return int(lib().plbm_check(self.h))

    def moments(self, on_device: bool = False):
        """(rho, ux, uy, theta) as FP64 [ny][nx] NumPy arrays (or torch CUDA tensors);
        3D handles: (rho, ux, uy, uz, theta), each [nz][ny][nx]."""
        shp = (self.ny, self.nx) if self.dim < 3 else (self.nz, self.ny, self.nx)
        k = 5 if self.dim == 3 else 4
        if on_device:
            outs = [self.torch.empty(shp, dtype=self.torch.float64, device=self.device) for _ in range(k)]
        else:
            outs = [np.empty(shp) for _ in range(k)]
        call = lib().plbm_moments3 if self.dim == 3 else lib().plbm_moments
        _ok(call(self.h, *[_ptr(o) for o in outs], 1 if on_device else 0), self.h)
        return tuple(outs)

    def diagnostics(self) -> dict:
        d = PlbmDiag()
        _ok(lib().plbm_diagnostics(self.h, ctypes.byref(d)), self.h)
        return {k: getattr(d, k) for k, _ in PlbmDiag._fields_}

    def step_diagnostics(self, n: int) -> dict:
        """n steps, the last fused with the FP64 reductions (plbm_step_diagnostics)."""
        d = PlbmDiag()
        _ok(lib().plbm_step_diagnostics(self.h, int(n), ctypes.byref(d)), self.h)
        return {k: getattr(d, k) for k, _ in PlbmDiag._fields_}

    def conserved(self) -> np.ndarray:
        """(mass, jx, jy, energy); 3D handles: (mass, jx, jy, jz, energy)."""
        out = np.zeros(5 if self.dim == 3 else 4)
        call = lib().plbm_conserved3 if self.dim == 3 else lib().plbm_conserved
        _ok(call(self.h, out.ctypes.data_as(_D)), self.h)
        return out

    def _pop_shape(self):
        return (self.q, self.ny, self.nx) if self.dim < 3 else (self.q, self.nz, self.ny, self.nx)

    def get_populations(self, on_device: bool = False):
        shp = self._pop_shape()
        out = (self.torch.empty(shp, dtype=self.torch.float64, device=self.device) if on_device
               else np.empty(shp))
        _ok(lib().plbm_get_populations(self.h, _ptr(out), 1 if on_device else 0), self.h)
        return out

    def set_populations(self, f, step: int = 0):
        if isinstance(f, np.ndarray):
            f = np.ascontiguousarray(f, dtype=np.float64)
            on = 0
        else:
            on = 1
        assert tuple(f.shape) == self._pop_shape()
        _ok(lib().plbm_set_populations(self.h, _ptr(f), on, int(step)), self.h)

    def checkpoint(self) -> np.ndarray:
        """Header + stored populations + checksum (plbm_checkpoint_save), as bytes."""
        n = int(lib().plbm_checkpoint_bytes(self.h))
        buf = np.empty(n, dtype=np.uint8)
        _ok(lib().plbm_checkpoint_save(self.h, buf.ctypes.data, n), self.h)
        return buf

    def restore(self, buf) -> int:
        """plbm_checkpoint_load; returns the status (PLBM_E_CHECKSUM is not raised)."""
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        return int(lib().plbm_checkpoint_load(self.h, buf.ctypes.data, buf.size))

    def info(self):
        q, pitch, nb = ctypes.c_int(), ctypes.c_int(), ctypes.c_size_t()
        _ok(lib().plbm_get_info(self.h, ctypes.byref(q), ctypes.byref(pitch), ctypes.byref(nb)), self.h)
        return {"q": q.value, "pitch": pitch.value, "population_bytes": nb.value}

    @classmethod
    def _wrap(cls, h, dim, v, nx, ny, prec, stream, torch):
        """A Solver view of a handle owned by a batch (not closed by this object)."""
        s = cls.__new__(cls)
        s.torch, s.h, s._ws, s._keep = torch, h, None, []
        s.device = torch.device("cuda", torch.cuda.current_device())
        s.stream = stream
        s.dim, s.v, s.q1 = dim, tuple(int(a) for a in v), len(v)
        s.q = s.q1 ** dim
        s.nx, s.ny, s.nz, s.prec = nx, ny, 1, prec
        s._borrowed = True
        return s

    def device_populations_ptr(self) -> int:
        p = ctypes.c_void_p()
        _ok(lib().plbm_device_populations(self.h, ctypes.byref(p)), self.h)
        return int(p.value)


# ---------------------------------------------------------------------------
# Domain decomposition along y (plbm_slab_rows, plbm_halo_plan, plbm_slabs_*).
# ---------------------------------------------------------------------------
def slab_rows(ny: int, nslabs: int, k: int):
    """(y0, rows) of slab k (host computation of the library)."""
    y0, rows = ctypes.c_int(), ctypes.c_int()
    _ok(lib().plbm_slab_rows(int(ny), int(nslabs), int(k), ctypes.byref(y0), ctypes.byref(rows)))
    return y0.value, rows.value


def halo_width(v) -> int:
    va = (ctypes.c_int * len(v))(*[int(a) for a in v])
    return int(lib().plbm_halo_width(len(v), va))


def halo_plan(v, side: int):
    """Populations a slab's halo needs: side -1 the rows below (v_y > 0), +1 above (v_y < 0)."""
    q1 = len(v)
    va = (ctypes.c_int * q1)(*[int(a) for a in v])
    pops = (ctypes.c_int * (q1 * q1))()
    n = ctypes.c_int()
    _ok(lib().plbm_halo_plan(q1, va, int(side), pops, ctypes.byref(n)))
    return [pops[i] for i in range(n.value)]


class Slabs:
    """A periodic 2D lattice split along y into slabs that exchange halo rows (one device)."""

    def __init__(self, v, omega, nx, ny, nslabs, theta0=1.0, prec="f32", device=0, u_max=0.0, stream=None):
        """stream: a torch.cuda.Stream (not the default stream) for every launch; None: the library's own."""
        self.v, self.nx, self.ny, self.n = tuple(int(a) for a in v), int(nx), int(ny), int(nslabs)
        self.q = len(v) ** 2
        self.stream = stream
        desc, self._keep = make_desc(2, v, omega, nx, ny, theta0=theta0, prec=prec, device=device, u_max=u_max,
                                     stream=None if stream is None else stream.cuda_stream)
        s = ctypes.c_void_p()
        st = lib().plbm_slabs_create(ctypes.byref(desc), self.n, ctypes.byref(s))
        if st != PLBM_OK:
            raise PlbmError(st, lib().plbm_slabs_last_error(None).decode())
        self.s = s

    def _ok(self, st):
        if st != PLBM_OK:
            raise PlbmError(st, lib().plbm_slabs_last_error(self.s).decode())

    def init(self, rho, ux, uy, theta):
        arrs = [np.ascontiguousarray(np.broadcast_to(a, (self.ny, self.nx)), dtype=np.float64)
                for a in (rho, ux, uy, theta)]
        self._ok(lib().plbm_slabs_init(self.s, *[a.ctypes.data for a in arrs]))

    def step(self, n=1):
        self._ok(lib().plbm_slabs_step(self.s, int(n)))

    def moments(self):
        out = [np.empty((self.ny, self.nx)) for _ in range(4)]
        self._ok(lib().plbm_slabs_moments(self.s, *[a.ctypes.data for a in out]))
        return tuple(out)

    def get_populations(self):
        f = np.empty((self.q, self.ny, self.nx))
        self._ok(lib().plbm_slabs_get_populations(self.s, f.ctypes.data))
        return f

    def slab(self, k):
        h, y0, rows = _H(), ctypes.c_int(), ctypes.c_int()
        self._ok(lib().plbm_slabs_slab(self.s, int(k), ctypes.byref(h), ctypes.byref(y0), ctypes.byref(rows)))
        return h, y0.value, rows.value

    def close(self):
        if getattr(self, "s", None):
            lib().plbm_slabs_destroy(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
