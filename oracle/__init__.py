"""Plain FP64 CPU oracle of the parametric lattice Boltzmann method.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import this package.  It shares
no code with the CUDA path (``paper_1402_5487_gb300``): no module here imports the
library or its binding.  The one import from that package is
``paper_1402_5487_gb300.inputs`` in ``oracle.kh_longrun``: the seeded input-field
generators that both sides take their inputs from, which hold none of the
method's arithmetic.

The arithmetic lives in ``plbm_oracle.c`` (plain C, FP64, ``-ffp-contract=off``),
loaded here through ctypes.  Companion tools written in NumPy:

* ``oracle.riemann``   exact Riemann solver of the Euler equations (Sec. 4,
  Table 3, the Rankine-Hugoniot relations printed there);
* ``oracle.stability`` linearised one-step operator, decay rates of the
  hydrodynamic modes (Sec. 2.1, nu = (1/omega - 1/2) theta,
  kappa = (d+2)/2 nu rho) and positivity ranges of r_i (Sec. 3.1).

Paper: J. W. Shim, "Parametric Lattice Boltzmann Method", arXiv:1402.5487.
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "plbm_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "libplbm_oracle.so")

MAXQ1 = 8
MAXQ = MAXQ1 * MAXQ1

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc, FP64, -ffp-contract=off, OpenMP)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
           "-fopenmp", "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class OrcLattice(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int),
        ("q1", ctypes.c_int),
        ("nx", ctypes.c_int),
        ("ny", ctypes.c_int),
        ("bc", ctypes.c_int),
        ("isothermal", ctypes.c_int),
        ("v", ctypes.c_int * MAXQ1),
        ("omega", ctypes.c_double),
        ("theta0", ctypes.c_double),
        ("C", ctypes.c_double * (MAXQ1 * MAXQ1)),
        ("ghost_left", ctypes.c_double * MAXQ),
        ("ghost_right", ctypes.c_double * MAXQ),
    ]


MAXQ1_3D = 5


class OrcLattice3(ctypes.Structure):
    _fields_ = [
        ("q1", ctypes.c_int),
        ("nx", ctypes.c_int),
        ("ny", ctypes.c_int),
        ("nz", ctypes.c_int),
        ("isothermal", ctypes.c_int),
        ("v", ctypes.c_int * MAXQ1_3D),
        ("omega", ctypes.c_double),
        ("theta0", ctypes.c_double),
        ("C", ctypes.c_double * (MAXQ1_3D * MAXQ1_3D)),
    ]


_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)
_LP = ctypes.POINTER(OrcLattice)
_LP3 = ctypes.POINTER(OrcLattice3)


def _load(path: str):
    L = ctypes.CDLL(path)
    L.orc_sizeof_lattice.restype = ctypes.c_int
    L.orc_vandermonde_inverse.argtypes = [ctypes.c_int, _D, _D]
    L.orc_vandermonde_inverse.restype = ctypes.c_int
    L.orc_mb_moments.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int, _D]
    L.orc_r1d.argtypes = [ctypes.c_int, _D, ctypes.c_double, ctypes.c_double, _D]
    L.orc_feq.argtypes = [ctypes.c_int, ctypes.c_int, _D, ctypes.c_double,
                          ctypes.c_double, ctypes.c_double, ctypes.c_double, _D]
    L.orc_node_moments.argtypes = [_LP, _D, _D, _D, _D, _D]
    L.orc_collide_node.argtypes = [_LP, _D, _D]
    L.orc_step.argtypes = [_LP, _D, _D]
    L.orc_run.argtypes = [_LP, _D, _D, ctypes.c_long]
    L.orc_init.argtypes = [_LP, _D, _D, _D, _D, _D]
    L.orc_moments.argtypes = [_LP, _D, _D, _D, _D, _D]
    L.orc_conserved.argtypes = [_LP, _D, _D]
    L.orc_set_threads.argtypes = [ctypes.c_int]
    L.orc_max_threads.restype = ctypes.c_int
    if L.orc_sizeof_lattice() != ctypes.sizeof(OrcLattice):
        raise RuntimeError("oracle lattice struct size mismatch")
    if hasattr(L, "orc3_sizeof_lattice"):
        L.orc3_sizeof_lattice.restype = ctypes.c_int
        L.orc3_feq.argtypes = [ctypes.c_int, _D, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                               ctypes.c_double, ctypes.c_double, _D]
        L.orc3_node_moments.argtypes = [_LP3, _D, _D]
        L.orc3_collide_node.argtypes = [_LP3, _D, _D]
        L.orc3_step.argtypes = [_LP3, _D, _D]
        L.orc3_run.argtypes = [_LP3, _D, _D, ctypes.c_long]
        L.orc3_init.argtypes = [_LP3, _D, _D, _D, _D, _D, _D]
        L.orc3_moments.argtypes = [_LP3, _D, _D]
        L.orc3_conserved.argtypes = [_LP3, _D, _D]
        if L.orc3_sizeof_lattice() != ctypes.sizeof(OrcLattice3):
            raise RuntimeError("oracle 3D lattice struct size mismatch")
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _load(build())
        return _lib


@contextlib.contextmanager
def using_library(path: str):
    """Temporarily route every oracle call through another build of plbm_oracle.c.

    Used only by the mutation tests, which compile deliberately broken copies of
    the oracle and check that the pins reject them.
    """
    global _lib
    lib()
    saved = _lib
    with _lock:
        _lib = _load(path)
    try:
        yield
    finally:
        with _lock:
            _lib = saved


def compile_variant(source_text: str, out_path: str) -> str:
    """Compile a modified copy of the oracle source with the oracle's own flags."""
    src = out_path + ".c"
    with open(src, "w") as fh:
        fh.write(source_text)
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                    "-fopenmp", "-shared", "-fPIC", src, "-o", out_path, "-lm"], check=True)
    return out_path


def source_text() -> str:
    with open(_SRC) as fh:
        return fh.read()


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_D)


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def max_threads() -> int:
    return int(lib().orc_max_threads())


# --------------------------------------------------------------------------
# Coefficients and equilibrium (Eq. eq:rdr, Appendix)
# --------------------------------------------------------------------------

def vandermonde_inverse(v) -> np.ndarray:
    """C = V^{-1}, V[n, k] = v_k^n (Appendix); C[i, n] multiplies mu_n in r_i."""
    v = np.ascontiguousarray(v, dtype=np.float64)
    q = v.size
    C = np.zeros(q * q)
    if lib().orc_vandermonde_inverse(q, _dp(v), _dp(C)) != 0:
        raise ValueError("singular Vandermonde matrix (repeated velocities)")
    return C.reshape(q, q)


def mb_moments(u: float, theta: float, nmax: int) -> np.ndarray:
    """mu_0..mu_nmax of the 1D Maxwell-Boltzmann distribution (mean u, variance theta)."""
    mu = np.zeros(nmax + 1)
    lib().orc_mb_moments(float(u), float(theta), int(nmax), _dp(mu))
    return mu


def r1d(v, u: float, theta: float, C: np.ndarray | None = None) -> np.ndarray:
    """Eq. (eq:rdr): r_i = sum_j c_ij mu_{j-1} for the 1D velocity set v."""
    if C is None:
        C = vandermonde_inverse(v)
    C = np.ascontiguousarray(C, dtype=np.float64)
    q1 = C.shape[0]
    r = np.zeros(q1)
    lib().orc_r1d(q1, _dp(C), float(u), float(theta), _dp(r))
    return r


def feq(dim: int, v, rho, ux, uy, theta) -> np.ndarray:
    """f^eq = rho r (1D) or rho r^x (x) r^y (2D, p = ix*q1 + iy)."""
    C = np.ascontiguousarray(vandermonde_inverse(v))
    q1 = C.shape[0]
    out = np.zeros(q1 ** dim)
    lib().orc_feq(int(dim), q1, _dp(C), float(rho), float(ux), float(uy),
                  float(theta), _dp(out))
    return out


# --------------------------------------------------------------------------
# Lattice state
# --------------------------------------------------------------------------

class Lattice:
    """A lattice description for the oracle (one instance, FP64).

    bc: ``"periodic"`` or ``"fixed"`` (fixed ends in x: ghost nodes hold
    f^eq(left_state) / f^eq(right_state), each state = (rho, u, theta)).
    """

    def __init__(self, dim, v, omega, nx, ny=1, bc="periodic", theta0=1.0,
                 isothermal=False, left_state=None, right_state=None):
        v = [int(a) for a in v]
        if dim not in (1, 2):
            raise ValueError("dim must be 1 or 2")
        if not 1 <= len(v) <= MAXQ1:
            raise ValueError("1 <= q1 <= 8")
        self.dim, self.v, self.q1 = dim, v, len(v)
        self.q = self.q1 ** dim
        self.nx, self.ny = int(nx), (int(ny) if dim == 2 else 1)
        self.omega, self.theta0 = float(omega), float(theta0)
        self.isothermal = bool(isothermal)
        self.bc = bc
        self.C = vandermonde_inverse(v)
        s = OrcLattice()
        s.dim, s.q1, s.nx, s.ny = dim, self.q1, self.nx, self.ny
        s.bc = 1 if bc == "fixed" else 0
        s.isothermal = 1 if isothermal else 0
        for i, a in enumerate(v):
            s.v[i] = a
        s.omega, s.theta0 = self.omega, self.theta0
        for i, c in enumerate(self.C.ravel()):
            s.C[i] = c
        if bc == "fixed":
            if left_state is None or right_state is None:
                raise ValueError("fixed ends need left_state and right_state")
            gl = self._ghost(left_state)
            gr = self._ghost(right_state)
            for p in range(self.q):
                s.ghost_left[p] = gl[p]
                s.ghost_right[p] = gr[p]
        elif bc != "periodic":
            raise ValueError("bc must be 'periodic' or 'fixed'")
        self.struct = s

    def _ghost(self, state):
        rho, u, theta = (float(a) for a in state)
        if self.isothermal:
            theta = self.theta0
        return feq(self.dim, self.v, rho, u, 0.0, theta)

    @property
    def shape(self):
        return (self.q, self.ny, self.nx)

    def velocities(self) -> np.ndarray:
        """(q, dim) integer velocity of every population."""
        if self.dim == 1:
            return np.array(self.v, dtype=np.int64).reshape(-1, 1)
        return np.array([(a, b) for a in self.v for b in self.v], dtype=np.int64)

    def ref(self):
        return ctypes.byref(self.struct)

    # -- state operations ---------------------------------------------------
    def init(self, rho, ux, uy=None, theta=None) -> np.ndarray:
        """f(x, 0) = f^eq(rho, u, theta) at every node (post-collision state)."""
        n = self.nx * self.ny
        rho = np.ascontiguousarray(np.broadcast_to(rho, (self.ny, self.nx)), dtype=np.float64)
        ux = np.ascontiguousarray(np.broadcast_to(ux, (self.ny, self.nx)), dtype=np.float64)
        uy = np.zeros(n) if uy is None else np.ascontiguousarray(
            np.broadcast_to(uy, (self.ny, self.nx)), dtype=np.float64)
        th = np.full(n, self.theta0) if theta is None else np.ascontiguousarray(
            np.broadcast_to(theta, (self.ny, self.nx)), dtype=np.float64)
        f = np.zeros(self.shape)
        lib().orc_init(self.ref(), _dp(rho), _dp(ux), _dp(uy), _dp(th), _dp(f))
        return f

    def step(self, f: np.ndarray) -> np.ndarray:
        f = np.ascontiguousarray(f, dtype=np.float64)
        out = np.empty_like(f)
        lib().orc_step(self.ref(), _dp(f), _dp(out))
        return out

    def run(self, f: np.ndarray, nsteps: int) -> np.ndarray:
        a = np.array(f, dtype=np.float64, order="C", copy=True)
        b = np.empty_like(a)
        lib().orc_run(self.ref(), _dp(a), _dp(b), int(nsteps))
        return a

    def moments(self, f: np.ndarray):
        """(rho, ux, uy, theta), each (ny, nx); uy is zero in 1D."""
        f = np.ascontiguousarray(f, dtype=np.float64)
        shp = (self.ny, self.nx)
        rho, ux, uy, th = (np.zeros(shp) for _ in range(4))
        lib().orc_moments(self.ref(), _dp(f), _dp(rho), _dp(ux), _dp(uy), _dp(th))
        return rho, ux, uy, th

    def conserved(self, f: np.ndarray) -> np.ndarray:
        """(sum f, sum v_x f, sum v_y f, sum |v|^2 f) in compensated FP64."""
        f = np.ascontiguousarray(f, dtype=np.float64)
        out = np.zeros(4)
        lib().orc_conserved(self.ref(), _dp(f), _dp(out))
        return out

    def collide_node(self, fin) -> np.ndarray:
        fin = np.ascontiguousarray(fin, dtype=np.float64)
        out = np.zeros(self.q)
        lib().orc_collide_node(self.ref(), _dp(fin), _dp(out))
        return out

    def node_moments(self, fin):
        fin = np.ascontiguousarray(fin, dtype=np.float64)
        r, a, b, t = (ctypes.c_double() for _ in range(4))
        lib().orc_node_moments(self.ref(), _dp(fin), ctypes.byref(r), ctypes.byref(a),
                               ctypes.byref(b), ctypes.byref(t))
        return r.value, a.value, b.value, t.value


class Lattice3:
    """A periodic three-dimensional lattice for the oracle (FP64), Sec. 2.1's
    tensor product of three 1D rules.  Population p = (ix*q1 + iy)*q1 + iz;
    arrays f[p][z][y][x]; fields [z][y][x]."""

    def __init__(self, v, omega, nx, ny, nz, theta0=1.0, isothermal=False):
        v = [int(a) for a in v]
        if not 1 <= len(v) <= MAXQ1_3D:
            raise ValueError("1 <= q1 <= 5 in 3D")
        self.dim, self.v, self.q1 = 3, v, len(v)
        self.q = self.q1 ** 3
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.omega, self.theta0 = float(omega), float(theta0)
        self.isothermal = bool(isothermal)
        self.C = vandermonde_inverse(v)
        s = OrcLattice3()
        s.q1, s.nx, s.ny, s.nz = self.q1, self.nx, self.ny, self.nz
        s.isothermal = 1 if isothermal else 0
        for i, a in enumerate(v):
            s.v[i] = a
        s.omega, s.theta0 = self.omega, self.theta0
        for i, c in enumerate(self.C.ravel()):
            s.C[i] = c
        self.struct = s

    @property
    def shape(self):
        return (self.q, self.nz, self.ny, self.nx)

    def velocities(self) -> np.ndarray:
        return np.array([(a, b, c) for a in self.v for b in self.v for c in self.v], dtype=np.int64)

    def ref(self):
        return ctypes.byref(self.struct)

    def _field(self, a, default):
        shp = (self.nz, self.ny, self.nx)
        if a is None:
            return np.full(shp, float(default))
        return np.ascontiguousarray(np.broadcast_to(a, shp), dtype=np.float64)

    def feq(self, rho, ux, uy, uz, theta) -> np.ndarray:
        C = np.ascontiguousarray(self.C)
        out = np.zeros(self.q)
        lib().orc3_feq(self.q1, _dp(C), float(rho), float(ux), float(uy), float(uz), float(theta), _dp(out))
        return out

    def init(self, rho, ux=None, uy=None, uz=None, theta=None) -> np.ndarray:
        f = np.zeros(self.shape)
        lib().orc3_init(self.ref(), _dp(self._field(rho, 1.0)), _dp(self._field(ux, 0.0)),
                        _dp(self._field(uy, 0.0)), _dp(self._field(uz, 0.0)),
                        _dp(self._field(theta, self.theta0)), _dp(f))
        return f

    def step(self, f: np.ndarray) -> np.ndarray:
        f = np.ascontiguousarray(f, dtype=np.float64)
        out = np.empty_like(f)
        lib().orc3_step(self.ref(), _dp(f), _dp(out))
        return out

    def run(self, f: np.ndarray, nsteps: int) -> np.ndarray:
        a = np.array(f, dtype=np.float64, order="C", copy=True)
        b = np.empty_like(a)
        lib().orc3_run(self.ref(), _dp(a), _dp(b), int(nsteps))
        return a

    def moments(self, f: np.ndarray):
        """(rho, ux, uy, uz, theta), each [z][y][x]."""
        f = np.ascontiguousarray(f, dtype=np.float64)
        out = np.zeros((5, self.nz, self.ny, self.nx))
        lib().orc3_moments(self.ref(), _dp(f), _dp(out))
        return tuple(out)

    def conserved(self, f: np.ndarray) -> np.ndarray:
        """(sum f, sum v_x f, sum v_y f, sum v_z f, sum |v|^2 f), compensated FP64."""
        f = np.ascontiguousarray(f, dtype=np.float64)
        out = np.zeros(5)
        lib().orc3_conserved(self.ref(), _dp(f), _dp(out))
        return out

    def collide_node(self, fin) -> np.ndarray:
        fin = np.ascontiguousarray(fin, dtype=np.float64)
        out = np.zeros(self.q)
        lib().orc3_collide_node(self.ref(), _dp(fin), _dp(out))
        return out

    def node_moments(self, fin):
        fin = np.ascontiguousarray(fin, dtype=np.float64)
        m = np.zeros(5)
        lib().orc3_node_moments(self.ref(), _dp(fin), _dp(m))
        return tuple(m)


def rel_err(a, b) -> float:
    """max|a - b| / max|b| over all entries."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.max(np.abs(b))
    return float(np.max(np.abs(a - b)) / (den if den > 0 else 1.0))


def rel_err_vec(ax, ay, bx, by) -> float:
    """Vector relative error max|u_a - u_b| / max|u_b| (velocity fields)."""
    d = np.hypot(np.asarray(ax) - bx, np.asarray(ay) - by)
    den = np.max(np.hypot(bx, by))
    return float(np.max(d) / (den if den > 0 else 1.0))
