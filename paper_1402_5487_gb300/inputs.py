"""Seeded synthetic inputs shared by the CUDA path's tests/benchmark and the oracle.

This module holds initial fields and parameter draws only: no part of the
lattice Boltzmann arithmetic.  Every field is computed on the host in FP64 and
handed unchanged to both sides.

Workloads (lattice units, dx = dt = 1):

* Thermal shock tube (Sec. 4, Fig. 5v): D1Q5, velocities {0, +-1, +-3},
  1000 nodes, fixed ends, discontinuity between nodes 499 and 500.
* Kelvin-Helmholtz double shear layer (Sec. 3.2 and Sec. 4 shear-layer runs):
  u_x = u0 tanh((|y - L/2| - L/4) / delta), delta = L/80,
  u_y = eps sin(2 pi x / L), plus uniform noise in [-1e-4, 1e-4] on both
  components drawn from numpy's PCG64 (u_x then u_y, row-major), rho = 1,
  theta = theta0.  Node (i, j) sits at x = i, y = j.
* Shear wave: u_x = A sin(2 pi y / L), rho = 1, theta = theta0.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Velocity sets used by the workloads (integers, lattice units).
SET_013 = (0, 1, -1, 3, -3)
SET_012 = (0, 1, -1, 2, -2)
SET_023 = (0, 2, -2, 3, -3)
SET_D1Q3 = (0, 1, -1)


def kh_fields(L: int, theta0: float = 1.0, seed: int = 0, u0: float = 0.1,
              delta: float | None = None, eps: float = 0.005, noise: float = 1e-4,
              ny: int | None = None):
    """Double shear layer on an L x ny periodic grid; returns (rho, ux, uy, theta)."""
    nx = int(L)
    ny = nx if ny is None else int(ny)
    delta = (ny / 80.0) if delta is None else float(delta)
    y = np.arange(ny, dtype=np.float64)[:, None]
    x = np.arange(nx, dtype=np.float64)[None, :]
    ux = u0 * np.tanh((np.abs(y - ny / 2.0) - ny / 4.0) / delta) * np.ones((1, nx))
    uy = eps * np.sin(2.0 * np.pi * x / nx) * np.ones((ny, 1))
    if noise:
        rng = np.random.default_rng(seed)
        ux = ux + rng.uniform(-noise, noise, size=(ny, nx))
        uy = uy + rng.uniform(-noise, noise, size=(ny, nx))
    rho = np.ones((ny, nx))
    theta = np.full((ny, nx), float(theta0))
    return rho, np.ascontiguousarray(ux), np.ascontiguousarray(uy), theta


def paper_kh_fields(L: int = 128, a: float = 1.6, u0: float = 0.069, l0: float = 80.0, eps: float = 0.05,
                    theta0: float | None = None):
    """The paper's shear-layer initial condition (Sec. 4, 25-velocity model) in
    lattice units.  The paper's set {0, +-a, +-2a} sqrt(theta0) in units where the
    temperature is 1 is the lattice set {0, +-1, +-2} with theta0 = 1 / a^2, and
    its velocities scale by sqrt(theta0).  Domain [0, 1)^2 on L x L nodes, node
    (i, j) at (x, y) = (i / L, j / L):
    u_x = u0 tanh(l0 (y - 1/4)) for y <= 1/2, u0 tanh(l0 (3/4 - y)) otherwise;
    u_y = u0 eps sin(2 pi (x + 1/4)); rho = 1, theta = theta0.
    theta0 (optional) replaces 1 / a^2: the three-velocity models of Sec. 4 use
    {0, +-1} = {0, +-sqrt(zeta theta0)}, theta0 = 1 / zeta.
    Returns ((rho, ux, uy, theta) [L][L], theta0)."""
    theta0 = 1.0 / (a * a) if theta0 is None else float(theta0)
    s = math.sqrt(theta0)
    x = np.arange(L) / L
    y = np.arange(L) / L
    prof = np.where(y <= 0.5, np.tanh(l0 * (y - 0.25)), np.tanh(l0 * (0.75 - y)))
    ux = np.broadcast_to((u0 * s * prof)[:, None], (L, L))
    uy = np.broadcast_to((u0 * eps * s * np.sin(2 * np.pi * (x + 0.25)))[None, :], (L, L))
    one = np.ones((L, L))
    return tuple(np.ascontiguousarray(f) for f in (one, ux, uy, theta0 * one)), theta0


def taylor_green_fields(N: int, U: float, theta0: float):
    """Decaying Taylor-Green vortex on [0, 1)^2, node (i, j) at (i / N, j / N):
    u_x = U sin(2 pi x) cos(2 pi y), u_y = -U cos(2 pi x) sin(2 pi y),
    rho = 1 - U^2 / (4 theta0) (cos 4 pi x + cos 4 pi y) (the pressure of the
    incompressible solution over rho theta0), theta = theta0; fields [N][N]."""
    x = np.arange(N) / N
    X, Y = np.meshgrid(x, x, indexing="xy")
    k = 2 * np.pi
    ux = U * np.sin(k * X) * np.cos(k * Y)
    uy = -U * np.cos(k * X) * np.sin(k * Y)
    rho = 1 - (U * U / (4 * theta0)) * (np.cos(2 * k * X) + np.cos(2 * k * Y))
    return tuple(np.ascontiguousarray(f) for f in (rho, ux, uy, theta0 * np.ones((N, N))))


def kh3_fields(nx: int, ny: int, nz: int, u0: float = 0.1, theta0: float = 1.0, seed: int = 0):
    """Three-dimensional double shear layer (the 2D KH workload extended along y),
    fields [nz][ny][nx] in the order (rho, u_x, u_y, u_z, theta):
    u_x = u0 tanh((|z - nz/2| - nz/4) / delta), delta = nz / 16,
    u_z = 0.005 sin(2 pi x / nx), uniform noise in [-1e-4, 1e-4] on u_x then u_z
    (numpy default_rng(seed), C order), rho = 1, theta = theta0, u_y = 0."""
    rng = np.random.default_rng(seed)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ux = u0 * np.tanh((np.abs(z - nz / 2) - nz / 4) / (nz / 16))
    uz = 0.005 * np.sin(2 * np.pi * x / nx)
    ux = ux + rng.uniform(-1e-4, 1e-4, ux.shape)
    uz = uz + rng.uniform(-1e-4, 1e-4, uz.shape)
    one = np.ones_like(ux)
    return tuple(np.ascontiguousarray(a) for a in (one, ux, 0.0 * one, uz, theta0 * one))


def shear_wave_fields(L: int, theta0: float, amp: float = 1e-3, ny: int | None = None,
                      ux0: float = 0.0):
    """u_x = ux0 + amp sin(2 pi y / ny), rho = 1, u_y = 0, theta = theta0."""
    nx = int(L)
    ny = nx if ny is None else int(ny)
    y = np.arange(ny, dtype=np.float64)[:, None]
    ux = ux0 + amp * np.sin(2.0 * np.pi * y / ny) * np.ones((1, nx))
    return (np.ones((ny, nx)), np.ascontiguousarray(ux), np.zeros((ny, nx)),
            np.full((ny, nx), float(theta0)))


def shock_tube_fields(n: int = 1000, left=(1.1, 0.0, 0.5), right=(1.0, 0.0, 0.5),
                      x0: int | None = None):
    """Riemann initial data on n nodes: nodes x < x0 take `left`, the rest `right`.

    Each state is (rho, u, theta).  Returns 1 x n arrays (rho, ux, uy, theta).
    """
    x0 = n // 2 if x0 is None else int(x0)
    x = np.arange(n)
    sel = x < x0
    rho = np.where(sel, left[0], right[0]).astype(np.float64)[None, :]
    ux = np.where(sel, left[1], right[1]).astype(np.float64)[None, :]
    th = np.where(sel, left[2], right[2]).astype(np.float64)[None, :]
    return rho, ux, np.zeros_like(ux), th


@dataclass
class Instance:
    """One member of the batched sweep (a candidate before any admissibility gate)."""
    index: int
    L: int
    v: tuple
    omega: float
    theta0: float
    kind: str            # "kh" or "shear"
    seed: int
    fields: tuple = field(default=(), repr=False)
    prec: str | None = None      # storage precision; None: the batch's
    isothermal: bool = False     # theta in f^eq held at theta0 (Eq. eq:1d3v models)


def batch_candidates(n: int = 256, seed: int = 1000, size_lo: int = 64, size_hi: int = 1024,
                     sets=(SET_012, SET_013, SET_023), omega=(1.0, 1.9), theta=(0.6, 1.2),
                     max_draws: int = 64):
    """Seeded parameter draws for the batched sweep.

    Instance k uses ``default_rng(seed + k)``: side L uniform over the integers of
    [size_lo, size_hi] (odd and even alike), then up to ``max_draws`` candidate
    (set, omega, theta) triples; the caller
    keeps the first one that its admissibility gate accepts.  Even k are
    Kelvin-Helmholtz layers, odd k shear waves.
    Returns a list of (index, L, kind, [(v, omega, theta), ...]).
    """
    out = []
    for k in range(n):
        rng = np.random.default_rng(seed + k)
        L = int(rng.integers(size_lo, size_hi + 1))
        cands = []
        for _ in range(max_draws):
            v = sets[int(rng.integers(0, len(sets)))]
            om = float(rng.uniform(*omega))
            th = float(rng.uniform(*theta))
            cands.append((tuple(v), om, th))
        out.append((k, L, "kh" if k % 2 == 0 else "shear", cands))
    return out


def instance_fields(inst: Instance):
    """Initial fields of one batched instance (KH with noise seed = inst.seed, or a shear wave)."""
    if inst.kind == "kh":
        return kh_fields(inst.L, theta0=inst.theta0, seed=inst.seed)
    return shear_wave_fields(inst.L, theta0=inst.theta0, amp=1e-3)
