"""Long-horizon FP64 oracle snapshots of the Kelvin-Helmholtz double shear layer.

TEST INFRASTRUCTURE ONLY (part of the oracle package; calls nothing but the
oracle and the seeded input generator).  Runs the plain FP64 oracle on the
D2Q25 {0, +-1, +-3}^2 double shear layer (periodic, theta0 = 1, omega = 1.3,
seed 0, Sec. 3.2 / Sec. 4 shear-layer runs) and writes the macroscopic
fields rho, u_x, u_y, theta at the requested step counts to an ``.npz`` file.
Fields of lattices larger than 512 x 512 are stored on the sub-lattice of
every ``stride``-th node in x and y (nodes (stride*i, stride*j)), which keeps
a 2048 x 2048 run at 512 x 512 values per field.

Usage:
    python -m oracle.kh_longrun --size 2048 --steps 1000 10000 20000 --stride 4 --out kh2048.npz
"""
from __future__ import annotations

import argparse
import os
import time

import numpy as np


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--size", type=int, default=2048)
    ap.add_argument("--steps", type=int, nargs="+", default=[1000, 10000, 20000])
    ap.add_argument("--stride", type=int, default=None)
    ap.add_argument("--omega", type=float, default=1.3)
    ap.add_argument("--theta0", type=float, default=1.0)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--out", required=True)
    a = ap.parse_args(argv)

    import oracle as O
    from paper_1402_5487_gb300 import inputs as I

    L = a.size
    stride = a.stride if a.stride is not None else max(1, L // 512)
    rho, ux, uy, th = I.kh_fields(L, theta0=a.theta0, seed=a.seed)
    lat = O.Lattice(2, I.SET_013, a.omega, L, L, theta0=a.theta0)
    f = lat.init(rho, ux, uy, th)
    done = 0
    out = {"size": L, "stride": stride, "omega": a.omega, "theta0": a.theta0, "seed": a.seed,
           "velocities": np.array(I.SET_013), "steps": np.array(sorted(a.steps))}
    t0 = time.time()
    for n in sorted(a.steps):
        f = lat.run(f, n - done)
        done = n
        m = lat.moments(f)
        for name, field in zip(("rho", "ux", "uy", "theta"), m):
            out[f"{name}_{n}"] = np.ascontiguousarray(field[::stride, ::stride])
        print(f"step {n}: {time.time() - t0:.0f} s", flush=True)
        tmp = a.out + ".tmp.npz"
        np.savez(tmp, **out)
        os.replace(tmp, a.out)


if __name__ == "__main__":
    main()
