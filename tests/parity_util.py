"""Helpers shared by the GPU parity tests: run one workload on the CUDA path
(through the C ABI) and on the oracle, from the same seeded host inputs."""
import numpy as np

import oracle as O


def rel(a, b):
    return O.rel_err(a, b)


def field_errors(gpu, ref):
    """Per-field relative errors (R14 reading): max|a-b|/max|b| for rho and theta,
    vector norm for the velocity, and the same for populations if given."""
    (gr, gx, gy, gt), (rr, rx, ry, rt) = gpu, ref
    return {
        "rho": O.rel_err(gr, rr),
        "u": O.rel_err_vec(gx, gy, rx, ry),
        "theta": O.rel_err(gt, rt),
    }


def oracle_run(dim, v, omega, nx, ny, fields, steps, theta0=1.0, bc="periodic", left=None,
               right=None, isothermal=False, threads=None):
    if threads:
        O.set_threads(threads)
    lat = O.Lattice(dim, v, omega, nx, ny, bc=bc, theta0=theta0, isothermal=isothermal,
                    left_state=left, right_state=right)
    f = lat.init(*fields)
    f = lat.run(f, steps)
    return lat, f, lat.moments(f)


def gpu_run(dim, v, omega, nx, ny, fields, steps, prec="f64", theta0=1.0, bc="periodic", left=None,
            right=None, isothermal=False, chunks=1):
    from paper_1402_5487_gb300 import plbm
    s = plbm.Solver(dim, v, omega, nx, ny, theta0=theta0, prec=prec, bc=bc, left_state=left,
                    right_state=right, isothermal=isothermal)
    rho, ux, uy, th = fields
    s.init(rho, ux, uy if dim == 2 else None, None if isothermal else th)
    per = steps // chunks
    done = 0
    for c in range(chunks):
        k = per if c < chunks - 1 else steps - done
        s.step(k)
        done += k
    out = s.moments(), s.get_populations(), s
    return out


def patch_fields(fields, cx, cy, half, nx, ny):
    """Periodic window of side 2*half+1 centred on (cx, cy) of each [ny][nx] field."""
    xs = (np.arange(cx - half, cx + half + 1)) % nx
    ys = (np.arange(cy - half, cy + half + 1)) % ny
    return tuple(np.ascontiguousarray(a[np.ix_(ys, xs)]) for a in fields)
