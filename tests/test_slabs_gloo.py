"""Domain decomposition along y with a real exchange between processes (CPU, gloo).

Each of N gloo ranks owns the rows the library's plbm_slab_rows gives it, plus
w = plbm_halo_width rows on each side.  Every step the ranks send each other the
halo populations that plbm_halo_plan names (populations moving up for the rows
above a slab's lower neighbour, moving down for the rows below its upper one),
as host tensors through torch.distributed, and then advance their padded slab
with the FP64 oracle (a periodic lattice of rows + 2w rows: the slab's own rows
pull only from rows that are either its own or freshly exchanged).  After 100
steps rank 0 gathers the own rows, which must equal the undivided oracle run
bit for bit: the pull of Eq. (eq:srt) reaches at most w rows and the collision
is local, so each node sees exactly the values it would see undivided.

ny = 37 is not divisible by 2 or 4, so the slabs have different row counts.
A plan that names a wrong population, row or neighbour changes the result.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
V5 = (0, 1, -1, 3, -3)
NX, NY, OMEGA, STEPS = 23, 37, 1.3, 100


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import oracle as O
    from paper_1402_5487_gb300 import inputs as I, plbm
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        O.set_threads(1)
        w = plbm.halo_width(V5)
        y0, rows = plbm.slab_rows(NY, world, rank)
        lo_pops = plbm.halo_plan(V5, -1)   # the rows below need populations moving up
        hi_pops = plbm.halo_plan(V5, +1)   # the rows above need populations moving down
        up, down = (rank + 1) % world, (rank - 1) % world
        fields = I.kh_fields(NX, ny=NY)
        pad = [(y0 - w + j) % NY for j in range(rows + 2 * w)]
        lat = O.Lattice(2, V5, OMEGA, NX, rows + 2 * w, theta0=1.0)
        f = lat.init(*[np.ascontiguousarray(a[pad]) for a in fields])
        for _ in range(STEPS):
            # my last w own rows go up (they are the lower halo of the slab above);
            # my first w own rows go down (the upper halo of the slab below)
            send_up = torch.from_numpy(np.ascontiguousarray(f[lo_pops, rows:rows + w]))
            send_down = torch.from_numpy(np.ascontiguousarray(f[hi_pops, w:2 * w]))
            recv_lo = torch.empty_like(send_up)
            recv_hi = torch.empty_like(send_down)
            reqs = [dist.isend(send_up, up, tag=0), dist.isend(send_down, down, tag=1),
                    dist.irecv(recv_lo, down, tag=0), dist.irecv(recv_hi, up, tag=1)]
            for r in reqs:
                r.wait()
            f[lo_pops, 0:w] = recv_lo.numpy()
            f[hi_pops, rows + w:rows + 2 * w] = recv_hi.numpy()
            f = lat.step(f)
        own = torch.from_numpy(np.ascontiguousarray(f[:, w:w + rows]))
        if rank == 0:
            parts = [own]
            for k in range(1, world):
                _, rk = plbm.slab_rows(NY, world, k)
                buf = torch.empty((f.shape[0], rk, NX), dtype=torch.float64)
                dist.recv(buf, k)
                parts.append(buf)
            out["f"] = torch.cat(parts, dim=1).numpy()
        else:
            dist.send(own, 0)
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(300)
@pytest.mark.parametrize("world", [2, 4])
def test_gloo_slabs_equal_the_undivided_oracle(world):
    import oracle as O
    from paper_1402_5487_gb300 import build, inputs as I
    build.build()
    O.build()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        got = out["f"]
    lat = O.Lattice(2, V5, OMEGA, NX, NY, theta0=1.0)
    ref = lat.run(lat.init(*I.kh_fields(NX, ny=NY)), STEPS)
    assert np.array_equal(got, ref)


def test_partition_and_plan():
    from paper_1402_5487_gb300 import build, plbm
    build.build()
    for ny, n in ((37, 4), (2048, 3), (10, 1), (9, 3)):
        parts = [plbm.slab_rows(ny, n, k) for k in range(n)]
        assert parts[0][0] == 0 and sum(r for _, r in parts) == ny
        assert all(parts[k][0] + parts[k][1] == parts[k + 1][0] for k in range(n - 1))
        assert max(r for _, r in parts) - min(r for _, r in parts) <= 1
    assert plbm.halo_width(V5) == 3 and plbm.halo_width((0, 2, -4)) == 4
    lo, hi = plbm.halo_plan(V5, -1), plbm.halo_plan(V5, 1)
    assert lo == [i * 5 + j for i in range(5) for j in (1, 3)]     # v_y = +1, +3
    assert hi == [i * 5 + j for i in range(5) for j in (2, 4)]     # v_y = -1, -3
    with pytest.raises(plbm.PlbmError):
        plbm.slab_rows(3, 4, 0)
