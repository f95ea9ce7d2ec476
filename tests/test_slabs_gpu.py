"""Domain decomposition along y on the GPU (plbm_slabs_*): the decomposed lattice
equals the undivided one bit for bit.

The slabs exchange the halo populations of plbm_halo_plan with one device
copy launch per step and step as ordinary handles; Eq. (eq:srt) pulls from at
most max|v| = 3 rows, so every own row sees exactly the values of the undivided
lattice.  Cases: FP32 and FP16 storage on row pairs (even ny; the slabs take
even row counts), FP32 on the plain layout (odd ny) and FP64; 1 to 4 slabs, row
counts not divisible by the slab count; an odd number of steps (graph replays
of step pairs plus one single step).
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


@pytest.mark.parametrize("prec,nx,ny,nslabs", [("f32", 96, 74, 3), ("f32", 64, 62, 1), ("f16dev", 80, 70, 4),
                                               ("f32", 70, 53, 4), ("f64", 48, 41, 2)])
def test_decomposed_lattice_equals_the_undivided_one(prec, nx, ny, nslabs):
    fields = I.kh_fields(nx, ny=ny)
    one = plbm.Solver(2, V5, 1.3, nx, ny, theta0=1.0, prec=prec)
    one.init(*fields)
    one.step(41)
    ref_f, ref_m = one.get_populations(), one.moments()
    one.close()
    sl = plbm.Slabs(V5, 1.3, nx, ny, nslabs, theta0=1.0, prec=prec)
    rows = [sl.slab(k)[2] for k in range(nslabs)]
    assert sum(rows) == ny
    if prec != "f64" and ny % 2 == 0:
        assert all(r % 2 == 0 for r in rows)
    sl.init(*fields)
    sl.step(40)
    sl.step(1)
    assert np.array_equal(sl.get_populations(), ref_f)
    for a, b in zip(sl.moments(), ref_m):
        assert np.array_equal(a, b)
    sl.close()


def test_slab_errors():
    with pytest.raises(plbm.PlbmError):
        plbm.Slabs(V5, 1.3, 32, 10, 4)          # 4 slabs of 10 rows: fewer than 3 rows each
    with pytest.raises(plbm.PlbmError):
        plbm.Slabs(V5, 1.3, 32, 32, 0)


def test_bench_decomposition_2048_equals_the_undivided_lattice():
    # The bench variant: 2048^2 FP32 in four slabs of 512 rows.
    L = 2048
    fields = I.kh_fields(L)
    one = plbm.Solver(2, V5, 1.3, L, L, theta0=1.0, prec="f32")
    one.init(*fields)
    one.step(7)
    ref = one.get_populations()
    one.close()
    sl = plbm.Slabs(V5, 1.3, L, L, 4, theta0=1.0, prec="f32")
    assert [sl.slab(k)[2] for k in range(4)] == [512] * 4
    sl.init(*fields)
    sl.step(7)
    assert np.array_equal(sl.get_populations(), ref)
    sl.close()
