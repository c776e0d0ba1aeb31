"""The angular spread's table (Eqs. (5)-(6)) as the library builds it on the
host, against the oracle's exact inverse CDF, without a GPU.

The library tabulates y = psi / (v s(x)) over ln x and v = sqrt(-ln(1 - u)).
It builds the table from its own Bessel functions (Gauss-Legendre) and its
own cumulative.  The oracle inverts the CDF of the density directly.  The
step kernels read the table by bilinear interpolation in float32.  This
test repeats that lookup in numpy float32 on 2e4 random (x, u) pairs and
on the extreme words.  Inside the table's x range psi must agree within
5e-4; the GPU test checks the kernels' own lookup to the same bar.
"""
import math

import numpy as np
import pytest

import oracle as O

f32 = np.float32


@pytest.fixture(scope="module")
def table():
    from paper_1409_5574_gb300 import build, prad
    build.build()
    return prad, prad.prad_angle_table()


def _lookup(prad, T, x, w0, w1):
    NL, NV = prad.PRAD_ANG_NL, prad.PRAD_ANG_NV
    lx0, lx1, vmax = prad.PRAD_ANG_LX0, prad.PRAD_ANG_LX1, prad.PRAD_ANG_VMAX
    xf = x.astype(f32)
    lx = np.log(xf)
    fi = np.clip((lx - f32(lx0)) * f32((NL - 1) / (lx1 - lx0)), 0, NL - 1).astype(f32)
    i = np.minimum(fi.astype(np.int64), NL - 2)
    ti = fi - i.astype(f32)
    lo = w0 < 0x80000000
    u = (w0.astype(f32) * f32(2.0 ** -32) + f32(2.0 ** -33)).astype(f32)
    om = ((~w0).astype(np.uint32).astype(f32) * f32(2.0 ** -32) + f32(2.0 ** -33)).astype(f32)
    with np.errstate(divide="ignore"):
        w = np.where(lo, -np.log1p(-np.where(lo, u, f32(0))), -np.log(om)).astype(f32)
    v = np.sqrt(np.maximum(w, 0)).astype(f32)
    fj = np.minimum(v * f32((NV - 1) / vmax), f32(NV - 1))
    j = np.minimum(fj.astype(np.int64), NV - 2)
    tj = fj - j.astype(f32)
    y0 = T[i, j] + tj * (T[i, j + 1] - T[i, j])
    y1 = T[i + 1, j] + tj * (T[i + 1, j + 1] - T[i + 1, j])
    y = y0 + ti * (y1 - y0)
    sc = np.exp((f32(0.693147181) - lx) / f32(3) - np.log1p(xf) / f32(6))
    p = (y * v * sc).astype(np.float64)
    return np.where(w1 & 0x80000000, -p, p)


def test_table_shape_and_first_column(table):
    prad, T = table
    assert T.shape == (prad.PRAD_ANG_NL, prad.PRAD_ANG_NV)
    assert np.all(T[:, 0] == 0) and np.all(np.isfinite(T)) and np.all(T[:, 1:] > 0)


def test_table_lookup_matches_the_oracle_inverse_cdf(table):
    prad, T = table
    rng = np.random.default_rng(7)
    n = 20000
    x = np.exp(rng.uniform(math.log(1e-8), math.log(40.0), n)).astype(f32).astype(np.float64)
    w0 = rng.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32)
    w0[:8] = [0, 1, 2 ** 31 - 1, 2 ** 31, 2 ** 32 - 1, 2 ** 32 - 2, 1000, 2 ** 32 - 1000]
    w1 = rng.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32)
    got = _lookup(prad, T, x, w0, w1)
    ref = O.ang_sample(x, (w0.astype(np.float64) + 0.5) * 2.0 ** -32)
    ref = np.where(w1 & 0x80000000, -ref, ref)
    rel = np.abs(got / ref - 1.0)
    assert rel.max() < 5e-4 and np.median(rel) < 1e-4, (rel.max(), np.median(rel))


def test_table_needs_room(table):
    prad, _ = table
    import ctypes
    buf = np.empty(10, dtype=np.float32)
    rc = prad.load_library().prad_angle_table(buf.ctypes.data_as(ctypes.c_void_p), buf.size)
    assert rc == prad.PRAD_ERR_ARG
