"""Pins of the oracle's special functions against things other than itself.

Philox4x32-10 against the CUDA toolkit's curand host generator (a library run
on the CPU); F(x) of Eq. (8) against scipy's Bessel K and quadrature and the
closed-form Mellin moments of F; the proposal S of Eq. (11) and its CDF of
Eq. (12) against their closed forms; the uniform mapping at its extremes.
"""
import ctypes
import ctypes.util
import math

import numpy as np
import pytest

import oracle as O

scipy = pytest.importorskip("scipy")
from scipy import integrate, optimize, special, stats  # noqa: E402


# ---------------------------------------------------------------- Philox
def _curand():
    for name in ("libcurand.so", "libcurand.so.10",
                 "/usr/local/cuda/lib64/libcurand.so"):
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    return None


def _curand_blocks(lib, seed: int, offset_blocks: int, nblocks: int):
    gen = ctypes.c_void_p()
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), 161) == 0  # PHILOX4_32_10
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        assert lib.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(4 * offset_blocks)) == 0
        out = np.zeros(4 * nblocks, dtype=np.uint32)
        assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p),
                                  ctypes.c_size_t(out.size)) == 0
    finally:
        lib.curandDestroyGenerator(gen)
    return out.reshape(nblocks, 4)


@pytest.mark.parametrize("seed", [0, 1, 0x123456789ABCDEF0, 2**64 - 1])
def test_philox_matches_curand_host_generator(seed):
    """curand's host Philox4_32_10 stream: block b is ctr (0, 0, b, 0) under
    key (seed_lo, seed_hi) (layout found empirically). This pins the round
    function, the key schedule and word c2 for arbitrary keys."""
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not available")
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for off in (0, 4097, 12345):
        got = _curand_blocks(lib, seed, off, 8)
        ctr = np.array([[0, 0, (off + b) & 0xFFFFFFFF, 0] for b in range(8)],
                       dtype=np.uint32)
        np.testing.assert_array_equal(O.philox(ctr, key), got)


def test_philox_counter_words_all_matter():
    """Each counter word and each key word changes every output word."""
    base = O.philox([1, 2, 3, 4], [5, 6])[0]
    for k in range(4):
        c = [1, 2, 3, 4]
        c[k] ^= 1
        assert np.all(O.philox(c, [5, 6])[0] != base)
    for k in range(2):
        kk = [5, 6]
        kk[k] ^= 1
        assert np.all(O.philox([1, 2, 3, 4], kk)[0] != base)


def test_philox_uniformity():
    """Chi-square of the top byte over 2^14 consecutive counters."""
    ctr = np.zeros((1 << 14, 4), dtype=np.uint32)
    ctr[:, 0] = np.arange(1 << 14)
    ctr[:, 1] = 77
    out = O.philox(ctr, [1, 0])
    hist = np.bincount((out.ravel() >> 24).astype(np.int64), minlength=256)
    _, p = stats.chisquare(hist)
    assert p > 1e-4


# ---------------------------------------------------------------- F(x)
def _F_scipy(x):
    """x int_x^inf K_5/3, with scipy's kv, integrated in ln y (K_5/3(y) is
    below 1e-40 beyond y = 100)."""
    f = lambda s: special.kv(5.0 / 3.0, math.exp(s)) * math.exp(s)
    val, _ = integrate.quad(f, math.log(x), math.log(100.0), epsabs=0,
                            epsrel=1e-13, limit=500)
    return x * val


@pytest.mark.parametrize("x", [1e-6, 1e-3, 0.01, 0.1, 0.29, 1.0, 3.0, 10.0, 30.0])
def test_F_exact_vs_scipy_bessel(x):
    assert O.F_exact([x])[0] == pytest.approx(_F_scipy(x), rel=1e-9)


def test_F_mellin_moments():
    """int_0^inf F = 8 pi/(9 sqrt 3) (the normalisation stated with Eq. (10))
    and int_0^inf F/x = 5 pi/3, integrated here by scipy over F_exact."""
    f = lambda t: O.F_exact([t])[0]
    i1 = sum(integrate.quad(f, a, b, epsrel=1e-12, limit=400)[0]
             for a, b in ((0, 1e-6), (1e-6, 1e-2), (1e-2, 1), (1, 10), (10, 80)))
    assert i1 == pytest.approx(8 * math.pi / (9 * math.sqrt(3)), rel=1e-9)
    g = lambda y: O.F_exact([math.exp(y)])[0]       # int F/x dx = int F(e^y) dy
    i0 = integrate.quad(g, math.log(1e-14), math.log(80), epsrel=1e-12, limit=400)[0]
    c = 4 * math.pi / (math.sqrt(3) * math.gamma(1 / 3)) * 2 ** (-1 / 3)
    i0 += 3 * c * (1e-14) ** (1 / 3)                # exact tail below 1e-14
    assert i0 == pytest.approx(5 * math.pi / 3, rel=1e-9)
    # the oracle's own cumulative tables agree
    assert O.int_F(80.0) == pytest.approx(8 * math.pi / (9 * math.sqrt(3)), rel=1e-10)
    assert O.int_F_over_x(80.0) == pytest.approx(5 * math.pi / 3, rel=1e-10)


def test_F_asymptotes_and_maximum():
    c = 4 * math.pi / (math.sqrt(3) * math.gamma(1 / 3)) * 2 ** (-1 / 3)
    assert c == pytest.approx(2.1495282415, rel=1e-9)
    x = 1e-12
    assert O.F_exact([x])[0] / (c * x ** (1 / 3)) == pytest.approx(1.0, abs=1e-6)
    x = 40.0
    lead = math.sqrt(math.pi * x / 2) * math.exp(-x)
    assert O.F_exact([x])[0] / lead == pytest.approx(1 + 55 / (72 * x), rel=2e-3)
    res = optimize.minimize_scalar(lambda t: -O.F_exact([t])[0],
                                   bounds=(0.1, 0.6), method="bounded",
                                   options={"xatol": 1e-8})
    assert res.x == pytest.approx(0.2858, abs=2e-3)
    assert -res.fun == pytest.approx(0.9180, abs=5e-4)


def test_F_interpolant_vs_quadrature():
    rng = np.random.default_rng(3)
    x = np.exp(rng.uniform(math.log(1e-16), math.log(45.0), 4000))
    rel = np.abs(O.F(x) / O.F_exact(x) - 1.0)
    assert rel.max() < 1e-9


# ---------------------------------------------------------------- S, P
def test_proposal_constant_a():
    a = O.const_a()
    assert abs(a ** (4 / 3) + 7 / 9 * math.exp(-a) - 1) < 1e-15
    assert a == pytest.approx(0.69021, abs=5e-6)      # printed with Eq. (11)
    # the rounded value leaves int S - 1 ~ 2.6e-6
    ar = 0.69021
    assert abs(ar ** (4 / 3) + 7 / 9 * math.exp(-ar) - 1) > 1e-6


def test_S_normalised_and_P_consistent():
    a = O.const_a()
    i = (integrate.quad(O.S, 0, a, epsrel=1e-14)[0]
         + integrate.quad(O.S, a, 60, epsrel=1e-14)[0] + 7 / 9 * math.exp(-60))
    assert i == pytest.approx(1.0, abs=1e-12)
    for x in (1e-9, 0.1, a * (1 - 1e-12), a, 1.0, 5.0, 40.0):
        ref = integrate.quad(O.S, 0, min(x, a), epsrel=1e-14)[0]
        if x > a:
            ref += integrate.quad(O.S, a, x, epsrel=1e-14)[0]
        assert O.P(x) == pytest.approx(ref, rel=1e-11, abs=1e-15)


def test_Pinv_roundtrip():
    rng = np.random.default_rng(0)
    for R in np.concatenate([rng.uniform(0, 1, 200), [1e-18, 0.5, 0.6099, 0.61, 1 - 1e-12]]):
        assert O.P(O.Pinv(R)) == pytest.approx(R, rel=1e-13, abs=1e-18)


def test_S_small_x_matches_normalised_spectrum():
    """For x -> 0, S(x) = (4/3) x^(1/3) tracks (9 sqrt3 / 8 pi) F(x)."""
    x = 1e-9
    f = 9 * math.sqrt(3) / (8 * math.pi) * O.F_exact([x])[0]
    assert O.S(x) / f == pytest.approx(1.0, abs=1e-3)


def test_sample_x_extremes_and_branch():
    T = O.branch_threshold()
    assert T == 0x9C26B9CE251FFCB8   # round(a^(4/3) 2^64), a from Eq. (11)
    x, R = O.sample_x([0, 0, 0, 0])
    assert x == pytest.approx((0.5 * 2.0 ** -64) ** 0.75, rel=1e-14)
    assert R == pytest.approx(0.5 * 2.0 ** -32, rel=1e-15)
    x, R = O.sample_x([0xFFFFFFFF, 0xFFFFFFFF, 0xFFFFFFFF, 0])
    assert x == pytest.approx(-math.log(9 / 7 * 0.5 * 2.0 ** -64), rel=1e-14)
    assert R == pytest.approx(1 - 0.5 * 2.0 ** -32, rel=1e-15)
    a = O.const_a()
    lo = T - 1
    x1, _ = O.sample_x([lo & 0xFFFFFFFF, lo >> 32, 0, 0])
    x2, _ = O.sample_x([T & 0xFFFFFFFF, T >> 32, 0, 0])
    assert x1 <= a <= x2 * (1 + 1e-15)
    assert x1 == pytest.approx(a, rel=1e-12) and x2 == pytest.approx(a, rel=1e-12)


def test_sample_x_distribution_is_S():
    """x = P^-1(R') over Philox blocks follows S: KS against P."""
    ctr = np.zeros((20000, 4), dtype=np.uint32)
    ctr[:, 0] = np.arange(20000)
    blocks = O.philox(ctr, [9, 0])
    xs = np.array([O.sample_x(b)[0] for b in blocks])
    p = stats.kstest(xs, np.vectorize(O.P)).pvalue
    assert p > 1e-3


# ---------------------------------------------------------------- G, Q
@pytest.mark.parametrize("x", [1e-8, 1e-3, 0.1, 1.0, 5.0, 20.0])
def test_number_and_energy_cdfs_vs_scipy(x):
    g = lambda y: O.F_exact([math.exp(y)])[0]
    c = 4 * math.pi / (math.sqrt(3) * math.gamma(1 / 3)) * 2 ** (-1 / 3)
    lo = 1e-14
    num = 3 * c * lo ** (1 / 3) + integrate.quad(g, math.log(lo), math.log(x),
                                                 epsrel=1e-12, limit=400)[0]
    assert O.G([x])[0] == pytest.approx(num / (5 * math.pi / 3), rel=1e-9)
    en = integrate.quad(lambda t: O.F_exact([t])[0], 0, x, epsrel=1e-12, limit=400)[0]
    assert O.Q([x])[0] == pytest.approx(en / (8 * math.pi / (9 * math.sqrt(3))),
                                        rel=1e-8, abs=1e-14)


def test_Ginv_inverts_G():
    r = np.array([1e-6, 0.01, 0.3, 0.5, 0.9, 0.999])
    assert np.allclose(O.G(O.Ginv(r)), r, rtol=1e-10, atol=0)
