"""The emission's spread in angle about the velocity in the oracle (Eqs. (5)
and (6): the circular-motion spectrum by angle).

With x = omega / omega_c and psi = gamma theta (theta out of the plane of the
orbit) the energy radiated per unit x and psi is proportional to
sigma + pi = (1 + psi^2)^2 K_2/3(xi)^2 + (1 + psi^2) psi^2 K_1/3(xi)^2,
xi = (x/2)(1 + psi^2)^(3/2).  What fixes it independently of the oracle:

* K_1/3 and K_2/3 are scipy's modified Bessel functions;
* integrated over psi it is the angle-integrated spectrum of Eq. (8):
  int dpsi (sigma + pi) = (2 pi / sqrt 3) F(x) / x^2 (both signs of psi);
* the sigma polarisation carries 7/8 of the energy over all x and psi, and
  the total int x^2 (sigma + pi) dx dpsi is (2 pi / sqrt 3) int F = 16 pi^2 / 27;
* for x -> 0 the spread scales as x^(-1/3) (psi (x/2)^(1/3) has a limit
  law), for x -> infinity psi is Gaussian with variance 1/(3x);
* in orc_run with the spread on, a photon in a pure B field leaves the
  orbit plane by theta with gamma theta distributed as the density at the
  record's own x (probability-integral transform uniform, sign symmetric),
  and with it off the records are the collinear ones bit for bit.
"""
import math

import numpy as np
import pytest
from scipy import special, stats

import oracle as O
from paper_1409_5574_gb300 import workloads as W

HBAR, ME, C = 1.054571817e-34, 9.1093837015e-31, 299792458.0


def test_bessel_k_third_orders_match_scipy():
    z = np.logspace(-9, 2.6, 70)
    np.testing.assert_allclose(O.K13(z), special.kv(1 / 3, z), rtol=1e-12)
    np.testing.assert_allclose(O.K23(z), special.kv(2 / 3, z), rtol=1e-12)


@pytest.mark.parametrize("x", [1e-8, 1e-4, 1e-2, 0.3, 1.0, 3.0, 10.0, 40.0])
def test_angle_integral_is_the_synchrotron_spectrum(x):
    two_sided = 2.0 * O.ang_norm(np.array([x]))[0]
    expect = 2.0 * math.pi / math.sqrt(3.0) * O.F_exact(np.array([x]))[0] / x ** 2
    assert two_sided == pytest.approx(expect, rel=1e-10)


def _grid_integrals():
    lx = np.linspace(math.log(1e-5), math.log(45.0), 701)
    x = np.exp(lx)
    s = np.linspace(0.0, 9.0, 1201)           # psi = sinh s
    psi = np.sinh(s)
    X, S = np.meshgrid(x, s, indexing="ij")
    sig, pi = O.ang_parts(X, np.sinh(S))
    jac = np.cosh(S)                           # dpsi = cosh s ds
    Is = np.trapezoid(sig * jac, s, axis=1) * 2.0    # both signs of psi
    Ip = np.trapezoid(pi * jac, s, axis=1) * 2.0
    w = x ** 3                                 # x^2 dx = x^3 d(ln x)
    return np.trapezoid(w * Is, lx), np.trapezoid(w * Ip, lx), psi


def test_sigma_polarisation_carries_seven_eighths():
    es, ep, _ = _grid_integrals()
    assert es / ep == pytest.approx(7.0, rel=2e-4)
    assert es + ep == pytest.approx(16.0 * math.pi ** 2 / 27.0, rel=2e-4)


def test_sampler_inverts_the_cdf_and_follows_the_density():
    rng = np.random.default_rng(11)
    x = np.exp(rng.uniform(math.log(1e-6), math.log(30.0), 400))
    u = rng.uniform(0.0, 1.0, 400)
    psi = O.ang_sample(x, u)
    assert np.all(psi >= 0)
    np.testing.assert_allclose(O.ang_cdf(x, psi), u, rtol=0, atol=1e-10)
    # the CDF's slope is the density over its integral (scipy quadrature of
    # the oracle's own density at a few points, independent of Simpson)
    from scipy.integrate import quad
    for xx, pp in [(0.01, 3.0), (1.0, 0.4), (8.0, 0.2)]:
        dens = lambda q: sum(O.ang_parts(np.array([xx]), np.array([q])))[0]
        num = quad(dens, 0.0, pp, epsrel=1e-12, limit=200)[0]
        assert O.ang_cdf(np.array([xx]), np.array([pp]))[0] == pytest.approx(
            num / O.ang_norm(np.array([xx]))[0], rel=1e-9)


def test_spread_limits_small_and_large_x():
    u = np.array([0.1, 0.3, 0.5, 0.7, 0.9, 0.99])
    # x -> 0: psi scales as x^(-1/3)
    a = O.ang_sample(np.full(6, 8e-8), u)
    b = O.ang_sample(np.full(6, 1e-8), u)
    np.testing.assert_allclose(b / a, 2.0, rtol=2e-4)
    # x -> infinity: half-normal with variance 1 / (3 x) (the leading
    # correction is O(1/x))
    x = 400.0
    q = O.ang_sample(np.full(6, x), u)
    expect = special.erfinv(u) * math.sqrt(2.0) / math.sqrt(3.0 * x)
    np.testing.assert_allclose(q, expect, rtol=2e-2)


def _planar_const_b(n, seed):
    """Electrons circling in B = 1e4 T along z (momenta in the x-y plane),
    LL ledger only: gamma is conserved by the push, the orbit normal is z."""
    wl = W.const_b(n=n, nsteps=1, seed=seed)
    rng = np.random.default_rng(seed)
    g = rng.uniform(100.0, 1000.0, n)
    ph = rng.uniform(0.0, 2.0 * math.pi, n)
    um = np.sqrt(g * g - 1.0)
    wl.state.update(ux=um * np.cos(ph), uy=um * np.sin(ph), uz=np.zeros(n))
    return wl, g


def test_orc_run_turns_photons_out_of_the_orbit_plane():
    n, nsteps = 3000, 200
    wl, g0 = _planar_const_b(n, seed=21)
    kw = wl.problem_kwargs()
    base = O.run(O.Problem(**kw), wl.copy_state(), nsteps, capacity=1 << 18)
    off = O.run(O.Problem(**kw, ang_spread=0), wl.copy_state(), nsteps, capacity=1 << 18)
    on = O.run(O.Problem(**kw, ang_spread=1), wl.copy_state(), nsteps, capacity=1 << 18)
    for k in base["photons"]:
        np.testing.assert_array_equal(base["photons"][k], off["photons"][k])
    pa, pb = base["photons"], on["photons"]
    # the same records but for the direction
    for k in ("pid", "step", "eps", "weight", "x", "y", "z"):
        np.testing.assert_array_equal(pa[k], pb[k])
    m = pb["pid"].size
    assert m > 3000
    d = np.stack([pb["nx"], pb["ny"], pb["nz"]], 1)
    np.testing.assert_allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-14)
    # in-plane part along the collinear direction
    d0 = np.stack([pa["nx"], pa["ny"]], 1)
    ip = d[:, :2] / np.linalg.norm(d[:, :2], axis=1, keepdims=True)
    np.testing.assert_allclose((ip * d0).sum(1), 1.0, atol=1e-12)
    # gamma theta against the density at the record's x: the mean momentum
    # of a step has |u_a| = |u| cos(phi/2), phi the step's rotation angle
    Bn = 1.0e4 * W.Q_E / (W.M_E * wl.omega_ref)
    dtn = wl.dt * wl.omega_ref
    g = g0[pb["pid"]]
    rot = 2.0 * np.arctan(Bn * dtn / (2.0 * g))
    ua = np.sqrt(g * g - 1.0) * np.cos(rot / 2.0)
    ga = np.sqrt(1.0 + ua * ua)
    Om = Bn * ua / ga
    eps_r = HBAR * wl.omega_ref / (ME * C * C)
    x = pb["eps"] / (1.5 * eps_r * Om * ga * ga)
    psi = np.arcsin(d[:, 2]) * ga
    U = O.ang_cdf(x, np.abs(psi))
    assert stats.kstest(U, "uniform").pvalue > 0.01
    frac_up = np.mean(psi > 0)
    assert abs(frac_up - 0.5) < 4.0 * 0.5 / math.sqrt(m)
