"""Super-photon control and the wiggler-regime counter in the oracle.

Control (Monte Carlo method section: the number of super-photons per
particle and step, and the real photons one represents, set at runtime):
n_try trials of 1/n_try of dN each, and selection of a particle-step with
probability q at weight 1/q.  In a constant B the expected emitted energy
stays the synchrotron power (2/3) alpha hbar Omega^2 gamma^2 dt for every
setting, the record count scales with q, and n_try = 1, q = 1 is the plain
method bit for bit.

Wiggler regime (the text before Eq. (3)): a step counts as outside it when
Omega < omega_L |1 - dir beta_x|, Omega the effective-field frequency and
omega_L |1 - dir beta_x| the rate at which the particle crosses the wave's
phase.  A particle at rest in a wave of amplitude a0 sees Omega ~ a0 omega_L
and a phase rate ~ omega_L: outside the regime for a0 < 1, inside for
a0 > 1; a counter-propagating ultra-relativistic electron at a0 = 100 is
inside, and constant fields never count.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1409_5574_gb300 import workloads as W

HBAR, ME, C = 1.054571817e-34, 9.1093837015e-31, 299792458.0


def _cf(wl):
    s = wl.state
    u = np.stack([s["ux"], s["uy"], s["uz"]], 1)
    Bn = np.array(wl.B) * W.Q_E / (W.M_E * wl.omega_ref)
    bmag = np.linalg.norm(Bn)
    bhat = Bn / bmag
    dtn = wl.dt * wl.omega_ref
    upar = u @ bhat
    uperp = np.linalg.norm(u - upar[:, None] * bhat, axis=1)
    gam = np.sqrt(1 + (u * u).sum(1))
    theta = 2 * np.arctan(bmag * dtn / (2 * gam))
    ua_perp = uperp * np.cos(theta / 2)
    ga = np.sqrt(1 + upar ** 2 + ua_perp ** 2)
    Om = bmag * ua_perp / ga
    eps_r = HBAR * wl.omega_ref / (ME * C * C)
    return (2 / 3 * O.alpha() * eps_r * Om ** 2 * ga ** 2 * dtn).sum()


def _run(wl, nsteps, **ctrl):
    st = wl.copy_state()
    return O.run(O.Problem(**{**wl.problem_kwargs(), **ctrl}), st, nsteps,
                 capacity=1 << 20)


@pytest.mark.parametrize("n_try,q", [(4, 1.0), (1, 0.5), (3, 0.25)])
def test_control_keeps_the_synchrotron_power(n_try, q):
    wl = W.const_b(n=3000, nsteps=300, seed=5)
    res = _run(wl, 300, n_try=n_try, select_prob=q)
    base = _run(wl, 300)
    expect = _cf(wl) * 300
    e = res["photons"]["weight"] * res["photons"]["eps"]
    sigma = math.sqrt((e * e).sum())
    assert abs(e.sum() - expect) < 4 * sigma
    assert res["ledger"]["emit"].sum() == pytest.approx(e.sum(), rel=1e-12)
    # records: each trial emits with probability ~ dN / n_try, selection
    # keeps a fraction q of the particle-steps
    nb = base["stats"]["records"]
    assert abs(res["stats"]["records"] - q * nb) < 5 * math.sqrt(nb) + 0.01 * nb
    if q < 1:
        w = res["photons"]["weight"] / wl.state["w"][res["photons"]["pid"]]
        assert np.all(np.abs(w * q - np.round(w * q)) < 1e-9)   # k / q


def test_control_off_is_the_plain_method():
    wl = W.const_b(n=500, nsteps=50, seed=6)
    a, b = _run(wl, 50), _run(wl, 50, n_try=1, select_prob=1.0)
    for k in a["photons"]:
        np.testing.assert_array_equal(a["photons"][k], b["photons"][k])


def _at_rest(n, a0):
    wl = W.plane_wave(a0=a0, n=n, seed=7)
    for k in ("ux", "uy", "uz"):
        wl.state[k] = np.zeros(n)
    return wl


def test_wiggler_counter_limits():
    for a0, expect_all in ((0.5, True), (2.0, False)):
        wl = _at_rest(200, a0)
        res = _run(wl, 1)
        assert res["stats"]["wiggler_invalid"] == (200 if expect_all else 0), a0
    wl = W.plane_wave(a0=100.0, n=500, seed=8)      # counter-propagating, gamma 1000
    assert _run(wl, 20)["stats"]["wiggler_invalid"] == 0
    wl = W.const_b(n=200, nsteps=20, seed=9)
    assert _run(wl, 20)["stats"]["wiggler_invalid"] == 0


def test_oracle_result_does_not_depend_on_thread_count():
    """The oracle's particles are independent and its photon records are
    returned sorted by (pid, step): one thread and all threads give the same
    state, ledger and records (what the single-core timing relies on)."""
    wl = W.plane_wave(a0=500.0, n=300, periods=1, seed=8)
    cores = O.num_threads()
    out = []
    for nt in (1, cores):
        O.set_num_threads(nt)
        try:
            assert O.num_threads() == nt
            st = wl.copy_state()
            r = O.run(O.Problem(**wl.problem_kwargs()), st, 40, capacity=1 << 16)
        finally:
            O.set_num_threads(cores)
        out.append((st, r))
    (s1, r1), (s2, r2) = out
    for k in s1:
        np.testing.assert_array_equal(s1[k], s2[k])
    assert len(r1["photons"]["x"]) > 0
    for k in r1["photons"]:
        np.testing.assert_array_equal(r1["photons"][k], r2["photons"][k])
    for k in r1["ledger"]:
        np.testing.assert_array_equal(r1["ledger"][k], r2["ledger"][k])
