"""Pins of the float32 envelope that bounds the multi-step FP32 parity tests.

Over many steps a float32-held state departs from the FP64 oracle by more than
the per-particle 1e-5 a single FP32 step meets: the trajectory amplifies the
state's rounding.  These tests show it on the oracle alone (no GPU): the
oracle with its own state held in float32 (rounded after every step, or
started one unit in the last place away) departs from itself by more than
1e-5 on the Yee-grid, constant-B and plane-wave workloads.  The GPU tests then
bound each particle's departure by max(1e-5, envelope).

The helper's parts are pinned too: the rounding modes against their
definitions, and the step-by-step runs against one multi-step oracle run.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1409_5574_gb300 import workloads as W

import fp32_envelope as FE


def _f32_state(wl):
    return {k: v.astype(np.float32).astype(np.float64) for k, v in wl.state.items()}


def small_yee(nx=130, ny=100, n=6000 + 13, seed=3, a0=300.0):
    """The small periodic Yee case of the GPU Yee tests (seeded inputs)."""
    rng = np.random.default_rng(seed)
    dxn = 2 * np.pi / 32
    planes = W.yee_planes(nx, ny, a0, dxn, rng)
    wl = W.yee2d(n_grid=64, slab=32, n_particles=n, seed=seed, with_grid=False)
    wl.yee = planes
    wl.state["x"] = rng.uniform(-0.5, nx + 0.5, n) * dxn
    wl.state["y"] = rng.uniform(-0.5, ny + 0.5, n) * dxn
    return wl


def test_rounding_modes_follow_their_definitions():
    rng = np.random.default_rng(1)
    v = np.concatenate([rng.standard_normal(5000) * 10.0 ** rng.uniform(-8, 8, 5000),
                        np.float32(rng.standard_normal(100)).astype(np.float64), [0.0]])
    f = v.astype(np.float32)
    ulp = np.abs(np.nextafter(f, np.float32(np.inf)).astype(np.float64)
                 - np.nextafter(f, np.float32(-np.inf)).astype(np.float64)) / 2
    for mode in ("rn", "rz", "ru", "rd"):
        r = FE.f32_round(v, mode)
        assert np.array_equal(r, r.astype(np.float32).astype(np.float64))  # float32 values
        assert np.all(np.abs(r - v) <= ulp * 1.0000001)                   # within one unit
        exact = v.astype(np.float32).astype(np.float64) == v
        assert np.array_equal(r[exact], v[exact])                          # exact values kept
    assert np.array_equal(FE.f32_round(v, "rn"), f.astype(np.float64))
    assert np.all(FE.f32_round(v, "ru") >= v) and np.all(FE.f32_round(v, "rd") <= v)
    assert np.all(np.abs(FE.f32_round(v, "rz")) <= np.abs(v))
    n = FE.nudged({"ux": f.astype(np.float64), "w": v})
    assert np.array_equal(n["w"], v)                                       # weights untouched
    moved = np.abs(n["ux"] - f.astype(np.float64))
    assert np.all(moved > 0) and np.all(moved <= 2 * ulp * 1.0000001)


def test_step_by_step_runs_reproduce_one_oracle_run():
    """Unrounded one-step calls (with the step counter carried) equal one
    multi-step call bit for bit: the envelope's runs differ from the
    reference only by the rounding they add."""
    wl = W.plane_wave(a0=300.0, n=37, seed=5)
    prob = O.Problem(**wl.problem_kwargs())
    st0 = _f32_state(wl)
    ref = {k: v.copy() for k, v in st0.items()}
    O.run(prob, ref, 60, t0=7)
    st = FE.run_rounded(prob, st0, 60, None, t0=7)
    for k in FE.STATE:
        assert np.array_equal(st[k], ref[k]), k


def test_yee_envelope_exceeds_the_single_step_bar():
    """25 steps of the small Yee case (a0 = 300 standing wave + noise, gamma
    log-uniform in [10, 3000]): the oracle's own float32 departures reach
    1e-4, and more than 1% of the particles exceed 1e-5, in the rounded runs
    and also from a start one unit in the last place away."""
    wl = small_yee()
    prob = O.Problem(**wl.problem_kwargs())
    st0 = _f32_state(wl)
    ref = {k: v.copy() for k, v in st0.items()}
    O.run(prob, ref, 25, capacity=1 << 16)
    env = FE.envelope(prob, st0, 25, ref)
    assert env.max() > 1e-4 and np.mean(env > 1e-5) > 0.01, (env.max(), np.mean(env > 1e-5))
    ulp_only = FE.envelope(prob, st0, 25, ref, modes=("ulp",))
    assert ulp_only.max() > 1e-5 and np.mean(ulp_only > 1e-5) > 0.005


def test_constant_b_envelope_exceeds_the_single_step_bar():
    """500 steps of gyration with the LL kick in B = 500 m omega_L / e (the
    strongest constant-B ensembles of the batched workload): the rotation
    accumulates the per-step rounding past 1e-5."""
    omega = 2 * math.pi * W.C_LIGHT / 0.8e-6
    Bt = 500.0 * W.M_E * omega / W.Q_E
    rng = np.random.default_rng(2)
    n = 16
    gamma = rng.uniform(100.0, 1000.0, n)
    u = rng.standard_normal((n, 3))
    u *= (np.sqrt(gamma ** 2 - 1) / np.linalg.norm(u, axis=1))[:, None]
    st0 = {k: np.float32(v).astype(np.float64) for k, v in
           dict(x=np.zeros(n), y=np.zeros(n), z=np.zeros(n), ux=u[:, 0], uy=u[:, 1],
                uz=u[:, 2], w=np.ones(n)).items()}
    prob = O.Problem(omega_ref=omega, dt=(2 * math.pi / omega) / 200, rr_mode=O.RR_APPLY,
                     field_kind=O.FIELD_CONST, B=(0.0, 0.0, Bt))
    ref = {k: v.copy() for k, v in st0.items()}
    O.run(prob, ref, 500)
    env = FE.envelope(prob, st0, 500, ref)
    assert np.median(env) > 1e-5, env


def test_long_plane_wave_envelope():
    """4000 steps (20 periods) in the counter-propagating CP wave with the LL
    kick: the float32-held runs depart by more than 1e-4 for every particle at
    a0 = 100 and 500, so the full-length runs need the envelope too."""
    for a0 in (100.0, 500.0):
        wl = W.plane_wave(a0=a0, n=8, seed=9)
        prob = O.Problem(**wl.problem_kwargs())
        st0 = _f32_state(wl)
        ref = {k: v.copy() for k, v in st0.items()}
        O.run(prob, ref, 4000)
        env = FE.envelope(prob, st0, 4000, ref, modes=("rn", "rz", "ru", "rd"))
        assert env.min() > 1e-4, (a0, env)
