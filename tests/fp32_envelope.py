"""The FP64 oracle's own float32 envelope (test infrastructure; it calls only
the oracle).

A step path whose state (x, y, z, u) is float32 between steps cannot follow
the FP64 oracle more closely than the oracle follows itself when its own state
is held in float32.  `envelope()` measures that per particle: the largest
relative momentum departure max_k |u_k - u_ref_k| / |u_ref| from the plain
oracle run of

  * the oracle with its state rounded to the nearest float32 after every step;
  * the same with the state rounded toward zero, toward +inf and toward -inf
    after every step (a systematic error of one unit in the last place per
    step, the size of one float32 rounding that always falls the same way);
  * the plain oracle started from the float32 start moved by one unit in the
    last place in every state component, up or down by a seeded coin.

The momentum is u = p / (m c) (the Boris push of the Numerical implementation
section advances it); the runs differ from the reference only by float32
storage, so the departures are a property of the trajectory (its sensitivity
to the state's rounding), not of any implementation.
"""
from __future__ import annotations

from typing import Optional, Sequence

import numpy as np

import oracle as O

STATE = ("x", "y", "z", "ux", "uy", "uz")
MODES = ("rn", "rz", "ru", "rd", "ulp")


def f32_round(v: np.ndarray, mode: str) -> np.ndarray:
    """v (float64) held in float32: to nearest ("rn"), toward zero ("rz"),
    toward +inf ("ru") or toward -inf ("rd"); returned as float64."""
    v = np.asarray(v, dtype=np.float64)
    f = v.astype(np.float32)                 # round to nearest even
    d = f.astype(np.float64)
    up = np.nextafter(f, np.float32(np.inf))
    dn = np.nextafter(f, np.float32(-np.inf))
    if mode == "rn":
        pass
    elif mode == "ru":
        f = np.where(d < v, up, f)
    elif mode == "rd":
        f = np.where(d > v, dn, f)
    elif mode == "rz":
        f = np.where(np.abs(d) > np.abs(v), np.where(v > 0, dn, up), f)
    else:
        raise ValueError(mode)
    return f.astype(np.float64)


def momentum_rel(a: dict, ref: dict) -> np.ndarray:
    """Per particle max_k |u_k - ref_k| / |ref| over the three components."""
    ua = np.stack([a["ux"], a["uy"], a["uz"]], 1)
    ur = np.stack([ref["ux"], ref["uy"], ref["uz"]], 1)
    return np.abs(ua - ur).max(1) / np.maximum(np.linalg.norm(ur, axis=1), 1e-300)


def run_rounded(problem: O.Problem, state: dict, nsteps: int, mode: Optional[str],
                t0: int = 0, pid: Optional[np.ndarray] = None) -> dict:
    """The oracle one step per call from `state` (copied), the state rounded
    by `mode` after every step (None: not rounded, which reproduces one
    multi-step oracle run exactly)."""
    st = {k: np.array(v, dtype=np.float64) for k, v in state.items()}
    for s in range(nsteps):
        O.run(problem, st, 1, t0=t0 + s, pid=pid, capacity=1 << 10)
        if mode is not None:
            for k in STATE:
                if k in st:
                    st[k] = f32_round(st[k], mode)
    return st


def nudged(state: dict, seed: int = 0) -> dict:
    """The float32 state moved by one unit in the last place, each value up or
    down by a seeded coin (the state must hold float32 values)."""
    rng = np.random.default_rng(seed)
    out = {}
    for k, v in state.items():
        v = np.asarray(v, dtype=np.float64)
        if k in STATE:
            f = v.astype(np.float32)
            up = rng.integers(0, 2, f.size).astype(bool)
            f = np.where(up, np.nextafter(f, np.float32(np.inf)),
                         np.nextafter(f, np.float32(-np.inf)))
            out[k] = f.astype(np.float64)
        else:
            out[k] = v.copy()
    return out


def envelope(problem: O.Problem, state: dict, nsteps: int, reference: dict,
             t0: int = 0, pid: Optional[np.ndarray] = None,
             modes: Sequence[str] = MODES) -> np.ndarray:
    """Per particle, the largest momentum departure of the float32-held runs
    (`modes`) from `reference`, the plain oracle's state after `nsteps` steps
    from the same (float32-valued) `state`."""
    env = np.zeros(len(reference["ux"]))
    for m in modes:
        if m == "ulp":
            st = nudged(state)
            O.run(problem, st, nsteps, t0=t0, pid=pid, capacity=1 << 10)
        else:
            st = run_rounded(problem, state, nsteps, m, t0=t0, pid=pid)
        env = np.maximum(env, momentum_rel(st, reference))
    return env


# The bar is FACTOR x the envelope: the envelope's runs move the state by at
# most one float32 unit of |u| per step (storage rounding only), while an FP32
# kernel also rounds inside the step; its one-step departure is at most
# FACTOR units of |u| (test_gpu_parity.py checks it on every field kind), and
# a trajectory's departure grows in proportion to the per-step perturbation.
FACTOR = 3.0


def float32_units(u: dict, ref: dict) -> np.ndarray:
    """Per particle max_k |u_k - ref_k| in float32 units in the last place of
    |ref| (the spacing of float32 numbers at |ref|)."""
    ua = np.stack([u["ux"], u["uy"], u["uz"]], 1)
    ur = np.stack([ref["ux"], ref["uy"], ref["uz"]], 1)
    unit = np.spacing(np.linalg.norm(ur, axis=1).astype(np.float32)).astype(np.float64)
    return np.abs(ua - ur).max(1) / unit


def assert_within(rel: np.ndarray, env: np.ndarray, floor: float = 1e-5,
                  factor: float = FACTOR) -> None:
    """Every particle's GPU-vs-oracle departure within max(floor, factor x
    envelope)."""
    bound = np.maximum(floor, factor * env)
    bad = np.flatnonzero(rel > bound)
    assert bad.size == 0, (
        f"{bad.size} particles outside the float32 envelope; worst "
        f"{[(int(i), float(rel[i]), float(env[i])) for i in bad[np.argsort(-rel[bad])][:5]]}")
