"""FP64 CPU oracle for the synchrotron-emission particle step (arXiv:1409.5574).

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference arm of ``bench.py`` may import this package. The GPU
library (``paper_1409_5574_gb300``) never imports it, and the two share no
code: this package wraps ``prad_oracle.c`` (plain C, FP64, OpenMP over
particles) through ctypes, compiling it with gcc on first use.

Function map to the paper (arXiv:1409.5574):

* ``philox``           - counter-based RNG behind R', R of the Monte Carlo method
* ``F_exact``, ``F``   - Eq. (8), F(x) = x int_x^inf K_5/3
* ``S``, ``P``, ``Pinv`` - Eqs. (11)-(12), noise-reduction proposal and its CDF
* ``sample_x``         - omega_emit = omega(R') from one Philox block
* ``G``, ``Q``, ``Ginv`` - number / energy CDFs of the spectrum (Eq. (10))
* ``boris``            - Boris push (Numerical implementation section)
* ``heff_field``, ``heff_momentum`` - H_eff, field form and Eq. (9)
* ``run``              - the full per-step path with emission and LL ledger
* ``angular_histogram`` - Fig. 4, emitted energy by direction (FP64 numpy)
* ``K13``, ``K23``, ``ang_parts``, ``ang_norm``, ``ang_cdf``, ``ang_sample`` -
  Eqs. (5)-(6), the emission's spread in angle about the velocity

Every function is pinned by a ``-m "not gpu"`` test; see tests/test_oracle_*.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "prad_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile prad_oracle.c into oracle/_build/liboracle.so (gcc, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            so = build()
            L = ctypes.CDLL(so)
            d, i64, u64, u32, i32 = (ctypes.c_double, ctypes.c_int64,
                                     ctypes.c_uint64, ctypes.c_uint32,
                                     ctypes.c_int32)
            P = ctypes.c_void_p
            L.orc_init.restype = ctypes.c_int
            for name in ("orc_F_exact", "orc_F", "orc_S", "orc_P", "orc_Pinv",
                         "orc_G", "orc_Q", "orc_Ginv", "orc_int_F",
                         "orc_int_F_over_x"):
                getattr(L, name).restype = d
                getattr(L, name).argtypes = [d]
            L.orc_const_a.restype = d
            L.orc_alpha.restype = d
            L.orc_branch_threshold.restype = u64
            L.orc_num_threads.restype = ctypes.c_int
            L.orc_set_num_threads.argtypes = [ctypes.c_int]
            L.orc_sample_x.restype = d
            L.orc_sample_x.argtypes = [P, P]
            L.orc_S_of_words.restype = d
            L.orc_S_of_words.argtypes = [P]
            L.orc_philox4x32_10.argtypes = [P, P, P]
            for name in ("orc_G_batch", "orc_Q_batch", "orc_Ginv_batch",
                         "orc_F_batch", "orc_F_exact_batch"):
                getattr(L, name).argtypes = [P, P, i64]
            for name in ("orc_K13_batch", "orc_K23_batch", "orc_ang_norm_batch"):
                getattr(L, name).argtypes = [P, P, i64]
            for name in ("orc_ang_cdf_batch", "orc_ang_sample_batch"):
                getattr(L, name).argtypes = [P, P, P, i64]
            L.orc_ang_parts_batch.argtypes = [P, P, P, P, i64]
            L.orc_boris.argtypes = [P, P, P, d, d]
            L.orc_heff_field.restype = d
            L.orc_heff_field.argtypes = [P, P, P]
            L.orc_heff_momentum.restype = d
            L.orc_heff_momentum.argtypes = [P, P, d]
            L.orc_fields.argtypes = [P, d, d, d, i64, P, P]
            L.orc_run.restype = ctypes.c_int
            L.orc_run.argtypes = [P, i64, i32, i64] + [P] * 16
            L.orc_init()
            _lib = L
    return _lib


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _vec(fn_name: str, x) -> np.ndarray:
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    out = np.empty_like(x)
    getattr(lib(), fn_name)(_ptr(x), _ptr(out), ctypes.c_int64(x.size))
    return out


# ---- scalar / vector special functions ---------------------------------
def F_exact(x):
    """Eq. (8) by trapezoid quadrature of the cosh representation."""
    return _vec("orc_F_exact_batch", x)


def F(x):
    """Eq. (8), log-log cubic Hermite interpolant of F_exact."""
    return _vec("orc_F_batch", x)


def K13(z):
    """Modified Bessel function K_1/3 (cosh-integral trapezoid rule)."""
    return _vec("orc_K13_batch", z)


def K23(z):
    """Modified Bessel function K_2/3 (cosh-integral trapezoid rule)."""
    return _vec("orc_K23_batch", z)


def _vec2(fn_name: str, a, b) -> np.ndarray:
    a, b = np.broadcast_arrays(np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64))
    a = np.ascontiguousarray(a)
    b = np.ascontiguousarray(b)
    out = np.empty_like(a)
    getattr(lib(), fn_name)(_ptr(a), _ptr(b), _ptr(out), ctypes.c_int64(a.size))
    return out


def ang_parts(x, psi):
    """The two polarisation terms of Eq. (5) at x = omega/omega_c and
    psi = gamma theta: (sigma, pi) = ((1+psi^2)^2 K_2/3(xi)^2,
    (1+psi^2) psi^2 K_1/3(xi)^2), xi = (x/2)(1+psi^2)^(3/2) (Eq. (6))."""
    a, b = np.broadcast_arrays(np.asarray(x, dtype=np.float64), np.asarray(psi, dtype=np.float64))
    a = np.ascontiguousarray(a)
    b = np.ascontiguousarray(b)
    sig, pi = np.empty_like(a), np.empty_like(a)
    lib().orc_ang_parts_batch(_ptr(a), _ptr(b), _ptr(sig), _ptr(pi), ctypes.c_int64(a.size))
    return sig, pi


def ang_norm(x):
    """int_0^inf (sigma + pi) dpsi at fixed x (Simpson in asinh psi)."""
    return _vec("orc_ang_norm_batch", x)


def ang_cdf(x, psi):
    """Fraction of the one-sided psi integral below |psi| at fixed x."""
    return _vec2("orc_ang_cdf_batch", x, psi)


def ang_sample(x, u):
    """psi >= 0 with ang_cdf(x, psi) = u (the angular spread's inverse CDF)."""
    return _vec2("orc_ang_sample_batch", x, u)


def G(x):
    """Photon-number CDF int_0^x F(t)/t dt / (5 pi/3)."""
    return _vec("orc_G_batch", x)


def Q(x):
    """Energy CDF int_0^x F(t) dt / (8 pi / (9 sqrt 3)) (Eq. (10))."""
    return _vec("orc_Q_batch", x)


def Ginv(r):
    return _vec("orc_Ginv_batch", r)


def S(x: float) -> float:
    return lib().orc_S(float(x))


def P(x: float) -> float:
    return lib().orc_P(float(x))


def Pinv(R: float) -> float:
    return lib().orc_Pinv(float(R))


def const_a() -> float:
    return lib().orc_const_a()


def alpha() -> float:
    return lib().orc_alpha()


def branch_threshold() -> int:
    return int(lib().orc_branch_threshold())


def int_F(x: float) -> float:
    return lib().orc_int_F(float(x))


def int_F_over_x(x: float) -> float:
    return lib().orc_int_F_over_x(float(x))


def num_threads() -> int:
    return lib().orc_num_threads()


def set_num_threads(n: int) -> None:
    """Threads of the oracle's later parallel loops."""
    lib().orc_set_num_threads(int(n))


def philox(ctr, key) -> np.ndarray:
    """Philox4x32-10 on rows of ``ctr`` (n,4) with ``key`` (2,)."""
    ctr = np.ascontiguousarray(np.atleast_2d(np.asarray(ctr, dtype=np.uint32)))
    key = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    out = np.empty_like(ctr)
    L = lib()
    for i in range(ctr.shape[0]):
        L.orc_philox4x32_10(_ptr(ctr[i]), _ptr(key), _ptr(out[i]))
    return out


def sample_x(words) -> tuple:
    """x = P^-1(R') and R from one Philox output block (4 x uint32)."""
    w = np.ascontiguousarray(np.asarray(words, dtype=np.uint32))
    R = np.zeros(1, dtype=np.float64)
    x = lib().orc_sample_x(_ptr(w), _ptr(R))
    return x, float(R[0])


def S_of_words(words) -> float:
    """S of Eq. (11) on the branch the Philox block's sample falls in."""
    w = np.ascontiguousarray(np.asarray(words, dtype=np.uint32))
    return lib().orc_S_of_words(_ptr(w))


def boris(u, E, B, q: float, dtn: float) -> np.ndarray:
    u = np.array(u, dtype=np.float64)
    E = np.ascontiguousarray(E, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    lib().orc_boris(_ptr(u), _ptr(E), _ptr(B), float(q), float(dtn))
    return u


def heff_field(E, B, beta) -> float:
    E, B, beta = (np.ascontiguousarray(v, dtype=np.float64) for v in (E, B, beta))
    return lib().orc_heff_field(_ptr(E), _ptr(B), _ptr(beta))


def heff_momentum(u_old, u_new, dtn: float) -> float:
    a = np.ascontiguousarray(u_old, dtype=np.float64)
    b = np.ascontiguousarray(u_new, dtype=np.float64)
    return lib().orc_heff_momentum(_ptr(a), _ptr(b), float(dtn))


# ---- full step -----------------------------------------------------------
class _Problem(ctypes.Structure):
    _fields_ = [
        ("omega_ref", ctypes.c_double), ("dt", ctypes.c_double),
        ("charge", ctypes.c_double), ("seed", ctypes.c_uint64),
        ("ensemble", ctypes.c_uint32), ("rr_mode", ctypes.c_int32),
        ("heff_form", ctypes.c_int32), ("field_kind", ctypes.c_int32),
        ("dims", ctypes.c_int32), ("pad0", ctypes.c_int32),
        ("E", ctypes.c_double * 3), ("B", ctypes.c_double * 3),
        ("a0", ctypes.c_double), ("lam", ctypes.c_double),
        ("phase0", ctypes.c_double), ("dir", ctypes.c_int32),
        ("hand", ctypes.c_int32), ("yee", ctypes.c_void_p * 6),
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("dx", ctypes.c_double), ("dy", ctypes.c_double),
        ("x0", ctypes.c_double), ("y0", ctypes.c_double),
        ("n_try", ctypes.c_int32), ("ang_spread", ctypes.c_int32),
        ("select_prob", ctypes.c_double),
    ]


class _Photons(ctypes.Structure):
    _fields_ = [("capacity", ctypes.c_int64)] + [
        (n, ctypes.c_void_p) for n in
        ("x", "y", "z", "nx", "ny", "nz", "eps", "weight", "pid", "step")]


FIELD_CONST, FIELD_PLANE_WAVE, FIELD_YEE2D = 0, 1, 2
RR_OFF, RR_LEDGER, RR_APPLY = 0, 1, 2
HEFF_FIELD, HEFF_MOMENTUM = 0, 1


@dataclass
class Problem:
    """SI description of one run (same meaning as the GPU library's config)."""
    omega_ref: float
    dt: float
    charge: float = -1.0
    seed: int = 1
    ensemble: int = 0
    rr_mode: int = RR_LEDGER
    heff_form: int = HEFF_FIELD
    field_kind: int = FIELD_CONST
    dims: int = 3
    E: Sequence[float] = (0.0, 0.0, 0.0)
    B: Sequence[float] = (0.0, 0.0, 0.0)
    a0: float = 0.0
    lam: float = 0.8e-6
    phase0: float = 0.0
    direction: int = 1
    hand: int = 1
    yee: Optional[Sequence[np.ndarray]] = None
    dx: float = 1.0
    dy: float = 1.0
    x0: float = 0.0
    y0: float = 0.0
    n_try: int = 1
    select_prob: float = 1.0
    ang_spread: int = 0
    _keep: list = field(default_factory=list, repr=False)

    def to_c(self) -> _Problem:
        p = _Problem()
        p.omega_ref, p.dt, p.charge = self.omega_ref, self.dt, self.charge
        p.seed, p.ensemble = int(self.seed), int(self.ensemble)
        p.rr_mode, p.heff_form = self.rr_mode, self.heff_form
        p.field_kind, p.dims = self.field_kind, self.dims
        for k in range(3):
            p.E[k], p.B[k] = self.E[k], self.B[k]
        p.a0, p.lam, p.phase0 = self.a0, self.lam, self.phase0
        p.dir, p.hand = self.direction, self.hand
        if self.yee is not None:
            planes = [np.ascontiguousarray(a, dtype=np.float32) for a in self.yee]
            self._keep = planes
            for k in range(6):
                p.yee[k] = planes[k].ctypes.data
            p.ny, p.nx = planes[0].shape
        p.dx, p.dy, p.x0, p.y0 = self.dx, self.dy, self.x0, self.y0
        p.n_try, p.select_prob = int(self.n_try), float(self.select_prob)
        p.ang_spread = int(self.ang_spread)
        return p


def fields(problem: Problem, x: float, y: float, z: float, step: int):
    E = np.zeros(3)
    B = np.zeros(3)
    p = problem.to_c()
    lib().orc_fields(ctypes.byref(p), x, y, z, step, _ptr(E), _ptr(B))
    return E, B


def run(problem: Problem, state: dict, nsteps: int, t0: int = 0,
        capacity: int = 1 << 16, pid: Optional[np.ndarray] = None,
        ledger: Optional[dict] = None, trial_log: bool = False) -> dict:
    """Advance ``state`` (dict of float64 x,y,z,ux,uy,uz,w) in place.

    Returns photons (sorted by (pid, step)), stats and the ledger; with
    ``trial_log`` also the per-(particle, step) dN, R and sampled x.
    """
    L = lib()
    n = state["x"].size
    arr = {k: np.ascontiguousarray(state[k], dtype=np.float64)
           for k in ("x", "y", "z", "ux", "uy", "uz", "w")}
    if pid is None:
        pid = np.arange(n, dtype=np.uint32)
    pid = np.ascontiguousarray(pid, dtype=np.uint32)
    if ledger is None:
        ledger = {"emit": np.zeros(n), "ll": np.zeros(n)}
    ph = {k: np.zeros(capacity) for k in
          ("x", "y", "z", "nx", "ny", "nz", "eps", "weight")}
    ph["pid"] = np.zeros(capacity, dtype=np.uint32)
    ph["step"] = np.zeros(capacity, dtype=np.uint32)
    cph = _Photons()
    cph.capacity = capacity
    for k, v in ph.items():
        setattr(cph, k, v.ctypes.data)
    cursor = np.zeros(1, dtype=np.int64)
    stats = np.zeros(6, dtype=np.int64)
    tl = None
    if trial_log:
        tl = {k: np.zeros((n, nsteps)) for k in ("dN", "R", "x")}
    cp = problem.to_c()
    rc = L.orc_run(ctypes.byref(cp), n, nsteps, t0,
                   _ptr(arr["x"]), _ptr(arr["y"]), _ptr(arr["z"]),
                   _ptr(arr["ux"]), _ptr(arr["uy"]), _ptr(arr["uz"]),
                   _ptr(arr["w"]), _ptr(pid), _ptr(ledger["emit"]),
                   _ptr(ledger["ll"]), ctypes.byref(cph), _ptr(cursor),
                   _ptr(tl["dN"]) if tl else None,
                   _ptr(tl["R"]) if tl else None,
                   _ptr(tl["x"]) if tl else None, _ptr(stats))
    if rc != 0:
        raise RuntimeError(f"orc_run failed: {rc}")
    for k in arr:
        state[k] = arr[k]
    m = int(cursor[0])
    photons = {k: v[:m] for k, v in ph.items()}
    order = np.lexsort((photons["step"], photons["pid"]))
    photons = {k: v[order] for k, v in photons.items()}
    out = {"photons": photons, "ledger": ledger,
           "stats": dict(zip(("records", "dropped", "dn_gt1", "clamped",
                              "chi_gt1", "wiggler_invalid"), (int(s) for s in stats)))}
    if tl is not None:
        out["trials"] = tl
    return out


def angular_histogram(nx, ny, nz, eps, weight, axis, ref, ntheta: int, nphi: int,
                      theta_max: float) -> np.ndarray:
    """Fig. 4: emitted energy (eps x weight) of photon records by direction,
    [theta][phi]: theta the angle from ``axis`` in ntheta equal bins over
    [0, theta_max], phi the azimuth around it from the component of ``ref``
    perpendicular to it (phi = pi/2 along axis x ref) in nphi equal bins over
    [0, 2 pi).  Records beyond theta_max are not counted.  FP64 throughout."""
    a = np.asarray(axis, dtype=np.float64)
    a = a / np.linalg.norm(a)
    r = np.asarray(ref, dtype=np.float64)
    e1 = r - (r @ a) * a
    e1 = e1 / np.linalg.norm(e1)
    e2 = np.cross(a, e1)
    n = np.stack([np.asarray(v, dtype=np.float64) for v in (nx, ny, nz)], 1)
    th = np.arccos(np.clip(n @ a, -1.0, 1.0))
    ph = np.arctan2(n @ e2, n @ e1)
    ph = np.where(ph < 0.0, ph + 2.0 * np.pi, ph)
    keep = th <= theta_max
    it = np.minimum((th * (ntheta / theta_max)).astype(np.int64), ntheta - 1)
    ip = np.clip((ph * (nphi / (2.0 * np.pi))).astype(np.int64), 0, nphi - 1)
    e = np.asarray(eps, dtype=np.float64) * np.asarray(weight, dtype=np.float64)
    h = np.zeros((ntheta, nphi))
    np.add.at(h, (it[keep], ip[keep]), e[keep])
    return h
