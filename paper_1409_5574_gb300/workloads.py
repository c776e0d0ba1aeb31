"""Seeded synthetic workloads shaped like the paper's validation runs.

This module only builds inputs: SI problem descriptions and initial particle
states (numpy, seeded). It holds none of the method's arithmetic and imports
nothing else from this package, so the GPU library and the CPU oracle can both
consume what it produces.

Normalised units of the state arrays: length in c/omega_ref, momentum
u = p/(m_e c). Field planes of the Yee workload are in m_e c omega_ref / e
(E) and m_e omega_ref / e (B).

Workloads (the paper's constant-field check of its Comparison section and the
laser-plasma regime of its wakefield run, made synthetic):

* ``const_b``      10^4 electrons, gamma ~ U[100, 1000], isotropic momenta at
                   the origin, B = 10^4 T along z, E = 0, dt = 1e-3 of the
                   gyro-period at gamma = 100, 1000 steps, FP64.
* ``plane_wave``   2^20 electrons, gamma = 1000 along -x with 1% Gaussian
                   momentum spread, x ~ U[0, lambda), counter-propagating
                   circularly polarised wave, lambda = 0.8 um, a0 in
                   {100, 300, 500}, 200 steps per period for 20 periods.
* ``yee2d``        4096^2 staggered FP32 planes holding a standing-wave
                   snapshot (a0 = 300) plus 1% Gaussian noise, dx = lambda/32,
                   16M electrons uniform in the central 1024^2 cells,
                   gamma log-uniform in [10, 3000], isotropic, 1000 steps.
* ``ensembles``    many independent ensembles of log-uniform size with a0
                   uniform in [50, 500], plane-wave or constant-B fields.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Dict, List, Optional

import numpy as np

# SI constants used to state the workloads (CODATA 2018)
C_LIGHT = 299792458.0
Q_E = 1.602176634e-19
M_E = 9.1093837015e-31

FIELD_CONST, FIELD_PLANE_WAVE, FIELD_YEE2D = 0, 1, 2
RR_OFF, RR_LEDGER, RR_APPLY = 0, 1, 2
HEFF_FIELD, HEFF_MOMENTUM = 0, 1


@dataclass
class Workload:
    """An SI problem description plus a seeded initial state (float64)."""
    name: str
    omega_ref: float
    dt: float
    nsteps: int
    seed: int = 1
    charge: float = -1.0
    rr_mode: int = RR_LEDGER
    heff_form: int = HEFF_FIELD
    field_kind: int = FIELD_CONST
    dims: int = 3
    E: tuple = (0.0, 0.0, 0.0)
    B: tuple = (0.0, 0.0, 0.0)
    a0: float = 0.0
    lam: float = 0.8e-6
    phase0: float = 0.0
    direction: int = 1
    hand: int = 1
    yee: Optional[List[np.ndarray]] = None
    dx: float = 1.0
    dy: float = 1.0
    x0: float = 0.0
    y0: float = 0.0
    state: Dict[str, np.ndarray] = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.state["x"].size)

    def problem_kwargs(self) -> dict:
        """Keyword arguments shared by the oracle Problem and the GPU config."""
        return dict(omega_ref=self.omega_ref, dt=self.dt, charge=self.charge,
                    seed=self.seed, rr_mode=self.rr_mode,
                    heff_form=self.heff_form, field_kind=self.field_kind,
                    dims=self.dims, E=tuple(self.E), B=tuple(self.B),
                    a0=self.a0, lam=self.lam, phase0=self.phase0,
                    direction=self.direction, hand=self.hand, yee=self.yee,
                    dx=self.dx, dy=self.dy, x0=self.x0, y0=self.y0)

    def subset(self, idx: np.ndarray) -> "Workload":
        w = Workload(**{k: getattr(self, k) for k in self.__dataclass_fields__
                        if k != "state"})
        w.state = {k: np.array(v[idx]) for k, v in self.state.items()}
        return w

    def copy_state(self) -> Dict[str, np.ndarray]:
        return {k: np.array(v) for k, v in self.state.items()}


def _isotropic(rng: np.random.Generator, n: int) -> np.ndarray:
    v = rng.standard_normal((n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v


def const_b(n: int = 10_000, nsteps: int = 1000, seed: int = 1,
            B_tesla: float = 1.0e4, rr_mode: int = RR_LEDGER) -> Workload:
    omega_ref = Q_E * B_tesla / M_E            # cyclotron frequency at gamma=1
    dt = 1.0e-3 * 2.0 * math.pi * 100.0 / omega_ref
    rng = np.random.default_rng(seed)
    gamma = rng.uniform(100.0, 1000.0, n)
    umag = np.sqrt(gamma * gamma - 1.0)
    u = _isotropic(rng, n) * umag[:, None]
    st = dict(x=np.zeros(n), y=np.zeros(n), z=np.zeros(n),
              ux=u[:, 0].copy(), uy=u[:, 1].copy(), uz=u[:, 2].copy(),
              w=np.ones(n))
    return Workload(name=f"const_b n={n} B={B_tesla:g}T", omega_ref=omega_ref,
                    dt=dt, nsteps=nsteps, seed=seed, rr_mode=rr_mode,
                    field_kind=FIELD_CONST, B=(0.0, 0.0, B_tesla), state=st)


def plane_wave(a0: float = 500.0, n: int = 1 << 20, periods: int = 20,
               steps_per_period: int = 200, seed: int = 1,
               lam: float = 0.8e-6, gamma0: float = 1000.0,
               spread: float = 0.01, rr_mode: int = RR_APPLY) -> Workload:
    omega_ref = 2.0 * math.pi * C_LIGHT / lam
    dt = (2.0 * math.pi / omega_ref) / steps_per_period
    rng = np.random.default_rng(seed)
    u0 = math.sqrt(gamma0 * gamma0 - 1.0)
    u = np.zeros((n, 3))
    u[:, 0] = -u0
    u += rng.standard_normal((n, 3)) * (spread * u0)
    x = rng.uniform(0.0, 2.0 * math.pi, n)   # [0, lambda) in c/omega units
    st = dict(x=x, y=np.zeros(n), z=np.zeros(n), ux=u[:, 0].copy(),
              uy=u[:, 1].copy(), uz=u[:, 2].copy(), w=np.ones(n))
    return Workload(name=f"plane_wave a0={a0:g} n={n}", omega_ref=omega_ref,
                    dt=dt, nsteps=periods * steps_per_period, seed=seed,
                    rr_mode=rr_mode, field_kind=FIELD_PLANE_WAVE, a0=a0,
                    lam=lam, direction=1, hand=1, state=st)


def yee_planes(nx: int, ny: int, a0: float, dxn: float, rng,
               noise: float = 0.01) -> List[np.ndarray]:
    """Standing-wave snapshot at omega t = pi/4 on the staggered 2D grid.

    E_y = E0 sin(k x) cos(pi/4), B_z = E0 cos(k x) sin(pi/4) (normalised,
    k = 1 in c/omega units), each component sampled at its own staggered
    location, plus N(0, (noise E0)^2) on every value of all six planes.
    """
    E0 = a0
    i = np.arange(nx, dtype=np.float64)
    xe = i * dxn            # Ey node x
    xb = (i + 0.5) * dxn    # Bz node x
    planes = []
    for comp in range(6):
        p = (rng.standard_normal((ny, nx), dtype=np.float32)
             * np.float32(noise * E0))
        if comp == 1:
            p += (E0 * np.sin(xe) * math.cos(math.pi / 4)).astype(np.float32)[None, :]
        if comp == 5:
            p += (E0 * np.cos(xb) * math.sin(math.pi / 4)).astype(np.float32)[None, :]
        planes.append(np.ascontiguousarray(p))
    return planes


def yee2d(n_grid: int = 4096, slab: int = 1024, ppc: int = 16,
          nsteps: int = 1000, a0: float = 300.0, seed: int = 1,
          lam: float = 0.8e-6, n_particles: Optional[int] = None,
          rr_mode: int = RR_APPLY, with_grid: bool = True) -> Workload:
    omega_ref = 2.0 * math.pi * C_LIGHT / lam
    dt = (2.0 * math.pi / omega_ref) / 200.0
    dxn = 2.0 * math.pi / 32.0
    rng = np.random.default_rng(seed)
    planes = yee_planes(n_grid, n_grid, a0, dxn, rng) if with_grid else None
    n = n_particles if n_particles is not None else slab * slab * ppc
    lo = (n_grid - slab) // 2
    x = (lo + rng.uniform(0.0, slab, n)) * dxn
    y = (lo + rng.uniform(0.0, slab, n)) * dxn
    gamma = np.exp(rng.uniform(math.log(10.0), math.log(3000.0), n))
    u = _isotropic(rng, n) * np.sqrt(gamma * gamma - 1.0)[:, None]
    st = dict(x=x, y=y, z=np.zeros(n), ux=u[:, 0].copy(), uy=u[:, 1].copy(),
              uz=u[:, 2].copy(), w=np.ones(n))
    return Workload(name=f"yee2d {n_grid}^2 n={n}", omega_ref=omega_ref,
                    dt=dt, nsteps=nsteps, seed=seed, rr_mode=rr_mode,
                    field_kind=FIELD_YEE2D, dims=2, a0=a0, lam=lam,
                    yee=planes, dx=dxn, dy=dxn, x0=0.0, y0=0.0, state=st)


@dataclass
class EnsembleSet:
    """Independent ensembles of uneven size for the batched launch."""
    workloads: List[Workload]

    @property
    def sizes(self) -> np.ndarray:
        return np.array([w.n for w in self.workloads], dtype=np.int64)


def ensembles(count: int = 256, nmin: int = 1_000, nmax: int = 1_000_000,
              a0_range=(50.0, 500.0), nsteps: int = 500, seed: int = 1,
              lam: float = 0.8e-6) -> EnsembleSet:
    """Ensemble sizes log-uniform in [nmin, nmax], a0 ~ U(a0_range); each
    ensemble is a plane wave or a constant B of the same a0 (B = a0 m omega/e),
    chosen by a seeded coin."""
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(math.log(nmin), math.log(nmax), count)).astype(np.int64)
    a0s = rng.uniform(a0_range[0], a0_range[1], count)
    kinds = rng.integers(0, 2, count)
    out = []
    for e in range(count):
        if kinds[e] == 0:
            w = plane_wave(a0=float(a0s[e]), n=int(sizes[e]), periods=1,
                           steps_per_period=200, seed=seed + 1000 + e, lam=lam)
        else:
            omega_ref = 2.0 * math.pi * C_LIGHT / lam
            Bt = a0s[e] * M_E * omega_ref / Q_E
            r2 = np.random.default_rng(seed + 1000 + e)
            n = int(sizes[e])
            gamma = r2.uniform(100.0, 1000.0, n)
            u = _isotropic(r2, n) * np.sqrt(gamma * gamma - 1.0)[:, None]
            st = dict(x=np.zeros(n), y=np.zeros(n), z=np.zeros(n),
                      ux=u[:, 0].copy(), uy=u[:, 1].copy(), uz=u[:, 2].copy(),
                      w=np.ones(n))
            w = Workload(name=f"ens{e} const_b", omega_ref=omega_ref,
                         dt=(2.0 * math.pi / omega_ref) / 200.0, nsteps=nsteps,
                         seed=seed, rr_mode=RR_APPLY, field_kind=FIELD_CONST,
                         B=(0.0, 0.0, float(Bt)), state=st)
        w.nsteps = nsteps
        w.seed = seed
        out.append(w)
    return EnsembleSet(out)
