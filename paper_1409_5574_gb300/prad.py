"""ctypes binding of the prad C ABI (include/prad.h).

Argument marshalling only: every step of the particle path runs in the CUDA
kernels of ``_build/libprad.so``.  PyTorch provides device memory and streams.
There is no CPU fallback: if the library is missing or a call fails, this
module raises.

The function names mirror the C ABI (``prad_init``, ``prad_set_fields``,
``prad_push_emit``, ``prad_get_photons``, ``prad_energy_budget``, ...).
``Context`` bundles them for torch tensors.
"""
from __future__ import annotations

import ctypes
import math
import os
from typing import Dict, Optional, Sequence

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libprad.so")

# ---- constants mirrored from prad.h -------------------------------------
PRAD_OK, PRAD_ERR_ARG, PRAD_ERR_CUDA, PRAD_ERR_CAPACITY = 0, -1, -2, -3
PRAD_ERR_TIMEOUT, PRAD_ERR_STATE, PRAD_WARN_NAN = -4, -5, 1
PRAD_FP32, PRAD_FP64 = 0, 1
PRAD_SAMPLER_TABLE, PRAD_SAMPLER_MLP, PRAD_SAMPLER_MLP_FALLBACK = 0, 1, 2
PRAD_RR_OFF, PRAD_RR_LEDGER, PRAD_RR_APPLY = 0, 1, 2
PRAD_DIAG_WIGGLER = 1
PRAD_DIAG_ANGLE_SPREAD = 2
PRAD_HEFF_FIELD, PRAD_HEFF_MOMENTUM = 0, 1
PRAD_FIELD_CONST, PRAD_FIELD_PLANE_WAVE, PRAD_FIELD_YEE2D = 0, 1, 2

_i32, _i64, _u32, _u64, _dbl = (ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32,
                                 ctypes.c_uint64, ctypes.c_double)
_vp = ctypes.c_void_p


class prad_config(ctypes.Structure):
    _fields_ = [("precision", _i32), ("sampler", _i32), ("rr_mode", _i32),
                ("heff_form", _i32), ("dt", _dbl), ("omega_ref", _dbl),
                ("charge", _dbl), ("seed", _u64), ("ensemble", _u32),
                ("steps_per_launch", _i32), ("photon_capacity", _i64),
                ("max_particles", _i64), ("stream", _vp), ("block_size", _i32),
                ("blocks_per_sm", _i32), ("sort_interval", _i32), ("batch_chunk", _i32),
                ("use_graph", _i32), ("n_try", _i32), ("diagnostics", _i32),
                ("specialize", _i32), ("select_prob", _dbl)]


class prad_fields(ctypes.Structure):
    _fields_ = [("kind", _i32), ("dir", _i32), ("hand", _i32), ("periodic", _i32),
                ("E", _dbl * 3), ("B", _dbl * 3), ("a0", _dbl), ("lam", _dbl),
                ("phase0", _dbl), ("yee", _vp * 6), ("nx", _i32), ("ny", _i32),
                ("dx", _dbl), ("dy", _dbl), ("x0", _dbl), ("y0", _dbl)]


class prad_particles(ctypes.Structure):
    _fields_ = [("x", _vp), ("y", _vp), ("z", _vp), ("ux", _vp), ("uy", _vp),
                ("uz", _vp), ("w", _vp), ("pid", _vp), ("ledger_offset", _i64),
                ("pid0", _u32), ("pad0", _u32), ("t0", _i64)]


class prad_ensemble(ctypes.Structure):
    _fields_ = [("p", prad_particles), ("n", _i64), ("field", prad_fields),
                ("ensemble", _u32), ("pad0", _u32)]


class prad_tuning(ctypes.Structure):
    _fields_ = [("block_size", _i32), ("blocks_per_sm", _i32), ("batch_chunk", _i32),
                ("steps_per_launch", _i32), ("particle_steps_per_s", _dbl),
                ("candidates", _i32), ("pad0", _i32)]


class prad_photons(ctypes.Structure):
    _fields_ = [(n, _vp) for n in ("x", "y", "z", "nx", "ny", "nz", "eps",
                                   "weight", "pid", "step")]


class prad_stats(ctypes.Structure):
    _fields_ = [("records", _i64), ("dropped", _i64), ("dn_gt1", _i64),
                ("clamped", _i64), ("chi_gt1", _i64), ("mlp_fallback", _i64),
                ("nan_frozen", _i64), ("status", _i32), ("spec_launches", _i32),
                ("wiggler_invalid", _i64)]


# symbol -> (restype, argtypes); every function declared in include/prad.h
SIGNATURES = {
    "prad_init": (_i32, [ctypes.POINTER(_vp), ctypes.POINTER(prad_config)]),
    "prad_destroy": (_i32, [_vp]),
    "prad_last_error": (ctypes.c_char_p, [_vp]),
    "prad_set_fields": (_i32, [_vp, ctypes.POINTER(prad_fields)]),
    "prad_push_emit": (_i32, [_vp, ctypes.POINTER(prad_particles), _i64, _i32]),
    "prad_sort_by_tile": (_i32, [_vp, ctypes.POINTER(prad_particles), _i64]),
    "prad_push_emit_batch": (_i32, [_vp, ctypes.POINTER(prad_ensemble), _i32, _i32]),
    "prad_autotune_batch": (_i32, [_vp, ctypes.POINTER(prad_ensemble), _i32, _i32, _i64,
                                   ctypes.POINTER(prad_tuning)]),
    "prad_get_photons": (_i32, [_vp, ctypes.POINTER(prad_photons), _i64,
                                ctypes.POINTER(_i64), ctypes.POINTER(_i64), _i32, _i32]),
    "prad_angular_histogram": (_i32, [_vp, ctypes.POINTER(_dbl), ctypes.POINTER(_dbl), _i32,
                                      _i32, _dbl, ctypes.POINTER(_dbl)]),
    "prad_energy_budget": (_i32, [_vp, ctypes.POINTER(_dbl), ctypes.POINTER(_dbl),
                                  ctypes.POINTER(prad_stats)]),
    "prad_get_ledger": (_i32, [_vp, _vp, _vp, _i64, _i64, _i32]),
    "prad_reset": (_i32, [_vp]),
    "prad_mlp_set_weights": (_i32, [_vp, _vp, _i64]),
    "prad_mlp_get_weights": (_i32, [_vp, _vp, _i64]),
    "prad_mlp_train": (_i32, [_vp, _i64, _i32, ctypes.c_float, _u64,
                              ctypes.POINTER(ctypes.c_float)]),
    "prad_mlp_grad": (_i32, [_vp, _vp, _i64, _vp, ctypes.POINTER(_dbl)]),
    "prad_mlp_eval": (_i32, [_vp, _vp, _vp, _i64]),
    "prad_mlp_wait_selftest": (_i32, [_vp]),
    "prad_batch_balance": (_i32, [_vp, ctypes.POINTER(_dbl), ctypes.POINTER(_i32)]),
    "prad_ginv_eval": (_i32, [_vp, _vp, _vp, _i64]),
    "prad_angle_eval": (_i32, [_vp, _vp, _vp, _vp, _i64]),
    "prad_angle_table": (_i32, [_vp, _i64]),
    "prad_ledger_totals_noalloc": (_i32, [_vp, _vp, _i64, _vp, _vp]),
    "prad_ledger_totals_noalloc_error": (ctypes.c_char_p, []),
    "prad_philox": (_i32, [_vp, _vp, _u32, _u32, _vp, _i64]),
    "prad_eval_sampler": (_i32, [_vp, _vp, _vp, _vp, _i64]),
}

_lib = None


class PradError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"prad error {code}: {msg}")
        self.code = code


def load_library(path: Optional[str] = None) -> ctypes.CDLL:
    """Load libprad.so (raises OSError if it has not been built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or os.environ.get("PRAD_LIBRARY") or LIB_PATH
    if not os.path.exists(p):
        raise OSError(f"libprad.so not built ({p}); run "
                      "python -c 'import __graft_entry__ as g; g.build()'")
    lib = ctypes.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


def _check(rc: int, handle=None) -> int:
    if rc < 0:
        msg = load_library().prad_last_error(handle).decode(errors="replace")
        raise PradError(rc, msg)
    return rc


# ---- thin wrappers with the C names ------------------------------------
def prad_init(cfg: prad_config) -> int:
    h = _vp()
    _check(load_library().prad_init(ctypes.byref(h), ctypes.byref(cfg)))
    return h.value


def prad_destroy(h) -> None:
    _check(load_library().prad_destroy(h), h)


def prad_set_fields(h, f: prad_fields) -> None:
    _check(load_library().prad_set_fields(h, ctypes.byref(f)), h)


def prad_push_emit(h, p: prad_particles, n: int, nsteps: int) -> int:
    return _check(load_library().prad_push_emit(h, ctypes.byref(p), n, nsteps), h)


def prad_sort_by_tile(h, p: prad_particles, n: int) -> int:
    return _check(load_library().prad_sort_by_tile(h, ctypes.byref(p), n), h)


def prad_push_emit_batch(h, ens, nsteps: int) -> int:
    arr = (prad_ensemble * len(ens))(*ens)
    return _check(load_library().prad_push_emit_batch(h, arr, len(ens), nsteps), h)


def prad_autotune_batch(h, ens, probe_steps: int, sample: int) -> dict:
    arr = (prad_ensemble * len(ens))(*ens)
    t = prad_tuning()
    _check(load_library().prad_autotune_batch(h, arr, len(ens), probe_steps, sample,
                                              ctypes.byref(t)), h)
    return {k: getattr(t, k) for k, _ in prad_tuning._fields_ if k != "pad0"}


def prad_get_photons(h, out: Optional[prad_photons], cap: int, drain: bool,
                     out_on_device: bool):
    n_out, n_drop = _i64(), _i64()
    _check(load_library().prad_get_photons(
        h, ctypes.byref(out) if out is not None else None, cap, ctypes.byref(n_out),
        ctypes.byref(n_drop), int(drain), int(out_on_device)), h)
    return n_out.value, n_drop.value


def prad_angular_histogram(h, axis, ref, ntheta: int, nphi: int, theta_max: float):
    """Emitted energy of the held records by direction (ntheta x nphi numpy
    array, [theta][phi])."""
    import numpy as np
    out = np.zeros((ntheta, nphi), dtype=np.float64)
    ax = (_dbl * 3)(*[float(v) for v in axis])
    rf = (_dbl * 3)(*[float(v) for v in ref])
    _check(load_library().prad_angular_histogram(
        h, ax, rf, ntheta, nphi, float(theta_max),
        out.ctypes.data_as(ctypes.POINTER(_dbl))), h)
    return out


def prad_energy_budget(h):
    e, r, s = _dbl(), _dbl(), prad_stats()
    rc = _check(load_library().prad_energy_budget(h, ctypes.byref(e), ctypes.byref(r),
                                                  ctypes.byref(s)), h)
    stats = {k: getattr(s, k) for k, _ in prad_stats._fields_ if k != "pad0"}
    stats["rc"] = rc
    return e.value, r.value, stats


def prad_get_ledger(h, emit_ptr, ll_ptr, offset: int, n: int, on_device: bool) -> None:
    _check(load_library().prad_get_ledger(h, emit_ptr, ll_ptr, offset, n, int(on_device)), h)


def prad_reset(h) -> None:
    _check(load_library().prad_reset(h), h)


PRAD_MLP_NUM_PARAMS = 4481


def prad_mlp_set_weights(h, params) -> None:
    import numpy as np
    p = np.ascontiguousarray(params, dtype=np.float32)
    _check(load_library().prad_mlp_set_weights(h, p.ctypes.data, p.size), h)


def prad_mlp_get_weights(h):
    import numpy as np
    p = np.zeros(PRAD_MLP_NUM_PARAMS, dtype=np.float32)
    _check(load_library().prad_mlp_get_weights(h, p.ctypes.data, p.size), h)
    return p


def prad_mlp_train(h, steps: int, batch: int, lr: float, seed: int) -> float:
    loss = ctypes.c_float()
    _check(load_library().prad_mlp_train(h, steps, batch, lr, seed, ctypes.byref(loss)), h)
    return loss.value


def prad_mlp_grad(h, samples_ptr, n: int):
    import numpy as np
    g = np.zeros(PRAD_MLP_NUM_PARAMS, dtype=np.float32)
    loss = _dbl()
    _check(load_library().prad_mlp_grad(h, samples_ptr, n, g.ctypes.data, ctypes.byref(loss)), h)
    return g, loss.value


def prad_mlp_eval(h, in_ptr, out_ptr, n: int) -> None:
    _check(load_library().prad_mlp_eval(h, in_ptr, out_ptr, n), h)


def prad_batch_balance(h):
    """(load-balance efficiency, CTA count) of the last batched call."""
    eff, n = _dbl(), _i32()
    _check(load_library().prad_batch_balance(h, ctypes.byref(eff), ctypes.byref(n)), h)
    return eff.value, n.value


def prad_mlp_wait_selftest(h) -> int:
    """Status code of the bounded-wait self-test (PRAD_ERR_TIMEOUT expected)."""
    return load_library().prad_mlp_wait_selftest(h)


def prad_ginv_eval(h, r_ptr, out_ptr, n: int) -> None:
    _check(load_library().prad_ginv_eval(h, r_ptr, out_ptr, n), h)


PRAD_ANG_NL, PRAD_ANG_NV = 225, 257
PRAD_ANG_LX0, PRAD_ANG_LX1, PRAD_ANG_VMAX = -18.420680743952367, 3.6888794541139363, 4.8


def prad_angle_table():
    """The angular spread's table (PRAD_ANG_NL x PRAD_ANG_NV numpy float32),
    built on the host by the library; no device needed."""
    import numpy as np
    out = np.empty((PRAD_ANG_NL, PRAD_ANG_NV), dtype=np.float32)
    _check(load_library().prad_angle_table(out.ctypes.data_as(ctypes.c_void_p), out.size), None)
    return out


def prad_angle_eval(h, x_ptr, words_ptr, out_ptr, n: int) -> None:
    _check(load_library().prad_angle_eval(h, x_ptr, words_ptr, out_ptr, n), h)


def prad_ledger_totals_noalloc(emit_ptr, rr_ptr, n: int, out_ptr, stream_ptr=None) -> None:
    """Kahan totals of two caller-owned device FP64 arrays into a caller-owned
    device array of 2 doubles, without any device allocation."""
    L = load_library()
    rc = L.prad_ledger_totals_noalloc(emit_ptr, rr_ptr, n, out_ptr, stream_ptr)
    if rc < 0:
        raise PradError(rc, L.prad_ledger_totals_noalloc_error().decode(errors="replace"))


def prad_philox(h, ctr_ptr, k0: int, k1: int, out_ptr, n: int) -> None:
    _check(load_library().prad_philox(h, ctr_ptr, k0, k1, out_ptr, n), h)


def prad_eval_sampler(h, words_ptr, x_ptr, g_ptr, n: int) -> None:
    _check(load_library().prad_eval_sampler(h, words_ptr, x_ptr, g_ptr, n), h)


# ---- torch convenience ---------------------------------------------------
def _torch():
    import torch  # noqa: WPS433 (torch is only plumbing: memory and streams)
    return torch


def _ptr(t) -> Optional[int]:
    return None if t is None else t.data_ptr()


class Context:
    """A prad context with torch tensors as the particle and photon storage.

    ``problem`` keys follow ``workloads.Workload.problem_kwargs()``.
    ``specialize=True`` sets ``prad_config.specialize``: the standard FP32
    plane-wave and Yee steps run through kernels NVRTC compiles for this
    context's constants (same results; ``energy_budget()[2]["spec_launches"]``
    counts their launches).
    """

    def __init__(self, problem: Dict, precision: int = PRAD_FP32,
                 photon_capacity: int = 1 << 20, max_particles: int = 1 << 20,
                 steps_per_launch: int = 1, stream=None, block_size: int = 0,
                 blocks_per_sm: int = 0, sampler: int = PRAD_SAMPLER_TABLE,
                 ensemble: int = 0, sort_interval: int = 0, batch_chunk: int = 0,
                 use_graph: bool = False, n_try: int = 1, select_prob: float = 1.0,
                 diagnostics: int = 0, specialize: bool = False):
        torch = _torch()
        if not torch.cuda.is_available():
            raise RuntimeError("prad needs a CUDA device")
        self.torch = torch
        self.problem = dict(problem)
        self.precision = precision
        self.dtype = torch.float32 if precision == PRAD_FP32 else torch.float64
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        cfg = prad_config()
        cfg.precision = precision
        cfg.sampler = sampler
        cfg.rr_mode = problem.get("rr_mode", PRAD_RR_LEDGER)
        cfg.heff_form = problem.get("heff_form", PRAD_HEFF_FIELD)
        cfg.dt = problem["dt"]
        cfg.omega_ref = problem["omega_ref"]
        cfg.charge = problem.get("charge", -1.0)
        cfg.seed = int(problem.get("seed", 1))
        cfg.ensemble = int(ensemble or problem.get("ensemble", 0))
        cfg.steps_per_launch = steps_per_launch
        cfg.photon_capacity = photon_capacity
        cfg.max_particles = max_particles
        cfg.stream = self.stream.cuda_stream
        cfg.block_size = block_size
        cfg.blocks_per_sm = blocks_per_sm
        cfg.sort_interval = sort_interval
        cfg.batch_chunk = batch_chunk
        cfg.use_graph = int(use_graph)
        cfg.n_try = n_try
        cfg.select_prob = select_prob
        cfg.diagnostics = diagnostics
        cfg.specialize = int(specialize)
        self.cfg = cfg
        self.capacity = photon_capacity
        self.max_particles = max_particles
        self.h = prad_init(cfg)
        self._yee_keep = None
        self.set_fields(problem)

    # -- fields ------------------------------------------------------------
    @staticmethod
    def make_fields(problem: Dict) -> prad_fields:
        """prad_fields of an analytic (CONST or PLANE_WAVE) problem dict."""
        f = prad_fields()
        f.kind = problem.get("field_kind", PRAD_FIELD_CONST)
        f.dir = int(problem.get("direction", 1))
        f.hand = int(problem.get("hand", 1))
        f.periodic = 1
        for k in range(3):
            f.E[k] = problem.get("E", (0, 0, 0))[k]
            f.B[k] = problem.get("B", (0, 0, 0))[k]
        f.a0 = problem.get("a0", 0.0)
        f.lam = problem.get("lam", 0.8e-6)
        f.phase0 = problem.get("phase0", 0.0)
        return f

    def set_fields(self, problem: Dict) -> None:
        torch = self.torch
        f = prad_fields()
        f.kind = problem.get("field_kind", PRAD_FIELD_CONST)
        f.dir = int(problem.get("direction", 1))
        f.hand = int(problem.get("hand", 1))
        f.periodic = 1
        for k in range(3):
            f.E[k] = problem.get("E", (0, 0, 0))[k]
            f.B[k] = problem.get("B", (0, 0, 0))[k]
        f.a0 = problem.get("a0", 0.0)
        f.lam = problem.get("lam", 0.8e-6)
        f.phase0 = problem.get("phase0", 0.0)
        if f.kind == PRAD_FIELD_YEE2D:
            planes = problem["yee"]
            dev = [p if (hasattr(p, "is_cuda") and p.is_cuda)
                   else torch.as_tensor(p, dtype=torch.float32).cuda().contiguous()
                   for p in planes]
            self._yee_keep = dev
            for k in range(6):
                f.yee[k] = dev[k].data_ptr()
            f.ny, f.nx = dev[0].shape
            f.dx, f.dy = problem["dx"], problem["dy"]
            f.x0, f.y0 = problem.get("x0", 0.0), problem.get("y0", 0.0)
        self.fields = f
        prad_set_fields(self.h, f)

    # -- state ---------------------------------------------------------------
    def to_device(self, state: Dict, device="cuda", with_pid: bool = False,
                  pid0: int = 0) -> Dict:
        """Copy a state dict to the device in the context precision; with
        ``with_pid`` add an int32 id array pid0 + i (ids move with particles
        that a tile sort reorders)."""
        torch = self.torch
        out = {k: torch.as_tensor(v, dtype=self.dtype).to(device).contiguous()
               for k, v in state.items()}
        if self.fields.kind == PRAD_FIELD_YEE2D:
            out.pop("z", None)
        if with_pid:
            n = out["x"].numel()
            out["pid"] = (torch.arange(n, dtype=torch.int64, device=device) + pid0).to(torch.int32)
        return out

    def _particles(self, st: Dict, t0: int, pid0: int, ledger_offset: int) -> prad_particles:
        p = prad_particles()
        p.x, p.y = _ptr(st["x"]), _ptr(st["y"])
        p.z = _ptr(st.get("z"))
        p.ux, p.uy, p.uz, p.w = _ptr(st["ux"]), _ptr(st["uy"]), _ptr(st["uz"]), _ptr(st["w"])
        p.pid = _ptr(st.get("pid"))
        p.ledger_offset = ledger_offset
        p.pid0 = pid0
        p.t0 = t0
        return p

    def push_emit(self, st: Dict, nsteps: int, t0: int = 0, pid0: int = 0,
                  ledger_offset: int = 0) -> None:
        """Advance the particles of ``st`` (torch tensors x y z ux uy uz w and an
        optional int32 ``pid``; ``z`` may be absent for the Yee grid)."""
        n = st["x"].numel()
        prad_push_emit(self.h, self._particles(st, t0, pid0, ledger_offset), n, nsteps)

    def ensembles(self, states, problems, t0: int = 0, pid0s=None, ledger_offsets=None,
                  ensemble_ids=None):
        """prad_ensemble structs for lists of device states and problem dicts
        (the default pid0 / ledger offsets are the running particle counts)."""
        out, off = [], 0
        for k, (st, pb) in enumerate(zip(states, problems)):
            n = st["x"].numel()
            e = prad_ensemble()
            e.p = self._particles(st, t0, off if pid0s is None else pid0s[k],
                                  off if ledger_offsets is None else ledger_offsets[k])
            e.n = n
            e.field = self.make_fields(pb)
            e.ensemble = k if ensemble_ids is None else ensemble_ids[k]
            out.append(e)
            off += n
        return out

    def push_emit_batch(self, ens, nsteps: int) -> None:
        prad_push_emit_batch(self.h, ens, nsteps)

    def autotune_batch(self, ens, probe_steps: int = 20, sample: int = 4096) -> dict:
        return prad_autotune_batch(self.h, ens, probe_steps, sample)

    def sort_by_tile(self, st: Dict, pid0: int = 0, ledger_offset: int = 0) -> None:
        n = st["x"].numel()
        prad_sort_by_tile(self.h, self._particles(st, 0, pid0, ledger_offset), n)

    def photons(self, drain: bool = False, on_device: bool = True,
                cap: Optional[int] = None) -> Dict:
        """Copy the held photon records into new torch tensors."""
        torch = self.torch
        held, dropped = prad_get_photons(self.h, None, 0, False, True)
        m = held if cap is None else min(held, cap)
        kw = dict(device="cuda") if on_device else dict(pin_memory=m > 0)
        out = {k: torch.empty(m, dtype=torch.float32, **kw)
               for k in ("x", "y", "z", "nx", "ny", "nz", "eps", "weight")}
        out["pid"] = torch.empty(m, dtype=torch.int32, **kw)
        out["step"] = torch.empty(m, dtype=torch.int32, **kw)
        ph = prad_photons()
        for k, v in out.items():
            setattr(ph, k, v.data_ptr() if m else None)
        held, dropped = prad_get_photons(self.h, ph if m else None, m, drain, on_device)
        out["dropped"] = dropped
        return out

    def batch_balance(self):
        """Load balance (mean / max CTA busy time) of the last batched call."""
        return prad_batch_balance(self.h)

    def drain(self):
        return prad_get_photons(self.h, None, 0, True, True)

    def energy_budget(self):
        return prad_energy_budget(self.h)

    def angular_histogram(self, axis=(1.0, 0.0, 0.0), ref=(0.0, 1.0, 0.0), ntheta: int = 45,
                          nphi: int = 72, theta_max: float = 0.5 * 3.141592653589793):
        return prad_angular_histogram(self.h, axis, ref, ntheta, nphi, theta_max)

    def ledger(self, offset: int = 0, n: Optional[int] = None):
        torch = self.torch
        n = self.max_particles - offset if n is None else n
        e = torch.empty(n, dtype=torch.float64, device="cuda")
        l = torch.empty(n, dtype=torch.float64, device="cuda")
        prad_get_ledger(self.h, e.data_ptr(), l.data_ptr(), offset, n, True)
        return e, l

    def reset(self) -> None:
        prad_reset(self.h)

    # -- learned sampler -------------------------------------------------------
    def mlp_train(self, steps: int, batch: int = 65536, lr: float = 3e-3,
                  seed: int = 7) -> float:
        return prad_mlp_train(self.h, steps, batch, lr, seed)

    def mlp_weights(self):
        return prad_mlp_get_weights(self.h)

    def mlp_set_weights(self, params) -> None:
        prad_mlp_set_weights(self.h, params)

    def mlp_eval(self, r, gamma, wdt):
        """ln x of the network for torch/numpy arrays r, gamma, omega_c dt."""
        torch = self.torch
        inp = torch.stack([torch.as_tensor(v, dtype=torch.float32).flatten()
                           for v in (r, gamma, wdt)], 1).cuda().contiguous()
        out = torch.empty(inp.shape[0], dtype=torch.float32, device="cuda")
        prad_mlp_eval(self.h, inp.data_ptr(), out.data_ptr(), inp.shape[0])
        return out

    def mlp_grad(self, r, gamma, wdt, lnx_target):
        torch = self.torch
        smp = torch.stack([torch.as_tensor(v, dtype=torch.float32).flatten()
                           for v in (r, gamma, wdt, lnx_target)], 1).cuda().contiguous()
        return prad_mlp_grad(self.h, smp.data_ptr(), smp.shape[0])

    def ginv(self, r):
        torch = self.torch
        rr = torch.as_tensor(r, dtype=torch.float32).flatten().cuda().contiguous()
        out = torch.empty_like(rr)
        prad_ginv_eval(self.h, rr.data_ptr(), out.data_ptr(), rr.numel())
        return out

    def angle_eval(self, x, words):
        """psi = gamma theta of the angular spread (PRAD_DIAG_ANGLE_SPREAD)
        for photon frequencies x (omega/omega_c) and Philox word pairs
        words (n x 2, uint32)."""
        import numpy as np
        torch = self.torch
        xx = torch.as_tensor(x, dtype=torch.float32).flatten().cuda().contiguous()
        ww = torch.as_tensor(np.ascontiguousarray(words, dtype=np.uint32).view(np.int32)
                             ).flatten().cuda().contiguous()
        if ww.numel() != 2 * xx.numel():
            raise ValueError("angle_eval: words must hold two words per x")
        out = torch.empty_like(xx)
        prad_angle_eval(self.h, xx.data_ptr(), ww.data_ptr(), out.data_ptr(), xx.numel())
        return out

    def close(self) -> None:
        if getattr(self, "h", None):
            prad_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
