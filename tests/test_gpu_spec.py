"""Run-time specialised step kernels (prad_config.specialize = 1) against
the ahead-of-time kernels, through the C ABI.

The specialised kernels are the same source compiled by NVRTC with the
context's constants as literals, so for every launch form they select
(fused multi-step launches; one-step launches, dense and with explicit
ids; the four plane-wave sign variants; a different seed, ensemble and
field amplitude; the learned samplers; the Yee grid's plain and tile-staged
kernels) the particle state, the photon records and the counters
must be the same bits, and the per-particle ledgers the same up to the
grouping of the FP64 atomic adds.  Launches outside the standard
configuration (the LL ledger mode, FP64) keep the ahead-of-time kernels.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_1409_5574_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_1409_5574_gb300 import prad


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    prad.load_library()


def _run(wl, nsteps, steps_per_launch, specialize, with_pid=False, precision=None,
         weights=None, **kw):
    precision = prad.PRAD_FP32 if precision is None else precision
    ctx = prad.Context(wl.problem_kwargs(), precision=precision, photon_capacity=1 << 20,
                       max_particles=wl.n, steps_per_launch=steps_per_launch,
                       specialize=specialize, **kw)
    if weights is not None:
        ctx.mlp_set_weights(weights)
    st = ctx.to_device(wl.state, with_pid=with_pid)
    ctx.push_emit(st, nsteps, t0=5)
    torch.cuda.synchronize()
    ph = ctx.photons(on_device=False)
    e, l, stats = ctx.energy_budget()
    le, ll = ctx.ledger()
    out = dict(state={k: v.cpu().numpy().copy() for k, v in st.items() if k != "pid"},
               ph={k: (v.numpy().copy() if hasattr(v, "numpy") else v) for k, v in ph.items()},
               e=e, l=l, stats=stats, le=le.cpu().numpy(), ll=ll.cpu().numpy())
    ctx.close()
    return out


def _photon_table(ph):
    key = ph["pid"].astype(np.int64) * 2**32 + ph["step"].astype(np.int64)
    names = ("x", "y", "z", "nx", "ny", "nz", "eps", "weight")
    o = np.lexsort(tuple(ph[k] for k in reversed(names)) + (key,))
    return key[o], np.stack([ph[k][o] for k in names], 1)


def _same(a, b):
    for k in a["state"]:
        np.testing.assert_array_equal(a["state"][k], b["state"][k], err_msg=k)
    np.testing.assert_allclose(a["le"], b["le"], rtol=1e-13, atol=0)
    np.testing.assert_allclose(a["ll"], b["ll"], rtol=1e-13, atol=0)
    ka, ta = _photon_table(a["ph"])
    kb, tb = _photon_table(b["ph"])
    np.testing.assert_array_equal(ka, kb)
    np.testing.assert_array_equal(ta, tb)
    for k in ("records", "dropped", "dn_gt1", "clamped", "chi_gt1", "nan_frozen", "status"):
        assert a["stats"][k] == b["stats"][k], k


def _wave(n=20000 + 37, a0=400.0, seed=11, hand=1, direction=-1):
    wl = W.plane_wave(a0=a0, n=n, seed=seed)
    wl.hand, wl.direction = hand, direction
    wl.state["ux"] = wl.state["ux"] * direction
    return wl


@pytest.mark.parametrize("form", ["fused", "one_step", "one_step_pid"])
def test_specialised_equals_compiled_in(form):
    wl = _wave()
    spl = 8 if form == "fused" else 1
    pid = form == "one_step_pid"
    base = _run(wl, 24, spl, False, with_pid=pid)
    spec = _run(wl, 24, spl, True, with_pid=pid)
    _same(base, spec)
    assert base["stats"]["records"] > 1000
    assert base["stats"]["spec_launches"] == 0
    assert spec["stats"]["spec_launches"] == (3 if form == "fused" else 24)


@pytest.mark.parametrize("hand,direction", [(1, 1), (-1, 1), (-1, -1)])
def test_specialised_sign_variants(hand, direction):
    wl = _wave(n=4096 + 5, a0=250.0, seed=3, hand=hand, direction=direction)
    for spl in (1, 6):
        _same(_run(wl, 12, spl, False), _run(wl, 12, spl, True))


def test_specialised_other_constants():
    """Another seed, ensemble and amplitude compile other literals; the
    tail launch of 10 steps in launches of 4 (4, 4, 2) uses the fused form
    throughout, and 9 steps in launches of 4 end with a one-step launch."""
    wl = _wave(n=3000, a0=120.0, seed=77)
    wl.seed = 987654321
    for nsteps in (10, 9):
        a = _run(wl, nsteps, 4, False, ensemble=5)
        b = _run(wl, nsteps, 4, True, ensemble=5)
        _same(a, b)
        assert b["stats"]["spec_launches"] == 3


@pytest.mark.parametrize("sampler", ["mlp", "mlp_fallback"])
def test_specialised_learned_sampler(sampler):
    """The learned samplers' step kernels (records finished by the
    tensor-core network) with any fixed weights: the same bits."""
    from oracle import mlp as M
    wts = M.glorot(11).astype(np.float32)
    samp = prad.PRAD_SAMPLER_MLP if sampler == "mlp" else prad.PRAD_SAMPLER_MLP_FALLBACK
    wl = _wave(n=8192 + 3, a0=500.0, seed=21)
    a = _run(wl, 16, 8, False, sampler=samp, weights=wts)
    b = _run(wl, 16, 8, True, sampler=samp, weights=wts)
    _same(a, b)
    assert a["stats"]["records"] > 1000
    assert b["stats"]["spec_launches"] == 2
    assert a["stats"]["mlp_fallback"] == b["stats"]["mlp_fallback"]


def _small_yee(n, seed=4, a0=300.0, nx=96, ny=80):
    rng = np.random.default_rng(seed)
    dxn = 2 * np.pi / 32
    wl = W.yee2d(n_grid=64, slab=32, n_particles=n, seed=seed, with_grid=False)
    wl.yee = W.yee_planes(nx, ny, a0, dxn, rng)
    wl.state["x"] = rng.uniform(0, nx, n) * dxn
    wl.state["y"] = rng.uniform(0, ny, n) * dxn
    return wl


def _run_by_id(wl, nsteps, specialize, **kw):
    """A run whose state is returned in id order (the tile sort reorders the
    particles, and the order within a tile may differ between runs)."""
    ctx = prad.Context(wl.problem_kwargs(), precision=prad.PRAD_FP32, photon_capacity=1 << 20,
                       max_particles=wl.n, specialize=specialize, **kw)
    st = ctx.to_device(wl.state, with_pid=True)
    ctx.push_emit(st, nsteps, t0=2)
    torch.cuda.synchronize()
    o = np.argsort(st["pid"].cpu().numpy().view(np.uint32))
    ph = ctx.photons(on_device=False)
    e, l, stats = ctx.energy_budget()
    le, ll = ctx.ledger()
    out = dict(state={k: v.cpu().numpy()[o] for k, v in st.items() if k != "pid"},
               ph={k: (v.numpy().copy() if hasattr(v, "numpy") else v) for k, v in ph.items()},
               e=e, l=l, stats=stats, le=le.cpu().numpy(), ll=ll.cpu().numpy())
    ctx.close()
    return out


@pytest.mark.parametrize("form", ["fused", "one_step", "tiled"])
def test_specialised_yee(form):
    """The Yee grid's kernels with the grid's size, spacing, origin and
    periods compiled in: the plain gather (fused and one-step launches) and
    the tile-staged kernel behind the tile sort."""
    wl = _small_yee(n=20000 + 11, nx=160, ny=96)
    kw = dict(sort_interval=5) if form == "tiled" else \
        dict(steps_per_launch=5 if form == "fused" else 1)
    a = _run_by_id(wl, 20, False, **kw)
    b = _run_by_id(wl, 20, True, **kw)
    _same(a, b)
    assert a["stats"]["records"] > 1000
    assert b["stats"]["spec_launches"] == (20 if form == "one_step" else 4)


def test_outside_the_standard_configuration_keeps_compiled_in_kernels():
    wl = _wave(n=2048)
    wl.rr_mode = W.RR_LEDGER  # LL kick booked, not applied: not the standard form
    a = _run(wl, 6, 3, True)
    assert a["stats"]["spec_launches"] == 0
    _same(_run(wl, 6, 3, False), a)
    b = _run(_wave(n=2048), 4, 1, True, precision=prad.PRAD_FP64)
    assert b["stats"]["spec_launches"] == 0


def test_control_variant_keeps_compiled_in_kernels():
    wl = _wave(n=2048)
    a = _run(wl, 6, 3, True, n_try=2)
    assert a["stats"]["spec_launches"] == 0
    _same(_run(wl, 6, 3, False, n_try=2), a)


def test_missing_nvrtc_fails_loudly_and_the_context_stays_usable():
    """Without NVRTC a specialised launch is an error with the reason, not a
    silent fallback; the context keeps working with specialize off (a child
    process, since NVRTC is opened once per process)."""
    code = """
import sys, torch
from paper_1409_5574_gb300 import prad, workloads as W
prad.load_library()
wl = W.plane_wave(a0=200.0, n=1000, seed=2)
ctx = prad.Context(wl.problem_kwargs(), precision=prad.PRAD_FP32, photon_capacity=1 << 16,
                   max_particles=wl.n, steps_per_launch=4, specialize=True)
st = ctx.to_device(wl.state)
try:
    ctx.push_emit(st, 4)
    print("NO ERROR")
except prad.PradError as e:
    print("ERROR", e)
ctx.close()
ctx = prad.Context(wl.problem_kwargs(), precision=prad.PRAD_FP32, photon_capacity=1 << 16,
                   max_particles=wl.n, steps_per_launch=4)
ctx.push_emit(ctx.to_device(wl.state), 4)
torch.cuda.synchronize()
print("RECORDS", ctx.energy_budget()[2]["records"])
ctx.close()
"""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, PRAD_NVRTC_LIBRARY="/nonexistent/libnvrtc.so.13")
    r = subprocess.run([sys.executable, "-c", code], cwd=root, env=env, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert "ERROR" in r.stdout and "NO ERROR" not in r.stdout, r.stdout
    assert "specialisation" in r.stdout and "NVRTC" in r.stdout, r.stdout
    n = int(r.stdout.split("RECORDS")[1].split()[0])
    assert n > 0


@pytest.mark.parametrize("n", [1, 31, 33])
def test_specialised_ragged_and_tiny_launches(n):
    """Launches of fewer particles than a warp or a block (the dense one-step
    form with one particle included) and an empty launch."""
    wl = _wave(n=n, a0=500.0, seed=5 + n)
    for spl in (1, 7):
        a = _run(wl, 14, spl, False)
        b = _run(wl, 14, spl, True)
        _same(a, b)
        assert b["stats"]["spec_launches"] == (14 if spl == 1 else 2)
    ctx = prad.Context(wl.problem_kwargs(), precision=prad.PRAD_FP32, photon_capacity=1 << 10,
                       max_particles=wl.n, specialize=True)
    st = {k: v[:0] for k, v in ctx.to_device(wl.state).items()}
    ctx.push_emit(st, 3)
    assert ctx.energy_budget()[2]["spec_launches"] == 0
    ctx.close()
