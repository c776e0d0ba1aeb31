"""One-step launches (the form a PIC code calls every time step: the next
particle's state and ledger entries prefetched, ledgers updated by
read-modify-write) against multi-step launches (state in registers for
all steps, ledgers updated by fire-and-forget atomics), through the C ABI.

Both forms run the same per-particle arithmetic, so the particle state, the
counters and the photon multiset must agree bit for bit, for every field
kind, with and without the LL ledger, at particle counts that do and do not
fill the last 256-thread block, with grids that walk several blocks of
particles per thread and with explicit id arrays.  The per-particle ledgers
differ only in the grouping of the FP64 adds (one per launch), so they
agree to FP64 rounding.  The FP32 parity tests against the oracle in
test_gpu_parity.py run through the one-step form (one step per launch).
"""
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


def _small_yee(n, seed=4, a0=300.0, nx=96, ny=80):
    rng = np.random.default_rng(seed)
    dxn = 2 * np.pi / 32
    wl = W.yee2d(n_grid=64, slab=32, n_particles=n, seed=seed, with_grid=False)
    wl.yee = W.yee_planes(nx, ny, a0, dxn, rng)
    wl.state["x"] = rng.uniform(0, nx, n) * dxn
    wl.state["y"] = rng.uniform(0, ny, n) * dxn
    return wl


def _run(wl, nsteps, steps_per_launch, blocks_per_sm=0, with_pid=False, cap=1 << 20, **kw):
    ctx = prad.Context(wl.problem_kwargs(), precision=prad.PRAD_FP32,
                       photon_capacity=cap, max_particles=wl.n,
                       steps_per_launch=steps_per_launch, blocks_per_sm=blocks_per_sm, **kw)
    st = ctx.to_device(wl.state, with_pid=with_pid)
    ctx.push_emit(st, nsteps, t0=3)
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
    """Records in a canonical order: by (pid, step), then by their values
    (with super-photon control a step can write several records)."""
    key = ph["pid"].astype(np.int64) * 2**32 + ph["step"].astype(np.int64)
    names = ("x", "y", "z", "nx", "ny", "nz", "eps", "weight")
    o = np.lexsort(tuple(ph[k] for k in reversed(names)) + (key,))
    cols = [ph[k][o] for k in names]
    return key[o], np.stack(cols, 1)


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
    assert a["stats"]["status"] == 0
    assert a["e"] == pytest.approx(b["e"], rel=1e-13)
    assert a["l"] == pytest.approx(b["l"], rel=1e-13)


CASES = {
    "planewave": lambda n: W.plane_wave(a0=500.0, n=n, seed=11),
    "planewave_rr_off": lambda n: W.plane_wave(a0=300.0, n=n, seed=12, rr_mode=W.RR_OFF),
    "const_b": lambda n: W.const_b(n=n, nsteps=20, seed=13),
    "yee2d": lambda n: _small_yee(n),
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("n", [256 * 37, 256 * 41 + 129])
def test_one_step_launches_equal_fused_launch(case, n):
    wl = CASES[case](n)
    a = _run(wl, 12, steps_per_launch=1)
    b = _run(wl, 12, steps_per_launch=12)
    assert a["stats"]["records"] > 0
    if case == "planewave_rr_off":
        assert not a["ll"].any()
    _same(a, b)


@pytest.mark.parametrize("with_pid", [False, True])
def test_one_step_with_super_photon_control_equals_fused(with_pid):
    """Super-photon control (3 trials per step at 1/3 of dN each, selection
    probability 1/2): a step can add several records' energies to a
    particle's emitted-energy ledger; one-step launches (implicit ids, and
    an id array) still give the state, photons and ledgers of one fused
    launch."""
    wl = W.plane_wave(a0=500.0, n=(1 << 16) + 77, seed=23)
    kw = dict(n_try=3, select_prob=0.5)
    a = _run(wl, 8, steps_per_launch=1, with_pid=with_pid, **kw)
    b = _run(wl, 8, steps_per_launch=8, **kw)
    assert a["stats"]["records"] > 0
    _same(a, b)


def test_one_step_many_particles_per_thread():
    """2^22 electrons on the default grid (four 256-thread blocks per SM):
    each thread of the one-step kernel walks ~27 particles through its
    prefetch pipeline; four one-step launches equal one fused launch."""
    wl = W.plane_wave(a0=500.0, n=1 << 22, seed=27)
    a = _run(wl, 4, steps_per_launch=1, cap=1 << 22)
    b = _run(wl, 4, steps_per_launch=4, cap=1 << 22)
    assert a["stats"]["records"] > 0 and a["stats"]["dropped"] == 0
    _same(a, b)


@pytest.mark.parametrize("bps", [1, 2])
def test_one_step_small_grids_and_id_arrays(bps):
    # 2^16 + 77 particles on 152 or 304 blocks: each thread walks one or two
    # particles, with the prefetch crossing the ragged end
    wl = W.plane_wave(a0=300.0, n=(1 << 16) + 77, seed=14)
    ref = _run(wl, 9, steps_per_launch=9)
    _same(_run(wl, 9, steps_per_launch=1, blocks_per_sm=bps), ref)
    _same(_run(wl, 9, steps_per_launch=1, blocks_per_sm=bps, with_pid=True), ref)


def test_one_step_tiny_counts():
    for n in (1, 31, 255, 257):
        wl = W.plane_wave(a0=500.0, n=n, seed=16)
        _same(_run(wl, 5, steps_per_launch=1), _run(wl, 5, steps_per_launch=5))


def _run_layout(wl, nsteps, with_pid=False, offset=0, ledger_offset=0):
    """One step per launch with the arrays optionally viewed `offset`
    elements into a larger buffer and the ledger entries at ledger_offset."""
    ctx = prad.Context(wl.problem_kwargs(), precision=prad.PRAD_FP32,
                       photon_capacity=1 << 20, max_particles=wl.n + ledger_offset,
                       steps_per_launch=1)
    st = ctx.to_device(wl.state, with_pid=with_pid)
    if offset:
        views = {}
        for k, v in st.items():
            buf = torch.zeros(v.numel() + offset, dtype=v.dtype, device=v.device)
            buf[offset:] = v
            views[k] = buf[offset:]
        st = views
    ctx.push_emit(st, nsteps, t0=3, ledger_offset=ledger_offset)
    torch.cuda.synchronize()
    ph = ctx.photons(on_device=False)
    e, l, stats = ctx.energy_budget()
    le, ll = ctx.ledger()
    sl = slice(ledger_offset, ledger_offset + wl.n)
    out = dict(state={k: v.cpu().numpy().copy() for k, v in st.items() if k != "pid"},
               ph={k: (v.numpy().copy() if hasattr(v, "numpy") else v) for k, v in ph.items()},
               e=e, l=l, stats=stats, le=le.cpu().numpy()[sl], ll=ll.cpu().numpy()[sl])
    ctx.close()
    return out


@pytest.mark.parametrize("n", [255, 256 * 41 + 129, (1 << 16) + 77])
def test_one_step_results_do_not_depend_on_layout(n):
    """One step per launch with implicit ids, with an explicit id array, with
    every array one element off a 16-byte boundary (views into larger
    buffers) and with an odd ledger offset: state, ledgers, counters and
    photons agree bit for bit."""
    wl = W.plane_wave(a0=500.0, n=n, seed=31)
    ref = _run_layout(wl, 6)
    assert ref["stats"]["records"] > 0 and ref["stats"]["status"] == 0
    for kw in (dict(with_pid=True), dict(offset=1), dict(ledger_offset=1)):
        other = _run_layout(wl, 6, **kw)
        for k in ref["state"]:
            np.testing.assert_array_equal(ref["state"][k], other["state"][k], err_msg=f"{kw} {k}")
        np.testing.assert_array_equal(ref["le"], other["le"])
        np.testing.assert_array_equal(ref["ll"], other["ll"])
        ka, ta = _photon_table(ref["ph"])
        kb, tb = _photon_table(other["ph"])
        np.testing.assert_array_equal(ka, kb)
        np.testing.assert_array_equal(ta, tb)
        for k in ("records", "dropped", "dn_gt1", "clamped", "chi_gt1", "nan_frozen", "status"):
            assert ref["stats"][k] == other["stats"][k], (kw, k)


@pytest.fixture(scope="module")
def mlp_params():
    """A trained learned sampler (10^7 device samples: enough for valid
    outputs; the equality below does not depend on its accuracy)."""
    wl = W.plane_wave(a0=300.0, n=16, seed=1)
    ctx = prad.Context(wl.problem_kwargs(), precision=prad.PRAD_FP32,
                       photon_capacity=1 << 10, max_particles=16)
    ctx.mlp_train(160, 65536, 3e-3, seed=3)
    p = ctx.mlp_weights()
    ctx.close()
    return p


@pytest.mark.parametrize("n", [256 * 37, 256 * 41 + 129])
def test_one_step_launches_equal_fused_launch_learned_sampler(mlp_params, n):
    """The learned sampler's step kernel (records staged as vectors with the
    network payload) in one-step and multi-step launches: the same state,
    counters and photon multiset (energies from the finishing kernel after
    each call), ledgers to FP64 rounding."""
    wl = W.plane_wave(a0=500.0, n=n, seed=21)
    out = []
    for spl in (1, 12):
        ctx = prad.Context(wl.problem_kwargs(), precision=prad.PRAD_FP32,
                           sampler=prad.PRAD_SAMPLER_MLP_FALLBACK, photon_capacity=1 << 20,
                           max_particles=wl.n, steps_per_launch=spl)
        ctx.mlp_set_weights(mlp_params)
        st = ctx.to_device(wl.state)
        ctx.push_emit(st, 12, t0=3)
        torch.cuda.synchronize()
        ph = ctx.photons(on_device=False)
        e, l, stats = ctx.energy_budget()
        le, ll = ctx.ledger()
        out.append(dict(state={k: v.cpu().numpy().copy() for k, v in st.items() if k != "pid"},
                        ph={k: (v.numpy().copy() if hasattr(v, "numpy") else v)
                            for k, v in ph.items()},
                        e=e, l=l, stats=stats, le=le.cpu().numpy(), ll=ll.cpu().numpy()))
        ctx.close()
    a, b = out
    assert a["stats"]["records"] > 0
    for k in ("records", "dropped", "dn_gt1", "clamped", "chi_gt1", "nan_frozen", "status"):
        assert a["stats"][k] == b["stats"][k], k
    _same(a, b)
