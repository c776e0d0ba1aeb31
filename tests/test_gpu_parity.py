"""GPU (sm_103a, through the C ABI) vs the FP64 CPU oracle, element by element.

Same seeded inputs on both sides, sizes that span several 256-thread tiles and
a ragged tail.  Tolerances (spec bar):
  * momentum per particle: |du| / |u| <= 1e-12 (FP64 path), <= 1e-5 (FP32);
  * photon multiset matched on (pid, step) >= 99.99%; every unmatched trial
    must sit within rounding of its decision threshold R = frac(dN);
  * matched photon energies <= 1e-5 relative (float32 records);
  * LL ledger totals <= 1e-10 (FP64) / 1e-4 (FP32); emitted totals <= 1e-4.
"""
import math

import numpy as np
import pytest

import fp32_envelope as FE
import oracle as O
from paper_1409_5574_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_1409_5574_gb300 import prad


def _run_gpu(wl, nsteps, precision, capacity=1 << 18, steps_per_launch=1, t0=0,
             block_size=0, blocks_per_sm=0):
    ctx = prad.Context(wl.problem_kwargs(), precision=precision,
                       photon_capacity=capacity, max_particles=wl.n,
                       steps_per_launch=steps_per_launch, block_size=block_size,
                       blocks_per_sm=blocks_per_sm)
    st = ctx.to_device(wl.state)
    ctx.push_emit(st, nsteps, t0=t0)
    torch.cuda.synchronize()
    ph = ctx.photons(on_device=False)
    emitted, ll, stats = ctx.energy_budget()
    led_e, led_l = ctx.ledger()
    out = dict(state={k: v.double().cpu().numpy() for k, v in st.items()},
               photons={k: (v.numpy() if hasattr(v, "numpy") else v) for k, v in ph.items()},
               emitted=emitted, ll=ll, stats=stats,
               led_emit=led_e.cpu().numpy(), led_ll=led_l.cpu().numpy())
    ctx.close()
    return out


def _run_oracle(wl, nsteps, capacity=1 << 18, t0=0):
    st = wl.copy_state()
    res = O.run(O.Problem(**wl.problem_kwargs()), st, nsteps, t0=t0,
                capacity=capacity, trial_log=True)
    res["state"] = st
    return res


def _momentum_rel(gs, os_):
    ug = np.stack([gs["ux"], gs["uy"], gs["uz"]], 1)
    uo = np.stack([os_["ux"], os_["uy"], os_["uz"]], 1)
    return np.abs(ug - uo).max(1) / np.maximum(np.linalg.norm(uo, axis=1), 1e-300)


def _check_photons(gpu, ref, t0, eps_rtol, flip_tol):
    gp, rp = gpu["photons"], ref["photons"]
    kg = gp["pid"].astype(np.int64) * 2**32 + gp["step"].astype(np.int64)
    kr = rp["pid"].astype(np.int64) * 2**32 + rp["step"].astype(np.int64)
    assert np.unique(kg).size == kg.size, "duplicate GPU records"
    common, ig, ir = np.intersect1d(kg, kr, return_indices=True)
    total = max(kg.size, kr.size)
    assert common.size >= 0.9999 * total - 1, (common.size, kg.size, kr.size)
    # matched: same multiplicity (weight) and energy
    wg, wr = gp["weight"][ig].astype(np.float64), rp["weight"][ir]
    same_w = np.isclose(wg, wr, rtol=1e-6)
    assert same_w.mean() >= 0.9999
    e_rel = np.abs(gp["eps"][ig] / rp["eps"][ir] - 1)
    assert np.all(e_rel[same_w] < eps_rtol), e_rel.max()
    # every unmatched trial is a near-threshold decision of the oracle
    tr = ref["trials"]
    for key in np.setxor1d(kg, kr):
        pid, step = int(key >> 32), int(key & 0xFFFFFFFF)
        s = step - t0
        dN, R = tr["dN"][pid, s], tr["R"][pid, s]
        frac = dN - math.floor(dN)
        assert abs(R - frac) <= flip_tol * max(1.0, dN), (pid, step, dN, R)
    return common.size, total


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    prad.load_library()


# ---------------------------------------------------------------- primitives
def test_philox_gpu_equals_oracle():
    rng = np.random.default_rng(11)
    ctr = rng.integers(0, 2**32, size=(4099, 4), dtype=np.uint64).astype(np.uint32)
    ctx = prad.Context(W.const_b(n=4).problem_kwargs(), max_particles=4, photon_capacity=4)
    d_ctr = torch.from_numpy(ctr.view(np.int32)).cuda()
    d_out = torch.empty_like(d_ctr)
    prad.prad_philox(ctx.h, d_ctr.data_ptr(), 0xDEADBEEF, 0x12345678, d_out.data_ptr(), 4099)
    got = d_out.cpu().numpy().view(np.uint32)
    ref = O.philox(ctr, [0xDEADBEEF, 0x12345678])
    np.testing.assert_array_equal(got, ref)
    ctx.close()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_sampler_gpu_vs_oracle(precision):
    """x = P^-1(R') and g = F/S of the device table against the oracle's
    x and F(x)/S(x), on Philox words plus the extreme and branch words."""
    p = prad.PRAD_FP32 if precision == "fp32" else prad.PRAD_FP64
    ctx = prad.Context(W.const_b(n=4).problem_kwargs(), precision=p,
                       max_particles=4, photon_capacity=4)
    ctr = np.zeros((20000, 4), dtype=np.uint32)
    ctr[:, 0] = np.arange(20000)
    words = O.philox(ctr, [5, 0])
    T = O.branch_threshold()
    extra = []
    for W64 in (0, 1, T - 1, T, T + 1, 2**64 - 1, 2**63, 2**32 - 1, 2**32):
        extra.append([W64 & 0xFFFFFFFF, W64 >> 32, 7, 0])
    words = np.concatenate([words, np.array(extra, dtype=np.uint32)])
    n = words.shape[0]
    dt = torch.float32 if p == prad.PRAD_FP32 else torch.float64
    d_w = torch.from_numpy(words.view(np.int32)).cuda()
    xg = torch.empty(n, dtype=dt, device="cuda")
    gg = torch.empty(n, dtype=dt, device="cuda")
    prad.prad_eval_sampler(ctx.h, d_w.data_ptr(), xg.data_ptr(), gg.data_ptr(), n)
    xg, gg = xg.double().cpu().numpy(), gg.double().cpu().numpy()
    xr = np.array([O.sample_x(w)[0] for w in words])
    gr = O.F(xr) / np.array([O.S_of_words(w) for w in words])
    xtol, gtol = (2e-6, 2e-6) if p == prad.PRAD_FP32 else (1e-13, 2e-8)
    assert np.max(np.abs(xg / xr - 1)) < xtol
    assert np.max(np.abs(gg / gr - 1)) < gtol
    ctx.close()


# ---------------------------------------------------------------- full step
def test_constB_fp64_parity():
    wl = W.const_b(n=2048 + 37, nsteps=200)
    gpu = _run_gpu(wl, 200, prad.PRAD_FP64)
    ref = _run_oracle(wl, 200)
    rel = _momentum_rel(gpu["state"], ref["state"])
    assert rel.max() <= 1e-12, rel.max()
    for k in ("x", "y", "z"):
        assert np.allclose(gpu["state"][k], ref["state"][k], rtol=1e-12, atol=1e-9)
    m, tot = _check_photons(gpu, ref, 0, eps_rtol=1e-6, flip_tol=1e-8)
    assert tot > 1000
    assert gpu["ll"] == pytest.approx(ref["ledger"]["ll"].sum(), rel=1e-10)
    assert np.allclose(gpu["led_ll"], ref["ledger"]["ll"], rtol=1e-10, atol=0)
    assert gpu["emitted"] == pytest.approx(ref["ledger"]["emit"].sum(), rel=1e-4)
    for k in ("dn_gt1", "clamped", "chi_gt1"):
        assert abs(gpu["stats"][k] - ref["stats"][k]) <= max(1, ref["stats"][k] // 1000)


def _f32_inputs(wl):
    """The FP32 path's inputs exactly (state rounded to float32)."""
    w = wl.subset(np.arange(wl.n))
    w.state = {k: v.astype(np.float32).astype(np.float64) for k, v in w.state.items()}
    return w


@pytest.mark.parametrize("a0", [100.0, 300.0, 500.0])
def test_planewave_fp32_parity(a0):
    nsteps = 40
    wl = _f32_inputs(W.plane_wave(a0=a0, n=4096 + 77, seed=7))
    gpu = _run_gpu(wl, nsteps, prad.PRAD_FP32)
    ref = _run_oracle(wl, nsteps)
    rel = _momentum_rel(gpu["state"], ref["state"])
    assert rel.max() <= 1e-5, rel.max()
    m, tot = _check_photons(gpu, ref, 0, eps_rtol=1e-5, flip_tol=2e-5)
    assert tot > 1000
    assert gpu["ll"] == pytest.approx(ref["ledger"]["ll"].sum(), rel=1e-4)
    assert gpu["emitted"] == pytest.approx(ref["ledger"]["emit"].sum(), rel=1e-4)
    assert gpu["stats"]["chi_gt1"] == pytest.approx(ref["stats"]["chi_gt1"], rel=1e-3, abs=2)


@pytest.mark.parametrize("hand", [1, -1])
@pytest.mark.parametrize("direction", [1, -1])
def test_planewave_signs_fp32_parity(hand, direction):
    """The standard kernels take the plane wave's handedness and direction
    as compile-time signs (four variants).  Each against the oracle (40
    one-step launches at a0 = 300, the electrons counter-propagating), and
    against the batched kernel, which reads the signs at run time: the
    same state and photons bit for bit."""
    wl = W.plane_wave(a0=300.0, n=4096 + 77, seed=9)
    wl.hand, wl.direction = hand, direction
    wl.state["ux"] = wl.state["ux"] * direction  # against the wave's direction
    wl = _f32_inputs(wl)
    nsteps = 40
    gpu = _run_gpu(wl, nsteps, prad.PRAD_FP32)
    ref = _run_oracle(wl, nsteps)
    rel = _momentum_rel(gpu["state"], ref["state"])
    assert rel.max() <= 1e-5, rel.max()
    m, tot = _check_photons(gpu, ref, 0, eps_rtol=1e-5, flip_tol=2e-5)
    assert tot > 1000
    assert gpu["ll"] == pytest.approx(ref["ledger"]["ll"].sum(), rel=1e-4)
    assert gpu["emitted"] == pytest.approx(ref["ledger"]["emit"].sum(), rel=1e-4)
    # the batched kernel (one ensemble, the same launch shape)
    ctx = prad.Context(wl.problem_kwargs(), precision=prad.PRAD_FP32,
                       photon_capacity=1 << 18, max_particles=wl.n, steps_per_launch=1)
    st = ctx.to_device(wl.state)
    ctx.push_emit_batch(ctx.ensembles([st], [wl.problem_kwargs()]), nsteps)
    torch.cuda.synchronize()
    ph = ctx.photons(on_device=False)
    for k in ("x", "y", "z", "ux", "uy", "uz"):
        np.testing.assert_array_equal(st[k].double().cpu().numpy(), gpu["state"][k], err_msg=k)
    kb = ph["pid"].numpy().astype(np.int64) * 2**32 + ph["step"].numpy().astype(np.int64)
    kg = gpu["photons"]["pid"].astype(np.int64) * 2**32 + gpu["photons"]["step"].astype(np.int64)
    ob, og = np.argsort(kb), np.argsort(kg)
    np.testing.assert_array_equal(kb[ob], kg[og])
    np.testing.assert_array_equal(ph["eps"].numpy()[ob], gpu["photons"]["eps"][og])
    ctx.close()


def _strong_constant_b(n=4096, a0=500.0, seed=2):
    """Isotropic electrons, gamma ~ U[100, 1000], in B = a0 m omega_L / e with
    the LL kick (the strongest constant-B ensembles of the batched mix)."""
    omega = 2 * math.pi * W.C_LIGHT / 0.8e-6
    rng = np.random.default_rng(seed)
    gamma = rng.uniform(100.0, 1000.0, n)
    u = rng.standard_normal((n, 3))
    u *= (np.sqrt(gamma ** 2 - 1) / np.linalg.norm(u, axis=1))[:, None]
    return W.Workload(name="strong constant B", omega_ref=omega,
                      dt=(2 * math.pi / omega) / 200, nsteps=1, rr_mode=W.RR_APPLY,
                      field_kind=W.FIELD_CONST, B=(0.0, 0.0, a0 * W.M_E * omega / W.Q_E),
                      state=dict(x=np.zeros(n), y=np.zeros(n), z=np.zeros(n), ux=u[:, 0].copy(),
                                 uy=u[:, 1].copy(), uz=u[:, 2].copy(), w=np.ones(n)))


def _small_yee_case(nx=130, ny=100, n=6000 + 13, seed=3):
    rng = np.random.default_rng(seed)
    dxn = 2 * np.pi / 32
    planes = W.yee_planes(nx, ny, 300.0, dxn, rng)
    wl = W.yee2d(n_grid=64, slab=32, n_particles=n, seed=seed, with_grid=False)
    wl.yee = planes
    wl.state["x"] = rng.uniform(-0.5, nx + 0.5, n) * dxn
    wl.state["y"] = rng.uniform(-0.5, ny + 0.5, n) * dxn
    return wl


@pytest.mark.parametrize("case", ["yee", "constant_b", "pw100", "pw300", "pw500"])
def test_one_step_departure_in_float32_units(case):
    """One FP32 step from identical float32 inputs departs from the oracle by
    at most FE.FACTOR (= 3) float32 units of |u| on every field kind: the
    kernel's own rounding per step, the factor the multi-step float32
    envelope bar allows over the envelope's one unit per step."""
    if case == "yee":
        wl = _small_yee_case()
    elif case == "constant_b":
        wl = _strong_constant_b()
    else:
        wl = W.plane_wave(a0=float(case[2:]), n=4096, seed=3)
    wl = _f32_inputs(wl)
    for t0 in (0, 1000):
        gpu = _run_gpu(wl, 1, prad.PRAD_FP32, t0=t0)
        ref = wl.copy_state()
        O.run(O.Problem(**wl.problem_kwargs()), ref, 1, t0=t0, capacity=1 << 16)
        units = FE.float32_units(gpu["state"], ref)
        assert units.max() <= FE.FACTOR, (case, t0, units.max())
        assert np.median(units) <= 1.0


def test_substeps_and_split_calls_are_bit_identical():
    """Fusing steps in one launch or splitting a run into calls gives the same
    bits (counter-based RNG, phase from a fixed-point step counter)."""
    wl = W.plane_wave(a0=300.0, n=3000, seed=2)
    a = _run_gpu(wl, 30, prad.PRAD_FP32, steps_per_launch=1)
    b = _run_gpu(wl, 30, prad.PRAD_FP32, steps_per_launch=7)
    c = _run_gpu(wl, 30, prad.PRAD_FP32, steps_per_launch=30, block_size=128,
                 blocks_per_sm=2)
    for k in a["state"]:
        np.testing.assert_array_equal(a["state"][k], b["state"][k])
        np.testing.assert_array_equal(a["state"][k], c["state"][k])
    # ledgers: float-float sums per launch, flushed to FP64 per launch, so
    # only the rounding of the flush depends on the substeps per launch
    np.testing.assert_allclose(a["led_ll"], b["led_ll"], rtol=1e-13)
    np.testing.assert_allclose(a["led_emit"], c["led_emit"], rtol=1e-13)
    assert a["emitted"] == pytest.approx(b["emitted"], rel=1e-13)
    assert a["emitted"] == pytest.approx(c["emitted"], rel=1e-13)
    for k in ("records", "dn_gt1", "clamped", "chi_gt1"):
        assert a["stats"][k] == b["stats"][k] == c["stats"][k]
    # split into two calls with t0
    ctx = prad.Context(wl.problem_kwargs(), precision=prad.PRAD_FP32,
                       photon_capacity=1 << 18, max_particles=wl.n)
    st = ctx.to_device(wl.state)
    ctx.push_emit(st, 12, t0=0)
    ctx.push_emit(st, 18, t0=12)
    e, l, _ = ctx.energy_budget()
    for k in a["state"]:
        np.testing.assert_array_equal(a["state"][k], st[k].double().cpu().numpy())
    assert e == pytest.approx(a["emitted"], rel=1e-13)
    assert l == pytest.approx(a["ll"], rel=1e-13)
    ctx.close()


def test_momentum_form_heff_parity():
    wl = W.plane_wave(a0=100.0, n=1500, seed=5)
    wl.heff_form = W.HEFF_MOMENTUM
    gpu = _run_gpu(wl, 20, prad.PRAD_FP64)
    ref = _run_oracle(wl, 20)
    assert _momentum_rel(gpu["state"], ref["state"]).max() <= 1e-12
    _check_photons(gpu, ref, 0, eps_rtol=1e-6, flip_tol=1e-9)
    assert gpu["ll"] == pytest.approx(ref["ledger"]["ll"].sum(), rel=1e-10)


# ---------------------------------------------------------------- edge cases
def test_edge_cases_empty_overflow_nan_zero_weight():
    wl = W.plane_wave(a0=500.0, n=700, seed=9)
    ctx = prad.Context(wl.problem_kwargs(), precision=prad.PRAD_FP32,
                       photon_capacity=64, max_particles=wl.n)
    st = ctx.to_device(wl.state)
    ctx.push_emit(st, 0)                     # no-op
    ctx.push_emit({k: v[:0] for k, v in st.items()}, 5)   # n = 0: no-op
    st["w"][:100] = 0.0                      # zero weight: no records
    st["ux"][100] = float("nan")             # frozen and counted
    ctx.push_emit(st, 10)
    torch.cuda.synchronize()
    ph = ctx.photons(on_device=False)
    held = ph["pid"].numel()
    assert held == 64 and ph["dropped"] > 0     # overflow counted, never written
    assert np.all(ph["pid"].numpy() >= 100)
    assert not np.any(ph["pid"].numpy() == 100)
    _, _, stats = ctx.energy_budget()
    # counted once per launch (10 launches of one step)
    assert stats["nan_frozen"] == 10 and stats["rc"] == prad.PRAD_WARN_NAN
    assert stats["records"] == 64 and stats["dropped"] == ph["dropped"]
    assert math.isnan(st["ux"][100].item())
    n, d = ctx.drain()
    assert (n, d) == (64, ph["dropped"])
    assert ctx.drain() == (0, 0)
    _, _, s2 = ctx.energy_budget()
    assert s2["records"] == 64 and s2["dropped"] == ph["dropped"]
    # argument errors come back as codes
    bad = prad.prad_particles()
    with pytest.raises(prad.PradError) as ei:
        prad.prad_push_emit(ctx.h, bad, 10, 1)
    assert ei.value.code == prad.PRAD_ERR_ARG
    with pytest.raises(prad.PradError):
        ctx.push_emit(st, 1, ledger_offset=wl.n)        # ledger range
    ctx.close()


def test_single_particle_and_ledger_determinism():
    wl = W.const_b(n=1, nsteps=50)
    gpu = _run_gpu(wl, 50, prad.PRAD_FP64)
    ref = _run_oracle(wl, 50)
    assert _momentum_rel(gpu["state"], ref["state"]).max() <= 1e-12
    # two-pass Kahan reduction is deterministic and matches an exact sum
    wl = W.plane_wave(a0=300.0, n=50_000, seed=4)
    ctx = prad.Context(wl.problem_kwargs(), precision=prad.PRAD_FP32,
                       photon_capacity=1 << 20, max_particles=wl.n)
    st = ctx.to_device(wl.state)
    ctx.push_emit(st, 20)
    e1, l1, _ = ctx.energy_budget()
    e2, l2, _ = ctx.energy_budget()
    assert (e1, l1) == (e2, l2)
    le, ll = ctx.ledger()
    assert math.fsum(ll.cpu().numpy()) == pytest.approx(l1, rel=1e-15)
    assert math.fsum(le.cpu().numpy()) == pytest.approx(e1, rel=1e-15)
    ctx.close()
