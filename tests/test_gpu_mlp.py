"""Learned inverse-CDF sampler on the GPU, through the C ABI.

* the device G^-1 table against the oracle's inverse number CDF;
* the tensor-core tile evaluator against the FP64 numpy net (same weights),
  and its bounded waits: a withheld MMA completion is reported, not hung on;
* the training kernels' gradient against the FP64 numpy backward;
* training on 2 x 10^8 device-generated samples reaches a spectral error
  sup_r |G(g(r)) - r| <= 0.5% (G from the oracle) from ~100% untrained, for
  gamma and omega_c dt inside and outside the trained range;
* the direct-scheme emission with the trained net reproduces the number
  spectrum (KS vs the oracle's G) and the synchrotron power in a constant B.
"""
import math

import numpy as np
import pytest

import oracle as O
from oracle import mlp as M
from paper_1409_5574_gb300 import workloads as W

torch = pytest.importorskip("torch")
stats = pytest.importorskip("scipy.stats")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_1409_5574_gb300 import prad


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    prad.load_library()


def _ctx(sampler=None, wl=None, **kw):
    wl = wl or W.plane_wave(a0=500.0, n=16)
    s = prad.PRAD_SAMPLER_TABLE if sampler is None else sampler
    return prad.Context(wl.problem_kwargs(), precision=prad.PRAD_FP32, sampler=s,
                        max_particles=max(16, wl.n), photon_capacity=kw.pop("cap", 1 << 20), **kw)


def _spectral_error(ctx, gamma, wdt, n=1_000_000):
    r = (np.arange(n) + 0.5) / n
    lnx = ctx.mlp_eval(r, np.full(n, gamma), np.full(n, wdt)).cpu().numpy().astype(np.float64)
    return np.max(np.abs(O.G(np.exp(lnx)) - r))


def test_ginv_table_vs_oracle():
    ctx = _ctx()
    lg = np.linspace(-20, 20, 4001)
    r = 1 / (1 + np.exp(-lg))
    r = r[(r > 1e-9) & (r < 1 - 1e-7)]
    got = ctx.ginv(r).cpu().numpy().astype(np.float64)
    ref = np.log(O.Ginv(r.astype(np.float32).astype(np.float64)))
    assert np.max(np.abs(got - ref)) < 2e-3
    ctx.close()


def test_tile_evaluator_matches_fp64_net():
    p = M.glorot(11)
    ctx = _ctx()
    ctx.mlp_set_weights(p.astype(np.float32))
    rng = np.random.default_rng(4)
    n = 5000 + 3
    r = rng.uniform(1e-6, 1 - 1e-6, n).astype(np.float32)
    g = np.exp(rng.uniform(np.log(5), np.log(5e4), n)).astype(np.float32)
    w = np.exp(rng.uniform(-6, 22, n)).astype(np.float32)
    got = ctx.mlp_eval(r, g, w).cpu().numpy().astype(np.float64)
    ref = M.ln_x(p.astype(np.float32).astype(np.float64), r.astype(np.float64),
                 g.astype(np.float64), w.astype(np.float64))
    d = np.abs(got - ref)
    assert np.median(d) < 5e-3 and d.max() < 5e-2, (np.median(d), d.max())
    ctx.close()


def test_tensor_core_wait_timeout_is_reported_and_context_recovers():
    """The evaluator with every MMA completion withheld: each bounded wait
    runs out (~2 s), the kernel frees its tensor memory and reports the
    timeout; the same context then evaluates as before."""
    p = M.glorot(12).astype(np.float32)
    ctx = _ctx()
    ctx.mlp_set_weights(p)
    r = np.linspace(0.01, 0.99, 300).astype(np.float32)
    g = np.full(300, 100.0, np.float32)
    w = np.full(300, 10.0, np.float32)
    before = ctx.mlp_eval(r, g, w).cpu().numpy()
    assert prad.prad_mlp_wait_selftest(ctx.h) == prad.PRAD_ERR_TIMEOUT
    after = ctx.mlp_eval(r, g, w).cpu().numpy()
    np.testing.assert_array_equal(before, after)
    assert ctx.energy_budget()[2]["status"] == 0
    ctx.close()


def test_training_gradient_matches_fp64_backward():
    p = M.glorot(5).astype(np.float32)
    ctx = _ctx()
    ctx.mlp_set_weights(p)
    rng = np.random.default_rng(8)
    n = 1000 + 29
    r = rng.uniform(1e-6, 1 - 1e-6, n).astype(np.float32)
    g = np.exp(rng.uniform(np.log(10), np.log(1e4), n)).astype(np.float32)
    w = np.exp(rng.uniform(-3, 19, n)).astype(np.float32)
    t = np.log(O.Ginv(r.astype(np.float64))).astype(np.float32)
    grad, loss = ctx.mlp_grad(r, g, w, t)
    lref, gref = M.loss_and_grad(p.astype(np.float64), r.astype(np.float64),
                                 g.astype(np.float64), w.astype(np.float64),
                                 t.astype(np.float64))
    assert loss == pytest.approx(lref, rel=2e-3)
    for a, b in ((M.OFF_W1, M.OFF_B1), (M.OFF_B1, M.OFF_W2), (M.OFF_W2, M.OFF_B2),
                 (M.OFF_B2, M.OFF_W3), (M.OFF_W3, M.OFF_B3), (M.OFF_B3, M.NUM_PARAMS)):
        err = np.linalg.norm(grad[a:b] - gref[a:b]) / np.linalg.norm(gref[a:b])
        assert err < 1e-2, (a, b, err)
    ctx.close()


@pytest.fixture(scope="module")
def trained():
    """Train once on 2 x 10^8 device-generated samples (3052 x 65536)."""
    ctx = _ctx()
    before = _spectral_error(ctx, 1000.0, 1e3, n=100_000)
    loss = ctx.mlp_train(3052, 65536, 3e-3, seed=7)
    params = ctx.mlp_weights()
    ctx.close()
    return params, before, loss


@pytest.mark.parametrize("gamma,wdt", [(1000.0, 1e3), (10.0, 0.1), (1e4, 1e8),
                                       (1e5, 1e12), (3.0, 1e-4)])
def test_trained_spectral_error_below_half_percent(trained, gamma, wdt):
    params, before, loss = trained
    ctx = _ctx()
    ctx.mlp_set_weights(params)
    err = _spectral_error(ctx, gamma, wdt)
    assert before > 0.05          # what training gains: from a useless sampler
    assert err <= 0.005, (gamma, wdt, err, loss)
    # mean photon energy E[x] = int_0^1 G^-1(r) dr = (8 pi/9 sqrt3)/(5 pi/3)
    n = 200_000
    r = (np.arange(n) + 0.5) / n
    x = np.exp(ctx.mlp_eval(r, np.full(n, gamma), np.full(n, wdt)).cpu().numpy())
    ex = (8 * math.pi / (9 * math.sqrt(3))) / (5 * math.pi / 3)
    assert abs(x.mean() / ex - 1) < 1e-2, x.mean() / ex
    ctx.close()


def test_direct_scheme_spectrum_and_power(trained):
    """Constant B (10^4 T, isotropic electrons, gamma in [100, 1000]; FP32,
    no LL kick): the direct
    scheme with the trained net emits the number spectrum G and, on average,
    the synchrotron power; the table scheme on the same GPU agrees."""
    params, _, _ = trained
    wl = W.const_b(n=4000, nsteps=500, seed=3)
    res = {}
    for name, smp in (("mlp", prad.PRAD_SAMPLER_MLP_FALLBACK), ("table", prad.PRAD_SAMPLER_TABLE)):
        ctx = _ctx(smp, wl=wl, cap=1 << 20)
        if smp != prad.PRAD_SAMPLER_TABLE:
            ctx.mlp_set_weights(params)
        st = ctx.to_device(wl.state)
        ctx.push_emit(st, 500)
        ph = ctx.photons(on_device=False)
        e, l, s = ctx.energy_budget()
        res[name] = (ph, e, l, s)
        ctx.close()
    # closed-form eps_c per particle (pure B, |u| conserved)
    s = wl.state
    u = np.stack([s["ux"], s["uy"], s["uz"]], 1)
    Bn = wl.B[2] * W.Q_E / (W.M_E * wl.omega_ref)
    dtn = wl.dt * wl.omega_ref
    gam = np.sqrt(1 + (u * u).sum(1))
    th = 2 * np.arctan(Bn * dtn / (2 * gam))
    uperp = np.hypot(u[:, 0], u[:, 1]) * np.cos(th / 2)
    ua2 = u[:, 2] ** 2 + uperp ** 2
    ga = np.sqrt(1 + ua2)
    Om = Bn * uperp / ga
    eps_r = 1.054571817e-34 * wl.omega_ref / (W.M_E * 299792458.0 ** 2)
    epsc = eps_r * 1.5 * Om * ga ** 2
    alpha = O.alpha()
    expect = (2 / 3 * alpha * eps_r * Om ** 2 * ga ** 2 * dtn).sum() * 500
    ph, e, l, st = res["mlp"]
    x = ph["eps"].numpy().astype(np.float64) / epsc[ph["pid"].numpy()]
    assert np.all(ph["weight"].numpy() == 1.0)
    p = stats.kstest(x, lambda v: O.G(np.atleast_1d(v))).pvalue
    assert x.size > 10000 and p > 0.01
    en = ph["eps"].numpy().astype(np.float64)
    sigma = math.sqrt((en * en).sum())
    assert abs(e - expect) < 4 * sigma
    assert st["mlp_fallback"] < 1e-3 * x.size
    # the table (S-proposal) scheme agrees within the combined sigma
    ph_t, e_t, _, _ = res["table"]
    et = ph_t["eps"].numpy().astype(np.float64) * ph_t["weight"].numpy()
    assert abs(e - e_t) < 4 * math.sqrt(sigma ** 2 + (et * et).sum())
    assert l == pytest.approx(res["table"][2], rel=1e-6)


def test_direct_scheme_full_buffer_keeps_energy(trained):
    """Constant B with a photon buffer of 1024 records (out of ~6300): the
    records beyond the capacity are counted as dropped and never written,
    take their energy from the G^-1 table at once (counted as fallbacks) and
    still enter the emitted-energy ledger, so the total matches the run with
    room for every record within the statistical sigma; the held records
    are finished by the tensor-core kernel like any other."""
    params, _, _ = trained
    wl = W.const_b(n=4000, nsteps=300, seed=5)
    res = {}
    for cap in (1024, 1 << 20):
        ctx = _ctx(prad.PRAD_SAMPLER_MLP_FALLBACK, wl=wl, cap=cap)
        ctx.mlp_set_weights(params)
        st = ctx.to_device(wl.state)
        for c in range(3):  # three calls: the finishing kernel resumes each time
            ctx.push_emit(st, 100, t0=100 * c)
        ph = ctx.photons(on_device=False)
        e, l, s = ctx.energy_budget()
        res[cap] = (ph, e, l, s)
        ctx.close()
    ph_s, e_s, l_s, s_s = res[1024]
    ph_b, e_b, l_b, s_b = res[1 << 20]
    assert s_b["dropped"] == 0 and s_b["records"] > 5000
    # same trials and decisions: every record of the big run is held or
    # dropped in the small one
    assert s_s["records"] == 1024
    assert s_s["records"] + s_s["dropped"] == s_b["records"]
    assert s_s["mlp_fallback"] >= s_s["dropped"]
    held = ph_s["eps"].numpy()
    assert held.size == 1024 and np.all(np.isfinite(held)) and np.all(held > 0)
    assert l_s == pytest.approx(l_b, rel=1e-12)
    # each record's uniform r is the same in both runs; the dropped ones take
    # x = G^-1(r) from the table instead of the network (both within the
    # spectral error of the exact inverse), so the totals agree closely
    assert e_s == pytest.approx(e_b, rel=1e-2), (e_s, e_b)
    assert s_s["status"] == 0 and s_b["status"] == 0
