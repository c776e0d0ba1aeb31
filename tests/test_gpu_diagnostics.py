"""Diagnostics through the C ABI: the angular distribution of the emitted
energy (Fig. 4) from the device histogram against the oracle's FP64
histogram of the same photon records."""
import math

import numpy as np
import pytest

import oracle as O
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


@pytest.mark.parametrize("axis,ref,nt,nph,tmax", [
    ((1.0, 0.0, 0.0), (0.0, 1.0, 0.0), 45, 72, math.pi / 2),   # front hemisphere
    ((-1.0, 0.0, 0.0), (0.0, 0.0, 1.0), 30, 36, math.pi),      # whole sphere, other axis
    ((0.2, 0.9, -0.3), (1.0, 0.0, 0.0), 64, 128, 1.0)])
def test_angular_histogram_matches_oracle(axis, ref, nt, nph, tmax):
    wl = W.plane_wave(a0=300.0, n=8192 + 5, seed=21)
    ctx = prad.Context(wl.problem_kwargs(), precision=prad.PRAD_FP32,
                       photon_capacity=1 << 20, max_particles=wl.n, steps_per_launch=50)
    st = ctx.to_device(wl.state)
    ctx.push_emit(st, 200)
    h = ctx.angular_histogram(axis, ref, nt, nph, tmax)
    ph = ctx.photons(on_device=False)
    rec = {k: ph[k].numpy() for k in ("nx", "ny", "nz", "eps", "weight")}
    ho = O.angular_histogram(rec["nx"], rec["ny"], rec["nz"], rec["eps"], rec["weight"], axis,
                             ref, nt, nph, tmax)
    assert ph["pid"].numel() > 10000
    e = rec["eps"].astype(np.float64) * rec["weight"]
    # bins agree except for records within rounding of a bin edge
    diff = np.abs(h - ho).sum()
    assert diff <= 1e-9 * ho.sum() + 4 * e.max(), (diff, ho.sum())
    assert h.sum() == pytest.approx(ho.sum(), rel=1e-9, abs=2 * e.max())
    ctx.close()


def test_angular_histogram_learned_sampler_and_errors():
    """Records of the learned sampler get their energy from the finishing
    kernel before the histogram reads them; argument errors are codes."""
    wl = W.plane_wave(a0=500.0, n=4096, seed=22)
    ctx = prad.Context(wl.problem_kwargs(), precision=prad.PRAD_FP32,
                       sampler=prad.PRAD_SAMPLER_MLP_FALLBACK, photon_capacity=1 << 20,
                       max_particles=wl.n, steps_per_launch=25)
    ctx.mlp_train(200, 65536, 3e-3, seed=7)
    st = ctx.to_device(wl.state)
    ctx.push_emit(st, 100)
    h = ctx.angular_histogram()
    ph = ctx.photons(on_device=False)
    ho = O.angular_histogram(ph["nx"].numpy(), ph["ny"].numpy(), ph["nz"].numpy(),
                             ph["eps"].numpy(), ph["weight"].numpy(), (1, 0, 0), (0, 1, 0),
                             45, 72, math.pi / 2)
    assert ho.sum() > 0 and h.sum() == pytest.approx(ho.sum(), rel=1e-6)
    for bad in [dict(ntheta=0), dict(nphi=200, ntheta=200), dict(theta_max=4.0),
                dict(axis=(0, 0, 0)), dict(axis=(1, 0, 0), ref=(2, 0, 0))]:
        with pytest.raises(prad.PradError) as ei:
            ctx.angular_histogram(**bad)
        assert ei.value.code == prad.PRAD_ERR_ARG
    ctx.close()


# ---------------------------------------------------- super-photon control
def _f32(wl):
    w = wl.subset(np.arange(wl.n))
    w.state = {k: v.astype(np.float32).astype(np.float64) for k, v in w.state.items()}
    return w


@pytest.mark.parametrize("n_try,q", [(3, 1.0), (1, 0.5), (4, 0.3)])
def test_super_photon_control_matches_oracle(n_try, q):
    """n_try trials and selection q on the GPU against the oracle's same
    Philox blocks (plane wave, FP32): the records of each (pid, step) agree
    except for decisions within rounding of their thresholds; totals agree."""
    from collections import Counter
    wl = _f32(W.plane_wave(a0=300.0, n=3000 + 17, seed=31))
    ctx = prad.Context(wl.problem_kwargs(), precision=prad.PRAD_FP32,
                       photon_capacity=1 << 20, max_particles=wl.n, n_try=n_try,
                       select_prob=q)
    st = ctx.to_device(wl.state)
    ctx.push_emit(st, 30)
    torch.cuda.synchronize()
    ph = ctx.photons(on_device=False)
    e_gpu, l_gpu, s_gpu = ctx.energy_budget()
    ctx.close()
    sto = wl.copy_state()
    ref = O.run(O.Problem(**{**wl.problem_kwargs(), "n_try": n_try, "select_prob": q}), sto,
                30, capacity=1 << 20)
    kg = Counter(zip(ph["pid"].numpy().tolist(), ph["step"].numpy().tolist()))
    ko = Counter(zip(ref["photons"]["pid"].tolist(), ref["photons"]["step"].tolist()))
    common = sum((kg & ko).values())
    total = max(sum(kg.values()), sum(ko.values()))
    assert total > 2000 and common >= 0.999 * total - 2, (common, total)
    assert e_gpu == pytest.approx(ref["ledger"]["emit"].sum(), rel=2e-3)
    assert l_gpu == pytest.approx(ref["ledger"]["ll"].sum(), rel=1e-4)
    if q < 1:
        wr = ph["weight"].numpy().astype(np.float64) / wl.state["w"][ph["pid"].numpy()]
        assert np.all(np.abs(wr * q - np.round(wr * q)) < 1e-4)


def test_selection_with_learned_sampler_and_n_try_rules():
    wl = W.plane_wave(a0=300.0, n=2048, seed=32)
    with pytest.raises(prad.PradError):
        prad.Context(wl.problem_kwargs(), sampler=prad.PRAD_SAMPLER_MLP_FALLBACK, n_try=2)
    with pytest.raises(prad.PradError):
        prad.Context(wl.problem_kwargs(), select_prob=1.5)
    res = {}
    for q in (1.0, 0.5):
        ctx = prad.Context(wl.problem_kwargs(), precision=prad.PRAD_FP32,
                           sampler=prad.PRAD_SAMPLER_MLP_FALLBACK, photon_capacity=1 << 20,
                           max_particles=wl.n, select_prob=q, steps_per_launch=20)
        ctx.mlp_train(300, 65536, 3e-3, seed=7)
        st = ctx.to_device(wl.state)
        ctx.push_emit(st, 60)
        ph = ctx.photons(on_device=False)
        e, _, s = ctx.energy_budget()
        res[q] = (e, ph["eps"].numpy().astype(np.float64) * ph["weight"].numpy(), s)
        ctx.close()
    (e1, r1, s1), (e2, r2, s2) = res[1.0], res[0.5]
    sigma = math.sqrt((r1 * r1).sum() + (r2 * r2).sum())
    assert abs(e1 - e2) < 4 * sigma
    assert abs(s2["records"] - 0.5 * s1["records"]) < 5 * math.sqrt(s1["records"])


# --------------------------------------------------------- wiggler regime
@pytest.mark.parametrize("a0", [0.5, 0.97, 1.03, 2.0])
def test_wiggler_counter_matches_oracle(a0):
    wl = W.plane_wave(a0=a0, n=5000, seed=33)
    rng = np.random.default_rng(4)
    for k in ("ux", "uy", "uz"):
        wl.state[k] = rng.normal(0.0, 0.05, wl.n)
    wl = _f32(wl)
    ctx = prad.Context(wl.problem_kwargs(), precision=prad.PRAD_FP32,
                       photon_capacity=1 << 20, max_particles=wl.n,
                       diagnostics=prad.PRAD_DIAG_WIGGLER)
    st = ctx.to_device(wl.state)
    ctx.push_emit(st, 20)
    _, _, s = ctx.energy_budget()
    ctx.close()
    ref = O.run(O.Problem(**wl.problem_kwargs()), wl.copy_state(), 20, capacity=1 << 20)
    got, want = s["wiggler_invalid"], ref["stats"]["wiggler_invalid"]
    assert abs(got - want) <= max(3, 1e-3 * want), (got, want)
    # off by default
    ctx = prad.Context(wl.problem_kwargs(), precision=prad.PRAD_FP32,
                       photon_capacity=1 << 16, max_particles=wl.n)
    st = ctx.to_device(wl.state)
    ctx.push_emit(st, 2)
    assert ctx.energy_budget()[2]["wiggler_invalid"] == 0
    ctx.close()
