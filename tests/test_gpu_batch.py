"""Batched ensembles in one persistent kernel (work items from an atomic
counter), CUDA-graph replay and the autotuner, GPU through the C ABI.

Per ensemble the batch must give exactly what prad_push_emit gives for the
same field and Philox ensemble word (same per-particle arithmetic), and both
must match the FP64 oracle; the uneven-size workload of 256 ensembles runs at
full size under the graph with autotuned launch parameters and is checked on
sampled particles.
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


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    prad.load_library()


def _f32(wl):
    w = wl.subset(np.arange(wl.n))
    w.state = {k: v.astype(np.float32).astype(np.float64) for k, v in w.state.items()}
    return w


def _small_set(seed=3):
    es = W.ensembles(count=7, nmin=50, nmax=30_000, nsteps=30, seed=seed)
    wls = [_f32(w) for w in es.workloads]
    wls[2] = wls[2].subset(np.arange(0))   # an empty ensemble
    return wls


def _ctx(wls, **kw):
    total = sum(w.n for w in wls)
    return prad.Context(wls[0].problem_kwargs(), precision=prad.PRAD_FP32,
                        photon_capacity=1 << 22, max_particles=max(total, 1), **kw)


def _collect(ctx, states):
    torch.cuda.synchronize()
    ph = ctx.photons(on_device=False)
    e, l, s = ctx.energy_budget()
    le, ll = ctx.ledger()
    return ([{k: v.double().cpu().numpy() for k, v in st.items()} for st in states],
            ph, e, l, s, le.cpu().numpy(), ll.cpu().numpy())


def _keys(ph):
    return np.sort(ph["pid"].numpy().astype(np.int64) * 2**32 + ph["step"].numpy())


def test_batch_equals_individual_launches():
    wls = _small_set()
    nsteps = 30
    total = sum(w.n for w in wls)
    ctx = _ctx(wls)
    sts = [ctx.to_device(w.state) for w in wls]
    ens = ctx.ensembles(sts, [w.problem_kwargs() for w in wls])
    ctx.push_emit_batch(ens, nsteps)
    states_a, ph_a, _, _, _, le_a, ll_a = _collect(ctx, sts)
    ctx.close()
    # the same ensembles one at a time through prad_push_emit (same field,
    # ensemble word, ids and ledger slice, all steps in one launch)
    keys, off = [], 0
    for k, w in enumerate(wls):
        if w.n:
            c2 = prad.Context(w.problem_kwargs(), precision=prad.PRAD_FP32,
                              photon_capacity=1 << 22, max_particles=total, ensemble=k,
                              steps_per_launch=nsteps)
            st = c2.to_device(w.state)
            c2.push_emit(st, nsteps, pid0=off, ledger_offset=off)
            torch.cuda.synchronize()
            ph2 = c2.photons(on_device=False)
            le2, ll2 = c2.ledger()
            for name in ("x", "y", "z", "ux", "uy", "uz"):
                np.testing.assert_array_equal(states_a[k][name], st[name].double().cpu().numpy())
            sl = slice(off, off + w.n)
            np.testing.assert_array_equal(ll_a[sl], ll2.cpu().numpy()[sl])
            np.testing.assert_array_equal(le_a[sl], le2.cpu().numpy()[sl])
            keys.append(_keys(ph2))
            c2.close()
        off += w.n
    np.testing.assert_array_equal(_keys(ph_a), np.sort(np.concatenate(keys)))


@pytest.fixture(scope="module")
def trained_params():
    """The learned sampler trained on 2 x 10^8 device-generated samples."""
    wl = W.plane_wave(a0=300.0, n=16)
    ctx = prad.Context(wl.problem_kwargs(), precision=prad.PRAD_FP32,
                       photon_capacity=1 << 10, max_particles=16)
    ctx.mlp_train(3052, 65536, 3e-3, seed=7)
    p = ctx.mlp_weights()
    ctx.close()
    return p


def _records(ph):
    key = ph["pid"].numpy().astype(np.int64) * 2**32 + ph["step"].numpy()
    o = np.argsort(key)
    return key[o], np.stack([ph[c].numpy()[o] for c in ("eps", "weight", "x", "nx")], 1)


def test_batch_learned_sampler_equals_individual_launches(trained_params):
    """Learned sampler in the batch kernel: queued emissions are evaluated
    before a block moves to another ensemble, so every record (its x from the
    network row of its own emission) equals the per-ensemble launch's."""
    wls = _small_set(seed=4)
    nsteps = 25
    total = sum(w.n for w in wls)
    smp = prad.PRAD_SAMPLER_MLP_FALLBACK
    ctx = _ctx(wls, sampler=smp, batch_chunk=512)
    ctx.mlp_set_weights(trained_params)
    sts = [ctx.to_device(w.state) for w in wls]
    ens = ctx.ensembles(sts, [w.problem_kwargs() for w in wls])
    ctx.push_emit_batch(ens, nsteps)
    states_a, ph_a, e_a, _, s_a, le_a, ll_a = _collect(ctx, sts)
    ctx.close()
    keys, recs, off = [], [], 0
    for k, w in enumerate(wls):
        if w.n:
            c2 = prad.Context(w.problem_kwargs(), precision=prad.PRAD_FP32, sampler=smp,
                              photon_capacity=1 << 22, max_particles=total, ensemble=k,
                              steps_per_launch=nsteps)
            c2.mlp_set_weights(trained_params)
            st = c2.to_device(w.state)
            c2.push_emit(st, nsteps, pid0=off, ledger_offset=off)
            torch.cuda.synchronize()
            ph2 = c2.photons(on_device=False)
            le2, ll2 = c2.ledger()
            for name in ("x", "y", "z", "ux", "uy", "uz"):
                np.testing.assert_array_equal(states_a[k][name], st[name].double().cpu().numpy())
            sl = slice(off, off + w.n)
            np.testing.assert_array_equal(ll_a[sl], ll2.cpu().numpy()[sl])
            np.testing.assert_allclose(le_a[sl], le2.cpu().numpy()[sl], rtol=1e-12, atol=0)
            kk, rr = _records(ph2)
            keys.append(kk)
            recs.append(rr)
            c2.close()
        off += w.n
    ka, ra = _records(ph_a)
    kb = np.concatenate(keys)
    o = np.argsort(kb)
    np.testing.assert_array_equal(ka, kb[o])
    np.testing.assert_array_equal(ra, np.concatenate(recs)[o])
    assert s_a["records"] == ka.size > 1000
    assert s_a["mlp_fallback"] < 1e-3 * ka.size + 5


def test_batch_matches_oracle_per_ensemble():
    wls = _small_set(seed=5)
    ctx = _ctx(wls)
    sts = [ctx.to_device(w.state) for w in wls]
    ens = ctx.ensembles(sts, [w.problem_kwargs() for w in wls])
    ctx.push_emit_batch(ens, 20)
    states, ph, e, l, s, le, ll = _collect(ctx, sts)
    ctx.close()
    off = 0
    for k, w in enumerate(wls):
        if w.n == 0:
            continue
        sel = np.arange(0, w.n, max(1, w.n // 50))
        sub = w.subset(sel)
        prob = O.Problem(**{**sub.problem_kwargs(), "ensemble": k})
        st = sub.copy_state()
        r = O.run(prob, st, 20, pid=(off + sel).astype(np.uint32), capacity=1 << 16)
        ug = np.stack([states[k][c][sel] for c in ("ux", "uy", "uz")], 1)
        uo = np.stack([st[c] for c in ("ux", "uy", "uz")], 1)
        rel = np.abs(ug - uo).max(1) / np.linalg.norm(uo, axis=1)
        assert rel.max() <= 1e-5, (k, rel.max())
        np.testing.assert_allclose(ll[off + sel], r["ledger"]["ll"], rtol=1e-4)
        off += w.n


def test_graph_replay_equals_direct_launches():
    wls = _small_set(seed=9)
    stream = torch.cuda.Stream()
    res = []
    for use_graph in (False, True, True):
        with torch.cuda.stream(stream):
            ctx = _ctx(wls, use_graph=use_graph, stream=stream)
            sts = [ctx.to_device(w.state) for w in wls]
            ens = ctx.ensembles(sts, [w.problem_kwargs() for w in wls])
            ctx.push_emit_batch(ens, 12)
            # a second call replays the captured graph (same shape, new t0)
            ens2 = ctx.ensembles(sts, [w.problem_kwargs() for w in wls], t0=12)
            ctx.push_emit_batch(ens2, 12)
            stream.synchronize()
            # the busy-clock array is zeroed and filled inside the graph too
            eff, ctas = ctx.batch_balance()
            assert 0.0 < eff <= 1.0 and ctas >= 1
            res.append(_collect(ctx, sts))
            ctx.close()
    for k in range(len(wls)):
        for c in ("x", "ux", "uy", "uz"):
            np.testing.assert_array_equal(res[0][0][k][c], res[1][0][k][c])
            np.testing.assert_array_equal(res[0][0][k][c], res[2][0][k][c])
    np.testing.assert_array_equal(_keys(res[0][1]), _keys(res[1][1]))
    assert res[0][3] == res[1][3]


def test_batch_balance_needs_a_batched_call():
    wls = _small_set(seed=5)
    ctx = _ctx(wls)
    with pytest.raises(prad.PradError) as ei:
        ctx.batch_balance()
    assert ei.value.code == prad.PRAD_ERR_STATE
    sts = [ctx.to_device(w.state) for w in wls]
    ctx.push_emit_batch(ctx.ensembles(sts, [w.problem_kwargs() for w in wls]), 4)
    eff, ctas = ctx.batch_balance()
    # a persistent launch: at most one CTA per resident slot of every SM
    assert 0.0 < eff <= 1.0
    assert 1 <= ctas <= torch.cuda.get_device_properties(0).multi_processor_count * 64
    ctx.close()


def test_autotune_leaves_state_and_caches():
    wls = _small_set(seed=11)
    ctx = _ctx(wls)
    sts = [ctx.to_device(w.state) for w in wls]
    before = [{k: v.clone() for k, v in st.items()} for st in sts]
    ens = ctx.ensembles(sts, [w.problem_kwargs() for w in wls])
    t = ctx.autotune_batch(ens, probe_steps=8, sample=2048)
    assert t["candidates"] > 4 and t["particle_steps_per_s"] > 0
    assert t["block_size"] in (128, 256) and t["batch_chunk"] in (512, 1024, 2048, 4096)
    for a, b in zip(sts, before):
        for k in a:
            assert torch.equal(a[k], b[k])
    _, _, st = ctx.energy_budget()
    assert st["records"] == 0
    t2 = ctx.autotune_batch(ens, probe_steps=8, sample=2048)
    assert t2["candidates"] == 0 and t2["batch_chunk"] == t["batch_chunk"]
    ctx.push_emit_batch(ens, 5)       # runs with the tuned shape
    ctx.close()


@pytest.mark.parametrize("sampler", ["table", "mlp_fallback"])
def test_full_size_uneven_ensembles_graph_autotuned(sampler, trained_params):
    """256 ensembles, sizes log-uniform in [1e3, 1e6], a0 ~ U[50, 500], plane
    wave or constant B, 500 steps in one persistent kernel per call under a
    captured graph with autotuned launch parameters, with the table sampler
    and with the learned sampler (table fallback); 4 sampled electrons of
    every 16th ensemble against the oracle."""
    es = W.ensembles(count=256, nsteps=500, seed=1)
    wls = [_f32(w) for w in es.workloads]
    total = sum(w.n for w in wls)
    smp = (prad.PRAD_SAMPLER_TABLE if sampler == "table" else prad.PRAD_SAMPLER_MLP_FALLBACK)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctx = prad.Context(wls[0].problem_kwargs(), precision=prad.PRAD_FP32,
                           photon_capacity=int(0.08 * total * 500) + (1 << 20),
                           max_particles=total, use_graph=True, stream=stream, sampler=smp)
        if sampler != "table":
            ctx.mlp_set_weights(trained_params)
        sts = [ctx.to_device(w.state) for w in wls]
        ens = ctx.ensembles(sts, [w.problem_kwargs() for w in wls])
        tune = ctx.autotune_batch(ens, probe_steps=10, sample=4096)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        ctx.push_emit_batch(ens, 500)
        ev1.record(stream)
        stream.synchronize()
    secs = ev0.elapsed_time(ev1) / 1e3
    eff, ctas = ctx.batch_balance()
    print(f"\nbatched ({sampler}): {total} particles x 500 steps in {secs * 1e3:.1f} ms = "
          f"{total * 500 / secs:.3e} particle-steps/s, tuning {tune}, "
          f"load balance {eff:.3f} over {ctas} CTAs")
    # work items of at most batch_chunk particles handed out by an atomic
    # counter keep the CTAs' busy times within a few items of each other
    assert 0.5 < eff <= 1.0
    e, l, s = ctx.energy_budget()
    assert s["dropped"] == 0 and s["status"] == 0
    off = 0
    for k, w in enumerate(wls):
        if k % 16 == 0:
            sel = np.array([0, w.n // 3, w.n // 2, w.n - 1])
            sub = w.subset(sel)
            prob = O.Problem(**{**sub.problem_kwargs(), "ensemble": k})
            st = sub.copy_state()
            pid = (off + sel).astype(np.uint32)
            r = O.run(prob, st, 500, pid=pid, capacity=1 << 16)
            g = sts[k]
            gs = {c: g[c][torch.from_numpy(sel).cuda()].double().cpu().numpy()
                  for c in ("ux", "uy", "uz")}
            # 500 FP32 steps of gyration / wave motion with the LL kick: every
            # particle within max(1e-5, its float32 envelope), the oracle's own
            # departure when its state is held in float32
            env = FE.envelope(prob, sub.copy_state(), 500, st, pid=pid)
            FE.assert_within(FE.momentum_rel(gs, st), env)
        off += w.n
    assert e / l == pytest.approx(1.0, abs=0.05)
    ctx.close()
