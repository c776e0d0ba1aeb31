"""Benchmark: particle-steps/s of the emission hot path on synthetic workloads.

Default workload (one bench step): the counter-propagating circularly
polarised plane wave, lambda = 0.8 um, 2^20 electrons with gamma = 1000 along
-x plus 1% Gaussian momentum spread, FP32 push with FP64 ledger, 20 laser
periods at 200 steps per period, table sampler, for each a0 in {100, 300, 500}
(3 x 2^20 x 4000 = 1.26e10 particle-steps per bench step).  Every particle-step
runs the whole path: gather, Boris push, H_eff, omega_c, LL kick and ledger,
Philox, S(x) sampling with the F table, photon append, emitted-energy ledger.

Timing: CUDA events on the launching stream around each bench step, L2 flushed
(256 MB write) between steps, max over ranks.  ``--impl reference`` times the
FP64 CPU oracle on the host cores on a bounded sample of the same workload.

Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-steps/s with emission (plain table vs MLP sampler) at <=1% spectral err"

# DRAM bytes (read + write) per launch of the dominant kernels from one-pass
# ncu captures (dram__bytes_read.sum + dram__bytes_write.sum) of the bench's
# own launches, valid for the kernel sources they were taken on (sha256 of
# KERNEL_SOURCES); reported as null once those sources change.
KERNEL_SOURCES = ["paper_1409_5574_gb300/csrc/push_emit.cu",
                  "paper_1409_5574_gb300/csrc/prad_internal.h",
                  "paper_1409_5574_gb300/csrc/mlp_device.cuh"]
NCU_TRAFFIC = {
    "src_sha256": "a8c6e06ab1c74e2aa6321feb8b27ed1ce1129bbdaecf0caa4de5c5c5f09aaac0",
    "fused": 253542724,   # mean bytes per launch over the 30 fused launches of one bench step
    "stream": 1333918720, # bytes per launch, 2^24 particles x 1 step, a0 = 500
}


def kernel_sha() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def ncu_traffic(kind: str, same_workload: bool = True):
    """The captured DRAM bytes per launch, if the kernel sources are the ones
    captured and the launch is the captured workload's."""
    if same_workload and NCU_TRAFFIC["src_sha256"] and NCU_TRAFFIC["src_sha256"] == kernel_sha():
        return NCU_TRAFFIC[kind]
    return None
UNIT = "particle-steps/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="prad", choices=["prad", "reference"])
    ap.add_argument("--particles", type=int, default=1 << 20)
    ap.add_argument("--a0", type=str, default="100,300,500")
    ap.add_argument("--periods", type=int, default=20)
    ap.add_argument("--nsub", type=int, default=0,
                    help="substeps fused per launch (0: tuned default)")
    ap.add_argument("--block", type=int, default=0)
    ap.add_argument("--bps", type=int, default=0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-mlp", action="store_true")
    ap.add_argument("--no-other", action="store_true",
                    help="skip the Yee, a0=500 2^26-electron and batched workloads")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    return ap.parse_args()


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples during the timed region (SM clock, reasons)."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [v.strip() for v in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- helpers
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(seconds: float, device) -> float:
    """The largest of every rank's `seconds` (one all-reduce over the process
    group on `device`); `seconds` itself when no group of more than one rank
    is initialised."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return seconds
    t = torch.tensor([seconds], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, seconds: float, world_size: int) -> float:
    """Whole-job throughput of identical per-rank work timed by the slowest
    rank."""
    return world_size * units_per_rank / seconds


def rank_inputs(rank: int, n: int) -> dict:
    """Seeds and particle-id offset of a rank's replica (independent
    particles: no two ranks share ids or random streams)."""
    return {"seed": 1 + 97 * rank, "pid0": rank * n}


def a0_list(s: str):
    return [float(v) for v in s.split(",") if v.strip()]


def workload_name(args) -> str:
    return (f"CP plane wave, lambda=0.8um, a0 in {{{args.a0}}}, {args.particles} electrons "
            f"gamma=1000 along -x +1% spread, {args.periods * 200} steps (200/period), "
            "FP32 push + FP64 ledger, table sampler, LL kick")


def _oracle_sample(args, budget_s: float):
    """Pick a bounded sample of the workload the oracle finishes in about
    budget_s: the first n electrons, the full step count, every a0."""
    import oracle as O
    from paper_1409_5574_gb300 import workloads as W
    O.lib()
    a0s = a0_list(args.a0)
    nsteps = args.periods * 200
    wl = W.plane_wave(a0=a0s[-1], n=4096, periods=1, seed=11)
    prob = O.Problem(**wl.problem_kwargs())
    O.run(prob, wl.copy_state(), 20, capacity=1 << 20)   # thread-pool start-up
    t = time.perf_counter()
    O.run(prob, wl.copy_state(), 200, capacity=1 << 20)
    rate = 4096 * 200 / (time.perf_counter() - t)
    n = max(64, min(args.particles, int(rate * budget_s / (nsteps * len(a0s)))))
    subs = []
    for a0 in a0s:
        wl = W.plane_wave(a0=a0, n=args.particles, periods=args.periods, seed=1)
        subs.append(wl.subset(slice(0, n)))
    return n, nsteps, subs


def _oracle_step(subs, nsteps) -> int:
    import oracle as O
    ps = 0
    for sub in subs:
        O.run(O.Problem(**sub.problem_kwargs()), sub.copy_state(), nsteps,
              capacity=1 << 22)
        ps += sub.n * nsteps
    return ps


def cpu_baseline(args, budget_s: float) -> dict:
    """The FP64 oracle, as it stands, on the host cores, timed on a bounded
    sample of the same workload."""
    import oracle as O
    n, nsteps, subs = _oracle_sample(args, budget_s)
    t = time.perf_counter()
    ps = _oracle_step(subs, nsteps)
    dt = time.perf_counter() - t
    cores = O.num_threads()
    out = {"value": ps / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"first {n} of {args.particles} electrons x {nsteps} steps for each "
                     f"a0 in {{{args.a0}}} ({ps:.3g} particle-steps, {dt:.1f} s)"}
    # the same oracle on one core, on a sample a quarter of the time long
    n1 = max(16, min(n, int(n * 0.25 / max(1, cores))))
    subs1 = [s.subset(slice(0, n1)) for s in subs]
    O.set_num_threads(1)
    try:
        t = time.perf_counter()
        ps1 = _oracle_step(subs1, nsteps)
        dt1 = time.perf_counter() - t
    finally:
        O.set_num_threads(cores)
    out["single_core"] = {"value": ps1 / dt1, "unit": UNIT,
                          "sample": f"first {n1} electrons of the same sample "
                                    f"({ps1:.3g} particle-steps, {dt1:.1f} s)"}
    return out


# ---------------------------------------------------------------- reference arm
def run_reference(args):
    """The oracle as the reference arm: W warm-up and K timed steps, each step
    the same bounded sample of the workload, on the host cores."""
    import oracle as O
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    per_step = max(0.5, args.cpu_seconds / max(1, args.steps + args.warmup))
    n, nsteps, subs = _oracle_sample(args, per_step)
    for _ in range(args.warmup):
        _oracle_step(subs, nsteps)
    t = time.perf_counter()
    ps = 0
    for _ in range(args.steps):
        ps += _oracle_step(subs, nsteps)
    dt = time.perf_counter() - t
    v = ps / dt
    sample = (f"first {n} of {args.particles} electrons x {nsteps} steps for each a0 in "
              f"{{{args.a0}}} per step")
    cb = {"value": v, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
          "sample": sample}
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(args), "sample": sample},
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------- other workloads
def other_workloads(prad, W, torch, params, rank):
    """One timed run of each of the other workload shapes (particle-steps/s;
    records drained between chunks, drain time excluded): the 2D Yee grid,
    the learned vs table sampler at 2^26 electrons and a0 = 500, and the
    batched uneven ensembles.  `params`: trained network (None: table only)."""
    out = {}

    def timed(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        b.synchronize()
        return a.elapsed_time(b) / 1e3

    # 2D Yee grid 4096^2 (standing wave a0 = 300 + 1% noise), 16M electrons,
    # 1000 steps, sorted by 32 x 32-cell tile every 16 steps
    wl = W.yee2d(nsteps=1000, seed=1 + rank)
    ctx = prad.Context(wl.problem_kwargs(), precision=prad.PRAD_FP32,
                       photon_capacity=1 << 28, max_particles=wl.n, sort_interval=16,
                       steps_per_launch=16)
    st = ctx.to_device(wl.state, with_pid=True)
    ctx.push_emit({k: v[:4096].clone() for k, v in st.items()}, 8)   # warm-up
    ctx.reset()
    ctx.drain()
    secs = 0.0
    for c in range(10):
        secs += timed(lambda: ctx.push_emit(st, 100, t0=100 * c))
        ctx.drain()
    out["yee2d"] = {"value": wl.n * 1000 / secs, "unit": UNIT,
                    "workload": "2D Yee 4096^2 FP32 planes, a0=300 standing wave + 1% noise, "
                                "16777216 electrons in the central 1024^2 cells, 1000 steps, "
                                "tile sort every 16 steps, table sampler"}
    ctx.close()
    del st, wl

    # learned vs table sampler: 2^26 electrons in the CP wave at a0 = 500,
    # 400 steps from the initial state (the emission-heavy first periods)
    n4 = 1 << 26
    wl = W.plane_wave(a0=500.0, n=n4, periods=2, seed=41 + rank)
    res, bal = {}, {}
    for name, smp in (("table", prad.PRAD_SAMPLER_TABLE),
                      ("mlp", prad.PRAD_SAMPLER_MLP_FALLBACK)):
        if smp != prad.PRAD_SAMPLER_TABLE and params is None:
            continue
        ctx = prad.Context(wl.problem_kwargs(), precision=prad.PRAD_FP32, sampler=smp,
                           photon_capacity=1 << 30, max_particles=n4, steps_per_launch=25)
        if smp != prad.PRAD_SAMPLER_TABLE:
            ctx.mlp_set_weights(params)
        st = ctx.to_device(wl.state)
        ctx.push_emit({k: v[:1 << 16].clone() for k, v in st.items()}, 25)   # warm-up
        ctx.reset()
        ctx.drain()
        secs = 0.0
        for c in range(16):
            secs += timed(lambda: ctx.push_emit(st, 25, t0=25 * c))
            ctx.drain()
        res[name] = n4 * 400 / secs
        ctx.close()
        del st
    out["planewave_a0_500_2e26"] = {
        "table": res.get("table"), "mlp": res.get("mlp"), "unit": UNIT,
        "mlp_vs_table": (res["mlp"] / res["table"]) if "mlp" in res else None,
        "workload": "CP plane wave a0=500, 67108864 electrons, 400 steps, 25 steps per launch"}
    del wl

    # batched: 256 ensembles, sizes log-uniform in [1e3, 1e6], a0 ~ U[50, 500],
    # plane wave or constant B, 500 steps, one persistent kernel per call,
    # captured graph, autotuned launch shape
    es = W.ensembles(count=256, nsteps=500, seed=1 + rank)
    total = int(sum(w.n for w in es.workloads))
    res, bal = {}, {}
    for name, smp in (("table", prad.PRAD_SAMPLER_TABLE),
                      ("mlp", prad.PRAD_SAMPLER_MLP_FALLBACK)):
        if smp != prad.PRAD_SAMPLER_TABLE and params is None:
            continue
        s2 = torch.cuda.Stream()
        with torch.cuda.stream(s2):
            ctx = prad.Context(es.workloads[0].problem_kwargs(), precision=prad.PRAD_FP32,
                               sampler=smp, photon_capacity=int(0.1 * total * 100) + (1 << 20),
                               max_particles=total, use_graph=True, stream=s2)
            if smp != prad.PRAD_SAMPLER_TABLE:
                ctx.mlp_set_weights(params)
            sts = [ctx.to_device(w.state) for w in es.workloads]
            probs = [w.problem_kwargs() for w in es.workloads]
            ctx.autotune_batch(ctx.ensembles(sts, probs), probe_steps=10, sample=4096)
            secs, effs = 0.0, []
            for c in range(5):
                ens = ctx.ensembles(sts, probs, t0=100 * c)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(s2)
                ctx.push_emit_batch(ens, 100)
                b.record(s2)
                b.synchronize()
                secs += a.elapsed_time(b) / 1e3
                effs.append(ctx.batch_balance())  # outside the events
                ctx.drain()
            res[name] = total * 500 / secs
            # mean over maximum of the CTAs' busy clocks, per call
            bal[name] = {"efficiency": sum(e for e, _ in effs) / len(effs),
                         "min_efficiency": min(e for e, _ in effs), "ctas": effs[0][1]}
            ctx.close()
            del sts
    out["batched_256"] = {
        "table": res.get("table"), "mlp": res.get("mlp"), "unit": UNIT,
        "mlp_vs_table": (res["mlp"] / res["table"]) if "mlp" in res else None,
        "load_balance": bal,
        "workload": f"256 ensembles, {total} electrons, 500 steps in 5 graph-replayed calls, "
                    "autotuned persistent kernel"}
    return out


# ---------------------------------------------------------------- GPU arm
def run_prad(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1409_5574_gb300 import prad, workloads as W

    ws, rank, local = dist_env()
    if ws > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    stream = torch.cuda.current_stream()
    a0s = a0_list(args.a0)
    nsteps = args.periods * 200
    n = args.particles
    # substeps per launch chosen by the sweep on GB300; the library sizes the
    # persistent grid from the kernel's occupancy unless --bps is given
    nsub = args.nsub if args.nsub > 0 else 400
    bps = args.bps if args.bps > 0 else 0

    # inputs: seeded synthetic states, one per a0, resident in HBM
    ri = rank_inputs(rank, n)
    wls = [W.plane_wave(a0=a0, n=n, periods=args.periods, seed=ri["seed"]) for a0 in a0s]
    cap = int(0.12 * n * nsteps) + (1 << 20)
    ctx = prad.Context(wls[0].problem_kwargs(), precision=prad.PRAD_FP32,
                       photon_capacity=cap, max_particles=n, steps_per_launch=nsub,
                       block_size=args.block, blocks_per_sm=bps)
    init = [ctx.to_device(w.state) for w in wls]
    work = {k: torch.empty_like(v) for k, v in init[0].items()}
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    pid0 = ri["pid0"]
    launches_per_run = math.ceil(nsteps / nsub)

    def one_step():
        recs = 0
        for w, st0 in zip(wls, init):
            ctx.set_fields(w.problem_kwargs())
            for k in work:
                work[k].copy_(st0[k], non_blocking=True)
            ctx.push_emit(work, nsteps, t0=0, pid0=pid0)
            held, dropped = ctx.drain()
            recs += held + dropped
        return recs

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()

    clocks = ClockSampler(dev)
    clocks.start()
    times = []
    records = 0
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    for _ in range(args.steps):
        flush.zero_()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        records += one_step()
        ev1.record(stream)
        ev1.synchronize()
        times.append(ev0.elapsed_time(ev1) / 1e3)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    ck = clocks.stop()
    t_total = max_over_ranks(sum(times), "cuda")
    ps_per_step = len(a0s) * n * nsteps
    value = job_rate(ps_per_step * args.steps, t_total, ws)

    # dominant kernel: average launch duration of the fused push kernel, from
    # events around one run's push_emit only (same stream, same launches)
    ctx.set_fields(wls[-1].problem_kwargs())
    for k in work:
        work[k].copy_(init[-1][k])
    ctx.drain()
    flush.zero_()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ctx.push_emit(work, nsteps, t0=0, pid0=pid0)
    e1.record(stream)
    e1.synchronize()
    run_s = e0.elapsed_time(e1) / 1e3
    held, dropped = ctx.drain()
    per_launch_s = run_s / launches_per_run
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    sm_mhz = peaks.get("sm_max_mhz", 2070.0)
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    # The fused kernel keeps the particle in registers for nsub steps, so it
    # is bound by issue of FP32/INT32 arithmetic: peak = SMs x 128 lanes x
    # clock.  Achieved = algorithmic operations of one particle-step x
    # particle-steps of one launch / launch time, with the hand count of the
    # method's arithmetic: plane-wave gather 9, Boris 42, step averages 12,
    # H_eff 21, clamp / omega_c / chi 9, LL ledger and kick 20, position 8,
    # Philox4x32-10 80, proposal sampling 30, dN and decision 10, emission
    # bookkeeping 8, counters 3 (252).
    alg_ops = 252.0
    alu_peak = nsm * 128 * sm_mhz * 1e6 / 1e12
    achieved = alg_ops * n * nsub / per_launch_s / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "Tops/s",
                "frac": achieved / alu_peak,
                "traffic": ncu_traffic("fused", n == 1 << 20 and nsub == 400 and nsteps == 4000
                                       and a0s == [100.0, 300.0, 500.0]),
                "kernel": "k_push_emit<float, PLANE_WAVE, TABLE, STD>",
                "launch": f"{n} particles x {nsub} steps",
                "ops_per_particle_step": alg_ops,
                "peak_source": f"{nsm} SMs x 128 FP32 lanes x {sm_mhz:.0f} MHz (sm_max_mhz of "
                               "MEASURED_PEAKS.json)"}

    # The same kernel in one-step-per-launch (PIC) mode on a state larger
    # than L2 streams the particles through HBM: report it against the
    # measured copy bandwidth as well.
    ns = 1 << 24
    wl_s = W.plane_wave(a0=a0s[-1], n=ns, periods=1, seed=5 + rank)
    ctx_s = prad.Context(wl_s.problem_kwargs(), precision=prad.PRAD_FP32,
                         photon_capacity=ns * 4, max_particles=ns, steps_per_launch=1)
    st_s = ctx_s.to_device(wl_s.state)
    ctx_s.push_emit(st_s, 4, t0=0)
    ctx_s.drain()
    torch.cuda.synchronize()
    k_s = 20
    e0.record(stream)
    ctx_s.push_emit(st_s, k_s, t0=4)
    e1.record(stream)
    e1.synchronize()
    t_s = e0.elapsed_time(e1) / 1e3 / k_s
    h_s, d_s = ctx_s.drain()
    # algorithmic bytes per particle-step: state R 28 + W 24, LL ledger R+W 16;
    # per record 40 B plus an emit-ledger R+W of 16 B
    rec_s = (h_s + d_s) / k_s
    bytes_s = ns * 68 + rec_s * 56
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    ach_s = bytes_s / t_s / 1e9
    roofline_stream = {"bound": "hbm", "achieved": ach_s, "peak": hbm_peak, "unit": "GB/s",
                       "frac": ach_s / hbm_peak,
                       "traffic": ncu_traffic("stream", a0s[-1] == 500.0),
                       "algorithmic_bytes": bytes_s,
                       "kernel": "k_push_emit<float, PLANE_WAVE, one-step> (next particle "
                                 "prefetched), 1 step per launch",
                       "launch": f"{ns} particles x 1 step (a0={a0s[-1]:g})",
                       "particle_steps_per_s": ns / t_s,
                       "peak_source": "MEASURED_PEAKS.json hbm_gbs" if peaks else "fallback"}
    ctx_s.close()
    del st_s

    # end to end through the public API: pinned host state -> device each run,
    # totals read back each run
    e2e = None
    if not args.no_e2e:
        host = [{k: v.cpu().pin_memory() for k, v in st.items()} for st in init]
        h2d = sum(v.numel() * v.element_size() for st in host for v in st.values())
        d2h = 0

        def e2e_step():
            nonlocal d2h
            d2h = 0
            for w, hs in zip(wls, host):
                ctx.set_fields(w.problem_kwargs())
                for k in work:
                    work[k].copy_(hs[k], non_blocking=True)
                ctx.reset()
                ctx.push_emit(work, nsteps, t0=0, pid0=pid0)
                em, ll, st = ctx.energy_budget()
                ctx.drain()
                d2h += 2 * 8 + 7 * 8 + 4 + 8
        e2e_step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        torch.cuda.synchronize()
        te = max_over_ranks(time.perf_counter() - t0, "cuda")
        e2e = {"value": job_rate(ps_per_step * args.steps, te, ws), "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    # The metric's other arm: the learned sampler (trained here on 10^8
    # device-generated samples) on the same workload and launch shape.
    mlp = None
    if not args.no_mlp:
        torch.cuda.synchronize()
        t_tr = time.perf_counter()
        train_loss = ctx.mlp_train(1526, 65536, 3e-3, seed=7)
        torch.cuda.synchronize()
        t_tr = time.perf_counter() - t_tr
        params = ctx.mlp_weights()
        ctx_m = prad.Context(wls[0].problem_kwargs(), precision=prad.PRAD_FP32,
                             sampler=prad.PRAD_SAMPLER_MLP_FALLBACK, photon_capacity=cap,
                             max_particles=n, steps_per_launch=nsub, block_size=args.block,
                             blocks_per_sm=bps)
        ctx_m.mlp_set_weights(params)
        # spectral error sup_r |G(g(r)) - r| to first order from the device
        # G^-1 table: |ln g - ln G^-1(r)| / (d ln G^-1 / dr) on a 2e5-point grid
        nr = 200_000
        rr = (torch.arange(nr, dtype=torch.float64) + 0.5) / nr
        lg = ctx_m.mlp_eval(rr, torch.full_like(rr, 1000.0),
                            torch.full_like(rr, 1e3)).double().cpu().numpy()
        lt = ctx_m.ginv(rr).double().cpu().numpy()
        dl_dr = np.gradient(lt, rr.numpy())
        bound = float(np.max(np.abs(lg - lt) / dl_dr))

        def mlp_step():
            for w, st0 in zip(wls, init):
                ctx_m.set_fields(w.problem_kwargs())
                for k in work:
                    work[k].copy_(st0[k], non_blocking=True)
                ctx_m.push_emit(work, nsteps, t0=0, pid0=pid0)
                ctx_m.drain()
        mlp_step()
        torch.cuda.synchronize()
        tm = 0.0
        for _ in range(args.steps):
            flush.zero_()
            m0, m1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            m0.record(stream)
            mlp_step()
            m1.record(stream)
            m1.synchronize()
            tm += m0.elapsed_time(m1) / 1e3
        _, _, mst = ctx_m.energy_budget()
        tm = max_over_ranks(tm, "cuda")
        v_mlp = job_rate(ps_per_step * args.steps, tm, ws)
        mlp = {"value": v_mlp, "unit": UNIT, "vs_table": v_mlp / value,
               "spectral_error": bound,
               "spectral_error_how": "first order from the device G^-1 table at gamma=1e3, "
                                     "omega_c dt=1e3 (tests check the exact error against "
                                     "the oracle's G)",
               "train_seconds": t_tr,
               "train_samples": 1526 * 65536, "train_loss": train_loss,
               "mlp_fallback": mst["mlp_fallback"], "sampler": "MLP_FALLBACK (direct scheme)"}
        ctx_m.close()

    others = None
    if not args.no_other:
        ctx.close()
        del init, work
        torch.cuda.empty_cache()
        others = other_workloads(prad, W, torch, None if args.no_mlp else params, rank)

    cb = None
    if rank == 0 and ws == 1:
        cb = cpu_baseline(args, budget_s=args.cpu_seconds)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 * t_total / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": workload_name(args), "particles_per_gpu": n,
                           "a0": a0s, "steps_per_run": nsteps, "sampler": "table",
                           "steps_per_launch": nsub, "ledger": "f64",
                           "l2": "flushed (256 MB write) between timed steps; the "
                                 f"{n * 44 / 1e6:.0f} MB state stays resident across a run",
                           "photon_records_per_step": records / args.steps,
                           "parallelism": f"independent particles, {ws} GPU(s)"},
                "roofline": roofline, "roofline_stream": roofline_stream,
                "mlp_sampler": mlp, "other_workloads": others, "cpu_baseline": cb, "e2e": e2e,
                "gpu_launches": args.steps * len(a0s) * launches_per_run,
                "clocks": ck}
        print(json.dumps(line), flush=True)
    ctx.close()
    if ws > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_prad(args)


if __name__ == "__main__":
    main()
