"""The bench's multi-GPU form is N independent replicas: host-side logic of
the rank reduction checked with two gloo ranks on the CPU (no GPU): every
rank sees the slowest rank's time, the whole-job rate counts every rank's
work, and replicas draw disjoint particle ids and their own seeds."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      RANK=str(rank), WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        env = bench.dist_env()
        local = 1.0 + 0.5 * rank          # rank r took 1 + r/2 seconds
        t = bench.max_over_ranks(local, "cpu")
        out.put((rank, env, t, bench.job_rate(1e6, t, ws), bench.rank_inputs(rank, 1000)))
    finally:
        dist.destroy_process_group()


def test_two_rank_reduction_and_replica_inputs():
    ws = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(ws))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, env, t, rate, inputs in res:
        assert env == (ws, rank, rank)
        assert t == 1.5                   # the slowest rank's time, on every rank
        assert rate == pytest.approx(2 * 1e6 / 1.5)
    ids = [set(range(r[4]["pid0"], r[4]["pid0"] + 1000)) for r in res]
    assert not ids[0] & ids[1]
    assert res[0][4]["seed"] != res[1][4]["seed"]


def test_single_process_needs_no_group():
    assert bench.max_over_ranks(2.5, "cpu") == 2.5
    assert bench.job_rate(10.0, 2.0, 1) == 5.0


def test_captured_traffic_reported_only_for_its_sources_and_workload(monkeypatch):
    """The bench attaches the ncu-captured DRAM bytes to its roofline objects
    only while the kernel sources are the captured ones and the launch is the
    captured workload; otherwise the field is null."""
    sha = bench.kernel_sha()
    monkeypatch.setitem(bench.NCU_TRAFFIC, "src_sha256", sha)
    monkeypatch.setitem(bench.NCU_TRAFFIC, "fused", 123)
    assert bench.ncu_traffic("fused") == 123
    assert bench.ncu_traffic("fused", same_workload=False) is None
    monkeypatch.setitem(bench.NCU_TRAFFIC, "src_sha256", "0" * 64)
    assert bench.ncu_traffic("fused") is None
