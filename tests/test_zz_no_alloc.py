"""Allocation-free totals, prad_ledger_totals_noalloc.

This entry point serves callers that cannot allocate device memory where
they need the ledger totals: a host code that owns a fixed device memory
pool, or a time loop in which a cudaMalloc (which synchronises the device and
may fail once the pool holds the memory) is not acceptable.  It keeps its
reduction partials in a static device array shared by every call.

Checked through the C ABI against prad_energy_budget on the same ledgers, on
two calls in a row (the second call finds the shared array as the first left
it), then on a smaller input after a larger one, and for the size limit.
This file is collected last so a first failure here comes after every other
test has run; it also passes alone in a fresh process.
"""
import math

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


def _totals(le, lr):
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    prad.prad_ledger_totals_noalloc(le.data_ptr(), lr.data_ptr(), le.numel(), out.data_ptr(),
                                    torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_noalloc_totals_match_energy_budget_on_two_calls():
    wl = W.plane_wave(a0=300.0, n=300_000 + 11, seed=4)
    ctx = prad.Context(wl.problem_kwargs(), precision=prad.PRAD_FP32,
                       photon_capacity=1 << 22, max_particles=wl.n)
    st = ctx.to_device(wl.state)
    ctx.push_emit(st, 25)
    emitted, rr, _ = ctx.energy_budget()
    le, lr = ctx.ledger()          # caller-owned device copies of the ledgers
    ctx.close()
    for _ in range(2):
        got = _totals(le, lr)
        assert got[0] == pytest.approx(emitted, rel=1e-13)
        assert got[1] == pytest.approx(rr, rel=1e-13)
        assert got[1] == pytest.approx(math.fsum(lr.cpu().numpy()), rel=1e-14)
    # a smaller input after a larger one: no partial of the earlier call leaks
    small_e, small_r = le[:1000].clone(), lr[:1000].clone()
    got = _totals(small_e, small_r)
    assert got[0] == pytest.approx(math.fsum(small_e.cpu().numpy()), rel=1e-14)
    assert got[1] == pytest.approx(math.fsum(small_r.cpu().numpy()), rel=1e-14)
    # empty input
    assert np.array_equal(_totals(small_e[:0], small_r[:0]), [0.0, 0.0])


def test_noalloc_rejects_sizes_beyond_the_static_limit():
    a = torch.zeros(4, dtype=torch.float64, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    with pytest.raises(prad.PradError) as ei:
        prad.prad_ledger_totals_noalloc(a.data_ptr(), a.data_ptr(), (1 << 28) + 1,
                                        out.data_ptr(), None)
    assert ei.value.code == prad.PRAD_ERR_ARG and "268435456" in str(ei.value)
    # the message describes the last call only: empty after a call that succeeds
    prad.prad_ledger_totals_noalloc(a.data_ptr(), a.data_ptr(), a.numel(), out.data_ptr(), None)
    torch.cuda.synchronize()
    assert prad.load_library().prad_ledger_totals_noalloc_error() == b""
    assert np.array_equal(out.cpu().numpy(), [0.0, 0.0])
