"""Continuous batching: requests admitted by device memory as slots free up,
their steps sharing launches with the requests already running, every result
identical alone and in the mix, and a request cancelled while running released
without disturbing the others."""
import numpy as np
import pytest

from paper_2511_21031_gb300 import workloads
from paper_2511_21031_gb300.serve import ServingEngine

pytestmark = pytest.mark.gpu


def _requests(n=10, rate=2e4, seed=31):
    return workloads.request_stream(n=n, rate=rate, seed=seed, n_steps=25, edge_lo=6, edge_hi=16,
                                    edge_median=10.0)


def test_each_result_is_the_same_alone_and_in_the_mix():
    reqs = _requests()
    assert len({r.work.n_cells for r in reqs}) > 2 and len({r.work.n_bins for r in reqs}) == 2
    cap = sum(r.work.bins_total for r in reqs)
    eng = ServingEngine(capacity_bins=cap, max_slots=len(reqs), keep_moments=True)
    mix = eng.run(reqs, clock="virtual")
    eng.close()
    assert mix["completed"] == len(reqs) and mix["flags"] == 0
    assert mix["concurrency"]["max"] >= 2                       # work overlapped on the device
    by_id = {c.rid: c for c in mix["completions"]}
    for r in reqs:
        e = ServingEngine(capacity_bins=r.work.bins_total, max_slots=1, keep_moments=True)
        alone = e.run([r], clock="virtual")
        e.close()
        a = alone["completions"][0]
        np.testing.assert_array_equal(a.moments, by_id[r.rid].moments)
        assert a.attempts == by_id[r.rid].attempts


def test_admission_waits_for_memory_and_every_request_completes():
    reqs = _requests(n=12, seed=32)
    biggest = max(r.work.bins_total for r in reqs)
    cap = 2 * biggest + 10                                      # room for ~2-3 requests at a time
    eng = ServingEngine(capacity_bins=cap, max_slots=8)
    rep = eng.run(reqs, clock="virtual")
    eng.close()
    assert rep["completed"] == len(reqs)
    assert rep["concurrency"]["max"] < len(reqs)                # memory, not arrivals, limited it
    comp = sorted(rep["completions"], key=lambda c: c.rid)
    waits = [c.admitted - c.arrival for c in comp]
    assert max(waits) > 0                                       # some requests queued for memory
    assert all(c.done >= c.admitted >= c.arrival - 1e-12 for c in comp)
    assert rep["latency_s"]["p99"] >= rep["latency_s"]["p50"] > 0


def test_request_larger_than_the_arena_is_reported():
    reqs = _requests(n=2, seed=33)
    eng = ServingEngine(capacity_bins=10, max_slots=2)
    with pytest.raises(RuntimeError):
        eng.run(reqs, clock="virtual")
    eng.close()


def test_request_cancelled_while_running_leaves_the_others_untouched():
    """A request cancelled after five launches is released at the next iteration boundary with
    the work done so far; every other request's result is still the one it gets alone."""
    reqs = _requests(n=6, seed=34)
    cap = sum(r.work.bins_total for r in reqs)
    eng = ServingEngine(capacity_bins=cap, max_slots=len(reqs), keep_moments=True)
    victim = reqs[0].rid
    launches = [0]
    step = eng.batch.step

    def step_then_cancel(*a, **k):
        step(*a, **k)
        launches[0] += 1
        if launches[0] == 5:
            eng.cancel(victim)
    eng.batch.step = step_then_cancel
    mix = eng.run(reqs, clock="virtual")
    eng.close()
    assert (mix["completed"], mix["cancelled"]) == (len(reqs) - 1, 1)
    by_id = {c.rid: c for c in mix["completions"]}
    v = by_id[victim]
    assert v.status == "cancelled" and v.moments is None
    assert 0 < v.bin_steps < reqs[0].work.bins_total * reqs[0].work.n_steps
    for r in reqs[1:]:
        e = ServingEngine(capacity_bins=r.work.bins_total, max_slots=1, keep_moments=True)
        alone = e.run([r], clock="virtual")
        e.close()
        a = alone["completions"][0]
        assert by_id[r.rid].status == "done"
        np.testing.assert_array_equal(a.moments, by_id[r.rid].moments)
        assert a.attempts == by_id[r.rid].attempts
