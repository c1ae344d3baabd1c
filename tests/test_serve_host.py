"""Host logic of the serving loop on the CPU.

The real ServingEngine.run drives a fake batch (an arena of a given number of
bin-states, admission while the bins fit) and a fake CUDA clock (every batched
step costs STEP_S seconds), on the engine's virtual clock, so the schedule is
exact and can be checked by hand: FIFO admission in arrival order, a head of
queue that waits for memory without being overtaken, arrivals joining at the
next iteration boundary, idle gaps, latency and bin-step accounting, the
per-step carrier pressure bound to each slot, and cancellation and timeouts
of queued and active requests.  The device side of the same loop
is covered by tests/test_gpu_serve.py."""
import contextlib
import math

import numpy as np
import pytest
import torch

from paper_2511_21031_gb300 import workloads
from paper_2511_21031_gb300.serve import ServingEngine

STEP_S = 1e-3


class FakeBatch:
    def __init__(self, capacity):
        self.capacity = capacity
        self.used = 0
        self.clock = 0.0
        self.slots = {}
        self.next_slot = 0
        self.admitted = []      # slots in admission order
        self.steps = []         # active slots at each batched step
        self.pressures = {}     # slot -> [p of each step]
        self.on_step = None     # called with the number of steps taken so far

    def try_admit(self, n_cells, n_bins, stream=None, **cfg):
        need = n_cells * n_bins
        if self.used + need > self.capacity:
            return None
        slot = self.next_slot
        self.next_slot += 1
        self.slots[slot] = dict(bins=need, p=None, steps=0)
        self.used += need
        self.admitted.append(slot)
        self.pressures[slot] = []
        return slot

    def bind(self, slot, p, dt, moments=None):
        self.slots[slot]["p"] = p

    def step(self, graph=True, stream=None):
        for slot, s in self.slots.items():
            assert s["p"] is not None, "slot stepped before its pressure was bound"
            self.pressures[slot].append(s["p"].clone().numpy())
            s["steps"] += 1
        self.steps.append(sorted(self.slots))
        self.clock += STEP_S
        if self.on_step:
            self.on_step(len(self.steps))

    def status(self, slot, stream=None):
        return {"flags": 0, "n_attempts": self.slots[slot]["steps"]}

    def release(self, slot, stream=None):
        self.used -= self.slots.pop(slot)["bins"]

    def close(self):
        pass


class _Event:
    def __init__(self, batch):
        self.batch = batch
        self.t = None

    def record(self, stream=None):
        self.t = self.batch.clock

    def synchronize(self):
        pass

    def elapsed_time(self, other):
        return (other.t - self.t) * 1e3


class _Cuda:
    def __init__(self, batch):
        self.batch = batch

    def stream(self, s):
        return contextlib.nullcontext()

    def Event(self, enable_timing=False):
        return _Event(self.batch)


class _Torch:
    """torch with its cuda namespace replaced by the fake clock."""

    def __init__(self, batch):
        self.cuda = _Cuda(batch)

    def __getattr__(self, name):
        return getattr(torch, name)


def engine(capacity):
    fb = FakeBatch(capacity)
    eng = object.__new__(ServingEngine)
    eng.torch = _Torch(fb)
    eng.batch = fb
    eng.graph = True
    eng.keep_moments = False
    eng.stream = None
    eng.dev = torch.device("cpu")
    eng._cancelled = set()
    return eng, fb


def req(rid, arrival, cells, n_bins=3, steps=4):
    w = workloads.Workload(f"r{rid}", cells, n_bins, 0.3, 1e-8, steps, 0.5, 1e5, ("random", 100 + rid))
    return workloads.Request(rid, arrival, w)


def by_rid(rep):
    return {c.rid: c for c in rep["completions"]}


def test_a_request_alone_takes_its_steps_and_is_counted_once():
    eng, fb = engine(capacity=1000)
    rep = eng.run([req(0, 0.0, cells=10, n_bins=3, steps=5)], clock="virtual")
    c = by_rid(rep)[0]
    assert rep["completed"] == 1 and rep["iterations"] == 5
    assert c.admitted == 0.0 and c.latency == pytest.approx(5 * STEP_S, rel=1e-12)
    assert c.bin_steps == 10 * 3 * 5 == rep["bin_steps"]
    assert c.attempts == 5
    assert rep["gpu_busy_s"] == pytest.approx(5 * STEP_S, rel=1e-12)
    assert rep["concurrency"] == {"mean": 1.0, "max": 1}
    assert fb.used == 0 and not fb.slots


def test_head_of_queue_waits_for_memory_and_is_not_overtaken():
    """r1 does not fit beside r0; r2 would, but it arrived after r1 and must not pass it."""
    eng, fb = engine(capacity=100)
    reqs = [req(0, 0.0, cells=20, n_bins=3, steps=3),      # 60 bins
            req(1, 0.0, cells=20, n_bins=3, steps=2),      # 60 bins: waits for r0
            req(2, 0.0, cells=5, n_bins=3, steps=2)]       # 15 bins: fits, but behind r1
    rep = eng.run(reqs, clock="virtual")
    c = by_rid(rep)
    assert fb.admitted == [0, 1, 2]
    assert fb.steps[:3] == [[0], [0], [0]]
    assert fb.steps[3:] == [[1, 2], [1, 2]]
    assert c[1].admitted == pytest.approx(3 * STEP_S) and c[2].admitted == pytest.approx(3 * STEP_S)
    assert c[0].latency == pytest.approx(3 * STEP_S)
    assert c[1].latency == pytest.approx(5 * STEP_S) and c[2].latency == pytest.approx(5 * STEP_S)
    assert rep["concurrency"]["max"] == 2
    assert rep["bin_steps"] == 60 * 3 + 60 * 2 + 15 * 2


def test_arrivals_join_running_requests_at_the_next_iteration_boundary():
    eng, fb = engine(capacity=1000)
    reqs = [req(0, 0.0, cells=10, steps=10), req(1, 2.5 * STEP_S, cells=10, steps=3)]
    rep = eng.run(reqs, clock="virtual")
    c = by_rid(rep)
    assert c[1].admitted == pytest.approx(3 * STEP_S)          # first boundary after 2.5 steps
    assert fb.steps[:3] == [[0]] * 3 and fb.steps[3:6] == [[0, 1]] * 3 and fb.steps[6:] == [[0]] * 4
    assert c[1].latency == pytest.approx(6 * STEP_S - 2.5 * STEP_S)
    assert c[0].latency == pytest.approx(10 * STEP_S)
    assert rep["iterations"] == 10


def test_idle_engine_jumps_to_the_next_arrival():
    eng, fb = engine(capacity=1000)
    rep = eng.run([req(0, 0.0, cells=4, steps=2), req(1, 1.0, cells=4, steps=2)], clock="virtual")
    c = by_rid(rep)
    assert c[1].admitted == pytest.approx(1.0)
    assert c[1].latency == pytest.approx(2 * STEP_S)
    assert rep["elapsed_s"] == pytest.approx(1.0 + 2 * STEP_S)
    assert rep["gpu_busy_s"] == pytest.approx(4 * STEP_S)
    lat = sorted(x.latency for x in c.values())
    assert rep["latency_s"]["p50"] == pytest.approx(np.percentile(lat, 50))
    assert rep["latency_s"]["max"] == pytest.approx(max(lat))


def test_request_larger_than_the_arena_is_reported():
    eng, _ = engine(capacity=50)
    with pytest.raises(RuntimeError, match="can never be admitted"):
        eng.run([req(0, 0.0, cells=20, n_bins=3)], clock="virtual")


def test_each_step_binds_the_workloads_own_carrier_pressure():
    """The pressure bound for step n is the workload's forcing sampled at (n + 1/2) dt, for
    requests admitted at different iterations."""
    eng, fb = engine(capacity=1000)
    reqs = [req(0, 0.0, cells=16, steps=4), req(1, 1.5 * STEP_S, cells=9, steps=3)]
    eng.run(reqs, clock="virtual")
    for slot, r in zip(fb.admitted, reqs):
        ps = fb.pressures[slot]
        assert len(ps) == r.work.n_steps
        for n, p in enumerate(ps):
            np.testing.assert_allclose(p, r.work.pressure_step(n), rtol=1e-15, atol=0.0)


def test_no_cancellation_or_timeout_by_default():
    eng, _ = engine(capacity=1000)
    rep = eng.run([req(0, 0.0, cells=4, steps=3)], clock="virtual")
    assert (rep["completed"], rep["cancelled"], rep["timed_out"]) == (1, 0, 0)
    assert rep["completions"][0].status == "done"


def test_cancelled_queued_request_never_takes_a_slot():
    eng, fb = engine(capacity=100)
    reqs = [req(0, 0.0, cells=20, steps=3), req(1, 0.0, cells=20, steps=2), req(2, 0.0, cells=5, steps=2)]
    eng.cancel(1)                                   # r1 would wait for r0's memory
    rep = eng.run(reqs, clock="virtual")
    c = by_rid(rep)
    assert c[1].status == "cancelled" and math.isnan(c[1].admitted) and c[1].bin_steps == 0
    assert fb.admitted == [0, 1]                    # slots of r0 and r2; r1 never admitted
    assert fb.steps[0] == [0, 1]                    # r2 no longer waits behind r1
    assert c[2].latency == pytest.approx(2 * STEP_S)
    assert (rep["completed"], rep["cancelled"]) == (2, 1)
    assert not eng._cancelled                       # cleared for the next run


def test_cancelled_active_request_is_released_at_the_next_boundary():
    eng, fb = engine(capacity=100)
    reqs = [req(0, 0.0, cells=20, steps=10), req(1, 0.0, cells=20, steps=2)]   # r1 waits for r0
    fb.on_step = lambda n: eng.cancel(0) if n == 4 else None
    rep = eng.run(reqs, clock="virtual")
    c = by_rid(rep)
    assert c[0].status == "cancelled" and c[0].done == pytest.approx(4 * STEP_S)
    assert c[0].bin_steps == 60 * 4 and c[0].attempts == 4
    assert c[1].admitted == pytest.approx(4 * STEP_S) and c[1].status == "done"
    assert fb.steps == [[0]] * 4 + [[1]] * 2 and fb.used == 0
    assert rep["bin_steps"] == 60 * 4 + 60 * 2
    assert rep["latency_s"]["p50"] == pytest.approx(c[1].latency)   # over finished requests only


def test_timeout_drops_queued_and_active_requests():
    eng, fb = engine(capacity=100)
    reqs = [req(0, 0.0, cells=20, steps=10), req(1, 0.0, cells=20, steps=2),
            req(2, 4.0 * STEP_S, cells=5, steps=2)]
    rep = eng.run(reqs, clock="virtual", timeout=4.5 * STEP_S)
    c = by_rid(rep)
    # r0 runs 5 steps and is over its time at the boundary at 5 ms; r1 waited for memory all
    # that time and times out in the queue; r2, queued behind r1 since 4 ms, is admitted at
    # that boundary and finishes
    assert c[0].status == "timeout" and c[0].bin_steps == 60 * 5 and c[0].done == pytest.approx(5 * STEP_S)
    assert c[1].status == "timeout" and math.isnan(c[1].admitted)
    assert c[2].status == "done" and c[2].admitted == pytest.approx(5 * STEP_S)
    assert c[2].latency == pytest.approx(3 * STEP_S)
    assert (rep["completed"], rep["timed_out"], rep["cancelled"]) == (1, 2, 0)
    assert fb.used == 0 and not fb.slots
