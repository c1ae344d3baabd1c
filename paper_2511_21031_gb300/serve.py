"""Continuous-batching request loop for bubble-source solves.

A request is one independent ensemble (cells x bins, forcing, n_steps flow
steps).  The engine keeps every admitted request's state resident in one
Batch arena and advances all of them together, one flow step per iteration,
with the batched persistent kernel:

  each iteration
    1. requests whose arrival time has passed join the FIFO wait queue;
    2. queued requests are admitted, in order, while a slot and contiguous
       arena space exist (admission by device memory; a refused head of queue
       waits for a release, so no request starves);
    3. every active request's pressure for its next step is evaluated on the
       device and bound to its slot;
    4. one batched step (CUDA-graph replay) advances every active request;
    5. requests that reached their last step are read out (status, moments)
       and released, which frees arena space for the queue.

Requests that arrive while others are running are therefore admitted at the
next iteration boundary and share the following launches with them.  Each
request's arithmetic is independent of the others (the kernel owns every
(cell, bin) of a slot alone), so its result is the same alone and in the mix.
Latency is completion time minus arrival time on the engine's clock.

Cancellation and timeouts are host-side and act at iteration boundaries, when
no launch is in flight: a cancelled request (cancel(rid)) or one still
unfinished `timeout` seconds after its arrival leaves the queue, or, if
active, is released with the work done so far; it completes with status
"cancelled" or "timeout" and no result, and its slot and arena space go to
the queue.
"""
from __future__ import annotations

import collections
import dataclasses
import math
import time
from typing import Dict, List, Optional

import numpy as np

from .batch import Batch


@dataclasses.dataclass
class _Active:
    req: object
    slot: int
    step: int
    theta: object
    p: object
    moments: object
    admitted_at: float


@dataclasses.dataclass
class Completion:
    rid: int
    arrival: float
    admitted: float          # NaN for a request that never left the queue
    done: float
    bin_steps: int           # work done (all of it for status "done")
    flags: int
    attempts: int
    moments: Optional[np.ndarray] = None
    status: str = "done"     # "done", "cancelled" or "timeout"

    @property
    def latency(self):
        return self.done - self.arrival


class ServingEngine:
    def __init__(self, capacity_bins: int, max_slots: int = 256, precision: str = "mixed",
                 max_bins: int = 31, launch=None, graph: bool = True, keep_moments: bool = False,
                 stream=None):
        import torch
        self.torch = torch
        self.batch = Batch(max_slots=max_slots, precision=precision, capacity_bins=capacity_bins,
                           max_bins=max_bins)
        if launch:
            self.batch.set_launch(*launch)
        self.graph = graph
        self.keep_moments = keep_moments
        self.stream = stream or torch.cuda.Stream()
        self.dev = torch.device("cuda", torch.cuda.current_device())
        self._cancelled = set()

    def cancel(self, rid: int):
        """Cancel request rid: it leaves the queue, or its slot is released, at the next
        iteration boundary (safe to call from another thread while run() serves)."""
        self.__dict__.setdefault("_cancelled", set()).add(rid)

    def _admit(self, req, now):
        w = req.work
        slot = self.batch.try_admit(w.n_cells, w.n_bins, stream=self.stream, s_lognormal=w.s,
                                    R0ref=w.R0ref, span_K=w.span_K, alpha0=w.alpha0, **w.fluid)
        if slot is None:
            return None
        t = self.torch
        theta = t.as_tensor(w.theta, device=self.dev)
        p = t.empty(w.n_cells, dtype=t.float64, device=self.dev)
        m = t.empty((7, w.n_cells), dtype=t.float64, device=self.dev)
        self.batch.bind(slot, p, w.dt, moments=m)
        return _Active(req, slot, 0, theta, p, m, now)

    def run(self, requests: List, clock: str = "wall", max_iterations: int = 10 ** 9,
            timeout: Optional[float] = None) -> Dict:
        """Serve the requests (sorted by arrival).  clock="wall": arrivals are
        released by wall time since start; clock="virtual": time advances by the
        GPU time of each iteration only (arrivals are released at iteration
        boundaries in virtual time).  timeout: seconds after its arrival within
        which a request must finish, else it is dropped (status "timeout")."""
        t = self.torch
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        waiting = collections.deque()
        active: List[_Active] = []
        done: List[Completion] = []
        t0 = time.perf_counter()
        vnow = 0.0
        iters = 0
        concurrency = []
        busy_s = 0.0
        total_bin_steps = 0

        def now():
            return time.perf_counter() - t0 if clock == "wall" else vnow

        cancelled = self.__dict__.setdefault("_cancelled", set())

        def dropped(req, tn):
            if req.rid in cancelled:
                return "cancelled"
            if timeout is not None and tn - req.arrival > timeout:
                return "timeout"
            return None

        while (pending or waiting or active) and iters < max_iterations:
            tn = now()
            if not active and not waiting and pending and pending[0].arrival > tn:
                # idle: jump (virtual) or sleep (wall) to the next arrival
                if clock == "wall":
                    time.sleep(max(0.0, pending[0].arrival - tn))
                else:
                    vnow = pending[0].arrival
                tn = now()
            while pending and pending[0].arrival <= tn:
                waiting.append(pending.popleft())
            # cancellations and timeouts, at the boundary (no launch in flight)
            if cancelled or timeout is not None:
                for r in [r for r in waiting if dropped(r, tn)]:
                    waiting.remove(r)
                    done.append(Completion(r.rid, r.arrival, float("nan"), tn, 0, 0, 0,
                                           status=dropped(r, tn)))
                keep = []
                for a in active:
                    why = dropped(a.req, tn)
                    if why is None:
                        keep.append(a)
                        continue
                    w = a.req.work
                    st = self.batch.status(a.slot, stream=self.stream)
                    self.batch.release(a.slot, stream=self.stream)
                    done.append(Completion(a.req.rid, a.req.arrival, a.admitted_at, tn,
                                           w.n_cells * w.n_bins * a.step, st["flags"], st["n_attempts"],
                                           status=why))
                active = keep
            while waiting:
                a = self._admit(waiting[0], tn)
                if a is None:
                    break
                waiting.popleft()
                active.append(a)
            if not active:
                if waiting:
                    raise RuntimeError(f"request {waiting[0].rid} can never be admitted: "
                                       f"{waiting[0].work.bins_total} bin-states exceed the arena")
                continue
            # pressure of each active request's next step, then one batched step
            with t.cuda.stream(self.stream):
                for a in active:
                    w = a.req.work
                    tt = (a.step + 0.5) * w.dt
                    p0 = w.fluid["p0"]
                    t.sin(a.theta + 2.0 * math.pi * w.freq * tt, out=a.p)
                    a.p.mul_(w.amp * p0).add_(p0)
                e0 = t.cuda.Event(enable_timing=True)
                e1 = t.cuda.Event(enable_timing=True)
                e0.record(self.stream)
                self.batch.step(graph=self.graph, stream=self.stream)
                e1.record(self.stream)
            e1.synchronize()
            gpu_s = e0.elapsed_time(e1) * 1e-3
            busy_s += gpu_s
            if clock == "virtual":
                vnow += gpu_s
            concurrency.append(len(active))
            iters += 1
            tdone = now()
            still = []
            for a in active:
                a.step += 1
                w = a.req.work
                total_bin_steps += w.n_cells * w.n_bins
                if a.step >= w.n_steps:
                    st = self.batch.status(a.slot, stream=self.stream)
                    mom = a.moments.cpu().numpy() if self.keep_moments else None
                    self.batch.release(a.slot, stream=self.stream)
                    done.append(Completion(a.req.rid, a.req.arrival, a.admitted_at, tdone,
                                           w.n_cells * w.n_bins * w.n_steps, st["flags"],
                                           st["n_attempts"], mom))
                else:
                    still.append(a)
            active = still
        elapsed = now()
        cancelled.clear()  # a cancellation applies to the run it was made for
        ok = [c for c in done if c.status == "done"]
        lat = np.array([c.latency for c in ok]) if ok else np.array([float("nan")])
        return {
            "completed": len(ok), "cancelled": sum(c.status == "cancelled" for c in done),
            "timed_out": sum(c.status == "timeout" for c in done),
            "iterations": iters, "elapsed_s": elapsed, "gpu_busy_s": busy_s,
            "bin_steps": total_bin_steps,
            "throughput_bin_steps_per_s": total_bin_steps / elapsed if elapsed > 0 else float("nan"),
            "gpu_throughput_bin_steps_per_s": total_bin_steps / busy_s if busy_s > 0 else float("nan"),
            "latency_s": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                          "max": float(np.max(lat))},
            "concurrency": {"mean": float(np.mean(concurrency)) if concurrency else 0.0,
                            "max": int(max(concurrency)) if concurrency else 0},
            "flags": int(np.bitwise_or.reduce([c.flags for c in done])) if done else 0,
            "completions": done,
        }

    def close(self):
        self.batch.close()


def main(argv=None):
    """Serve a seeded request stream; prints one JSON line per rate."""
    import argparse
    import json

    import torch

    from . import workloads
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--requests", type=int, default=16)
    ap.add_argument("--rates", type=float, nargs="+", default=[200.0])
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--capacity-bins", type=int, default=2_000_000_000)
    ap.add_argument("--clock", default="wall", choices=("wall", "virtual"))
    ap.add_argument("--launch", type=int, nargs=3, default=None)
    ap.add_argument("--timeout", type=float, default=None,
                    help="seconds after arrival within which a request must finish")
    args = ap.parse_args(argv)
    torch.cuda.set_device(0)
    for rate in args.rates:
        reqs = workloads.request_stream(n=args.requests, rate=rate, n_steps=args.steps)
        eng = ServingEngine(capacity_bins=args.capacity_bins, launch=args.launch)
        rep = eng.run(reqs, clock=args.clock, timeout=args.timeout)
        eng.close()
        rep.pop("completions")
        print(json.dumps(dict(rate=rate, requests=args.requests, **rep)), flush=True)


if __name__ == "__main__":
    main()
