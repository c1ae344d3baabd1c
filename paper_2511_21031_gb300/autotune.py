"""Launch-shape autotuner for the bubble kernels.

The batched kernel has three knobs: warps per CTA (each warp advances one bin
of 32 cells at a time), persistent CTAs per SM, and bins taken per
shared-memory grab.  The single-instance step kernel has one: warps per CTA.
The tuner times every candidate on a seeded sample of the real work (a small
batch of sampled instances, or the solver itself), restoring the state before
each candidate so that all see the same trials, and keeps the fastest.  The
choice is cached in a JSON file keyed by GPU, precision and the Nb mix.
"""
from __future__ import annotations

import json
import os
import statistics
import time

import numpy as np

BATCH_CANDIDATES = tuple((w, c, g) for w in (4, 8, 16) for c in (1, 2, 4, 8) for g in (1, 2)) + \
    tuple((1, c, 1) for c in (8, 16, 24, 32))  # one-warp CTAs sum their own terms
SOLVER_CANDIDATES = (1, 2, 4, 8, 16)
DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "autotune_cache.json")


def _gpu_name():
    import torch
    return torch.cuda.get_device_name(torch.cuda.current_device())


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save(path, data):
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def batch_key(instances, precision):
    nbs = sorted({w.n_bins for w in instances})
    cells = sum(w.n_cells for w in instances)
    return f"{_gpu_name()}|batch|{precision}|nb{nbs}|cells~1e{int(np.log10(max(cells, 1)))}"


def _time_events(fn, n):
    import torch
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record()
    for _ in range(n):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / n


# The sample must hold enough 32-cell tiles to give every resident warp several tiles, as the
# real batch does: a sample that leaves SMs idle under one-warp CTAs (one tile per CTA at a
# time) favours wide CTAs that split a tile's bins between their warps.
TILES_PER_RESIDENT_WARP = 8
MAX_WARPS_PER_SM = 64


def sample_instances(instances, sample, min_tiles, seed=0):
    """Indices of the tuning sample: at least `sample` instances drawn in a seeded order, and more
    until their tiles reach `min_tiles` (or every instance is in)."""
    order = np.random.default_rng(seed).permutation(len(instances))
    pick, tiles = [], 0
    for i in order:
        if len(pick) >= sample and tiles >= min_tiles:
            break
        pick.append(int(i))
        tiles += -(-instances[int(i)].n_cells // 32)
    return sorted(pick)


def tune_batch(instances, precision="mixed", sample=24, steps=2, warmup=1, seed=0,
               cache_path=DEFAULT_CACHE, candidates=BATCH_CANDIDATES, use_cache=True, verbose=False):
    """Pick (block_warps, ctas_per_sm, bins_per_grab) for a batch of these instances."""
    import torch

    from .batch import Batch
    key = batch_key(instances, precision)
    cache = _load(cache_path) if use_cache else {}
    if use_cache and key in cache:
        return dict(cache[key], cached=True)
    dev = torch.device("cuda", torch.cuda.current_device())
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    warps = min(MAX_WARPS_PER_SM, max(c * w for w, c, _ in candidates))
    pick = sample_instances(instances, sample, TILES_PER_RESIDENT_WARP * warps * n_sm, seed)
    insts = [instances[i] for i in pick]
    bins = sum(w.n_cells * w.n_bins for w in insts)
    b = Batch(max_slots=len(insts), precision=precision, capacity_bins=bins,
              max_bins=max(w.n_bins for w in insts))
    slots, keep = [], []
    for w in insts:
        s = b.admit(w.n_cells, w.n_bins, s_lognormal=w.s, R0ref=w.R0ref, span_K=w.span_K,
                    alpha0=w.alpha0, **{k: v for k, v in w.fluid.items()})
        p = w.pressure_step(0, xp=torch, device=dev)
        m = torch.empty((7, w.n_cells), dtype=torch.float64, device=dev)
        b.bind(s, p, w.dt, moments=m)
        slots.append(s)
        keep.append((p, m))
    b.step()  # first step: trial history for the queue order
    snap = [b.get_state(s) for s in slots]
    torch.cuda.synchronize()
    results = []
    for cand in candidates:
        b.set_launch(*cand)
        for s, st in zip(slots, snap):
            b.set_state(s, *st)
        for _ in range(warmup):
            b.step()
        for s, st in zip(slots, snap):
            b.set_state(s, *st)
        ms = _time_events(b.step, steps)
        results.append((ms, cand))
        if verbose:
            print("batch candidate", cand, f"{ms:.3f} ms")
    b.close()
    ms, best = min(results)
    worst = max(results)[0]
    out = dict(block_warps=best[0], ctas_per_sm=best[1], bins_per_grab=best[2], ms=ms,
               worst_ms=worst, sample_instances=len(insts), sample_bins=bins,
               candidates=len(candidates), when=time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime()))
    if use_cache:
        cache = _load(cache_path)
        cache[key] = out
        _save(cache_path, cache)
    return dict(out, cached=False)


def tune_solver(solver, pressures, dt, steps=2, candidates=SOLVER_CANDIDATES, verbose=False):
    """Pick warps per CTA for one Solver on its own state (restored after each candidate)."""
    import torch
    snap = solver.get_state()
    torch.cuda.synchronize()
    results = []
    for w in candidates:
        solver.set_block_warps(w)
        solver.set_state(*snap)
        solver.step(pressures[0], dt)  # warm
        solver.set_state(*snap)
        it = iter(range(steps))

        def one():
            k = next(it)
            solver.step(pressures[min(k, len(pressures) - 1)], dt)
        ms = _time_events(one, steps)
        results.append((ms, w))
        if verbose:
            print("solver candidate", w, f"{ms:.3f} ms")
    solver.set_state(*snap)
    solver.status()
    ms, best = min(results)
    solver.set_block_warps(best)
    return dict(block_warps=best, ms=ms, all={w: m for m, w in results})


def median_ms(times):
    return statistics.median(times) if times else float("nan")
