"""Throughput of the bubble source update on GB300: bin-steps/s.

One step = one flow step of the whole hot path over the workload: every
(cell, bin) advanced with adaptive SSP-RK3(2) sub-steps under its cell's
pressure, and the 7 quadrature moments of every cell written (one fused
kernel per step).  bin-steps = cells x bins x flow steps (sub-steps are not
counted).

Default workload: 128^3 cells x Nb = 31 lognormal bins (s = 0.5), water,
plane acoustic wave of 1.2 p0 at 100 kHz with 5 % seeded phase jitter,
dt = 5e-9 s, adaptive FP64 (tol 1e-4).  The state (1.3 GB) is larger than
L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload grid128|grid256_mixed|small] [--precision fp64|mixed]

Under torchrun every rank advances its own 128^3 block (weak scaling, no
data-path collective); rank 0 prints one JSON line.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2511_21031_gb300 import dist as pdist  # noqa: E402
from paper_2511_21031_gb300 import workloads  # noqa: E402

METRIC = "bin-steps/s (cells x bins x flow steps)"
NOMINAL_FP64_FLOPS_PER_CLK_PER_SM = 4.0   # nominal 1.25 TFLOP/s / (152 SMs x 2.07 GHz)
NOMINAL_FP32_FLOPS_PER_CLK_PER_SM = 256.0  # 128 FP32 lanes x 2 (FMA)
N_SM = 152
SM_MAX_MHZ = 2070.0
# FP64 flops (DFMA = 2, DADD/DMUL = 1) the FP64 step kernel's FP64 pipe executes per trial (one
# sub-step attempt: 3 Keller-Miksis right-hand sides, stage combination, error norm, controller)
# and per bin-step outside the trial loop (load, start of the step, the closing pass's bubble
# pressure and quadrature sums): least-squares fit of ncu's
# smsp__sass_thread_inst_executed_op_d{fma,add,mul}_pred_on over nine launches of the 64^3 x 31
# grid with traced trial counts (residual 1e-3).  These are the DP operations the FP64 roofline
# counts.  (The accept test's two FP64 products run only for errors within 2^-16 of tol; the
# FP32 estimate decides the rest.  The gas factor a flow step starts from comes from the
# previous step's moment pass.)
FP64_FLOPS_PER_TRIAL = 104.84
FP64_FLOPS_PER_BINSTEP = 8.50
# Operations of the trial that the integer pipe forms instead (pab_intmul.cuh), in the flops the
# FP64 instructions they replace would count: each right-hand side's two products (2) and its
# reciprocal's refinement (3 FMAs, 6), three right-hand sides a trial.  Reported beside the
# roofline (achieved_with_int_pipe), not in it.  (The first stage's k1 = h f products also run
# there; the first stage's FMAs form them a second time, so they were never counted.)
FP64_INT_PIPE_FLOPS_PER_TRIAL = 24.0
# and per bin-step the seven products of the closing pass's quadrature terms (w R^2, w R^3,
# w R^2 Rdot, w R^3 Rdot^2, the viscous and surface-tension term).
FP64_INT_PIPE_FLOPS_PER_BINSTEP = 7.0
# A trial with FP64 products and reciprocal, as the mixed kernels run their FP64 trials near
# collapse: the FP64-pipe fit of that build (130.84 per trial, less the two recomputed products).
FP64_PRODUCT_TRIAL_FLOPS = 128.84
# DRAM bytes per bin-step of the step kernel (ncu dram__bytes_{read,write}.sum on the
# 64^3 x 31 grid, 421.0 MB / 8.13M bin-steps, the carried gas factors included); scaled by
# bin-steps.
FP64_DRAM_BYTES_PER_BINSTEP = 51.8
FP64_PIPE_ACTIVE_NCU = 0.904
# The mixed step kernel on a 64^3 x 31 launch (ncu --set full, 4-warp CTAs): DRAM
# bytes per bin-step (part of the 162 MB state stays in L2; 42 B algorithmic) and
# the utilisations that bound it (issue slots first).
MIXED_DRAM_BYTES_PER_BINSTEP = 36.1
MIXED_ISSUE_ACTIVE_NCU = 0.759
MIXED_FP64_PIPE_ACTIVE_NCU = 0.575
MIXED_FMA_PIPE_ACTIVE_NCU = 0.340
# The batch kernel on 16 instances (ncu --set full, one-warp CTAs, 72 registers):
# DRAM bytes per bin-state and utilisations.
BATCH_DRAM_BYTES_PER_BINSTEP = 43.9
BATCH_ISSUE_ACTIVE_NCU = 0.872
BATCH_FP64_PIPE_ACTIVE_NCU = 0.538
BATCH_FMA_PIPE_ACTIVE_NCU = 0.474
BATCH_COUNTERS_BUILD = "current (72 registers)"
HBM_FALLBACK_GBS = 6800.0


def _hbm_peak():
    """(GB/s, source): the measured copy bandwidth of this machine's GPUs, else the fallback."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured copy bandwidth (MEASURED_PEAKS.json)"
    except (OSError, ValueError, KeyError):
        return HBM_FALLBACK_GBS, "fallback 6.8 TB/s (no measured peak available)"


def _dist():
    return pdist.env_rank()


def _mixed_roofline(bin_steps_per_s, batched=False):
    """A mixed kernel against its ceilings: HBM traffic at this rate against the measured
    copy bandwidth (live), and the issue and pipe utilisations of its ncu capture."""
    peak, src = _hbm_peak()
    if batched:
        per, iss, f64, fma, prof, build = (BATCH_DRAM_BYTES_PER_BINSTEP, BATCH_ISSUE_ACTIVE_NCU,
                                           BATCH_FP64_PIPE_ACTIVE_NCU, BATCH_FMA_PIPE_ACTIVE_NCU,
                                           "profiles/batch_kernel_mixed_16inst.md", BATCH_COUNTERS_BUILD)
    else:
        per, iss, f64, fma, prof, build = (MIXED_DRAM_BYTES_PER_BINSTEP, MIXED_ISSUE_ACTIVE_NCU,
                                           MIXED_FP64_PIPE_ACTIVE_NCU, MIXED_FMA_PIPE_ACTIVE_NCU,
                                           "profiles/step_kernel_mixed.md", "current")
    gbs = per * bin_steps_per_s / 1e9
    return {"bound": "issue", "achieved_hbm_gbs": gbs, "hbm_peak_gbs": peak, "hbm_frac": gbs / peak,
            "hbm_peak_source": src, "issue_active_ncu": iss, "fp64_pipe_active_ncu": f64,
            "fma_pipe_active_ncu": fma, "counters": prof, "counters_build": build}


# FP32 and FP64 flops (FFMA/DFMA = 2, FADD/FMUL/DADD/DMUL = 1) of the mixed step kernel per FP32
# trial, per FP64 (collapse) trial and per bin-step outside the trial loop: least-squares fit of
# ncu's smsp__sass_thread_inst_executed_op_{f,d}{fma,add,mul}_pred_on over traced launches
# (profiles/step_kernel_mixed.md).  None until that capture exists for the current build.
# An FP64 (collapse) trial is the trial with FP64 products: FP64_PRODUCT_TRIAL_FLOPS.
MIXED_FLOPS = {"fp32_per_trial": 342.36, "fp64_per_trial": 1.52, "fp64_per_fp64_trial": FP64_PRODUCT_TRIAL_FLOPS,
               "fp32_per_binstep": 68.17, "fp64_per_binstep": 11.63,
               "source": "profiles/step_kernel_mixed.md (fit over nine 64^3 launches)"}
# The batch kernel runs the same trial arithmetic; its 16-instance capture agrees with this fit to
# 3 % (FP32) and 11 % (FP64) (profiles/batch_kernel_mixed_16inst.md).
BATCH_FLOPS = dict(MIXED_FLOPS, source="profiles/step_kernel_mixed.md fit, checked against "
                                       "profiles/batch_kernel_mixed_16inst.md")


def _fp64_peak_derived():
    return NOMINAL_FP64_FLOPS_PER_CLK_PER_SM * N_SM * SM_MAX_MHZ * 1e6


def _fp32_peak_derived():
    return NOMINAL_FP32_FLOPS_PER_CLK_PER_SM * N_SM * SM_MAX_MHZ * 1e6


def _mixed_compute_roofline(bin_steps_per_s, trials_per_bin_step, fp64_fraction, batched=False):
    """A mixed kernel against both compute ceilings: its FP32 and FP64 flops per second (the
    ncu-fitted flops per trial and per bin-step applied to the counted trials) over the derived
    FP32 and FP64 peaks, beside the HBM and issue figures of _mixed_roofline."""
    roof = _mixed_roofline(bin_steps_per_s, batched=batched)
    fit = BATCH_FLOPS if batched else MIXED_FLOPS
    if not fit:
        roof.update({"fp32_tflops": None, "fp64_tflops": None, "fp32_frac": None, "fp64_frac": None})
        return roof
    t32 = trials_per_bin_step * (1.0 - fp64_fraction)
    t64 = trials_per_bin_step * fp64_fraction
    f32 = bin_steps_per_s * (t32 * fit["fp32_per_trial"] + fit["fp32_per_binstep"])
    f64 = bin_steps_per_s * (t32 * fit["fp64_per_trial"] + t64 * fit["fp64_per_fp64_trial"]
                             + fit["fp64_per_binstep"])
    roof.update({"fp32_tflops": f32 / 1e12, "fp64_tflops": f64 / 1e12,
                 "fp32_frac": f32 / _fp32_peak_derived(), "fp64_frac": f64 / _fp64_peak_derived(),
                 "flops_fit": fit.get("source")})
    return roof


def make_workload(name, rank, edge=0):
    if name == "grid128":
        return workloads.config_grid128(seed=pdist.rank_seed(2, rank), edge=edge or 128)
    if name == "grid256_mixed":
        return workloads.config_grid256_mixed(seed=pdist.rank_seed(3, rank))
    if name == "small":
        return workloads.config_small(seed=pdist.rank_seed(1, rank))
    raise SystemExit(f"unknown workload {name}")


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region.

    nvidia-smi numbers the GPUs in its own (PCI) order and ignores CUDA_VISIBLE_DEVICES, so a
    torch device index may name another GPU there: every GPU is sampled with its index and
    UUID, and the samples of the one whose UUID is the torch device's are kept (those with the
    torch index when the UUID is not known)."""

    FIELDS = ("index,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index, uuid=None):
        self.index = index
        self.uuid = uuid
        self.proc = None
        self.lines = []

    @staticmethod
    def device_uuid(index):
        """The torch device's UUID, or None where this torch does not report it."""
        try:
            import torch
            u = str(torch.cuda.get_device_properties(index).uuid).strip()
            return u or None
        except Exception:
            return None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        return self.summarise(self.lines, self.index, self.uuid)

    @staticmethod
    def summarise(lines, index, uuid=None):
        """Median SM clock, maximum clock and the throttle reasons seen active in the samples
        of the GPU with this UUID (else this nvidia-smi index)."""
        def norm(u):
            u = u.strip().lower()
            return u[4:] if u.startswith("gpu-") else u
        rows = [[p.strip() for p in ln.split(",")] for ln in lines]
        rows = [r for r in rows if len(r) >= 10]
        mine = [r for r in rows if uuid and norm(r[1]) == norm(uuid)]
        matched = "uuid"
        if not mine:
            mine = [r for r in rows if r[0] == str(index)]
            matched = "index"
        sm, mx, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in mine:
            try:
                clk, top = float(r[2]), float(r[3])
            except ValueError:
                continue
            sm.append(clk)
            mx = top
            for n, v in zip(names, r[6:10]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm), "gpu": mine[0][1] if matched == "uuid" else f"index {index}",
                "matched_by": matched}


def cpu_baseline(wl, seconds=12.0, sample_cells=16384):
    """The oracle as it stands on the host cores, on a seeded sample of the workload's cells."""
    import oracle
    cells = np.sort(np.random.default_rng(11).choice(wl.n_cells, min(sample_cells, wl.n_cells),
                                                      replace=False))
    sub = wl.subset(cells)
    P = oracle.Params(**sub.fluid)
    R0, _ = oracle.bins(sub.n_bins, sub.R0ref, sub.s, sub.span_K)
    R = np.repeat(R0[:, None], sub.n_cells, axis=1).copy()
    V = np.zeros_like(R)
    h = np.zeros(R.shape, dtype=np.float32)
    steps = 0
    t0 = time.perf_counter()
    while True:
        oracle.step(P, R0, sub.pressure_step(steps), sub.dt, R, V, h)
        steps += 1
        if time.perf_counter() - t0 >= seconds or steps >= wl.n_steps:
            break
    el = time.perf_counter() - t0
    cores = oracle.max_threads()
    return {"value": sub.n_cells * sub.n_bins * steps / el, "unit": "bin-steps/s", "cores": cores,
            "kind": "oracle",
            "sample": f"{sub.n_cells} seeded cells x {sub.n_bins} bins x {steps} flow steps of {wl.name}"}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    wl = make_workload(args.workload, 0)
    import oracle
    cells = np.sort(np.random.default_rng(11).choice(wl.n_cells, min(16384, wl.n_cells), replace=False))
    sub = wl.subset(cells)
    P = oracle.Params(**sub.fluid)
    R0, _ = oracle.bins(sub.n_bins, sub.R0ref, sub.s, sub.span_K)
    R = np.repeat(R0[:, None], sub.n_cells, axis=1).copy()
    V = np.zeros_like(R)
    h = np.zeros(R.shape, dtype=np.float32)
    for n in range(args.warmup):
        oracle.step(P, R0, sub.pressure_step(n), sub.dt, R, V, h)
    t0 = time.perf_counter()
    for n in range(args.warmup, args.warmup + args.steps):
        oracle.step(P, R0, sub.pressure_step(n), sub.dt, R, V, h)
    el = time.perf_counter() - t0
    value = sub.n_cells * sub.n_bins * args.steps / el
    cores = oracle.max_threads()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "bin-steps/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": el * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl.name, "cells": wl.n_cells, "bins": wl.n_bins, "dt": wl.dt,
                       "sample_cells": sub.n_cells},
            "cpu_baseline": {"value": value, "unit": "bin-steps/s", "cores": cores, "kind": "oracle",
                             "sample": f"{sub.n_cells} seeded cells x {sub.n_bins} bins per step"},
            "e2e": {"value": value, "unit": "bin-steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _time_steps(solver, wl, ps, args, stream, clocks=None, keep_start=False):
    """Warm up, then time args.steps flow steps (one fused launch each) with CUDA events.
    keep_start: also return the state the timed steps started from."""
    import torch

    from paper_2511_21031_gb300 import pab
    ws, _, _ = _dist()
    mom = torch.empty((pab.N_MOMENTS, wl.n_cells), dtype=torch.float64, device=ps[0].device)
    if getattr(args, "trace_trials", False):
        # profiling aid: trials of every launch (a sync after each; not a timing run)
        trace = []
        with torch.cuda.stream(stream):
            for n in range(args.warmup + args.steps):
                solver.step(ps[n], wl.dt, moments=mom)
                trace.append(solver.status(stream=stream)["n_attempts"])
        return dict(trace=trace)
    with torch.cuda.stream(stream):
        for n in range(args.warmup):
            solver.step(ps[n], wl.dt, moments=mom)
    solver.status(stream=stream)
    start = solver.get_state(stream=stream) if keep_start else None
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
        time.sleep(0.3)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        t_start.record(stream)
        for k in range(args.steps):
            ev[k][0].record(stream)
            solver.step(ps[args.warmup + k], wl.dt, moments=mom)
            ev[k][1].record(stream)
        t_end.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clk = clocks.stop() if clocks else None
    ms_total = t_start.elapsed_time(t_end)
    launch_ms = [a.elapsed_time(b) for a, b in ev]
    st = solver.status(stream=stream)
    ms_total = pdist.max_over_ranks(ms_total, device=ps[0].device)
    return dict(ms_total=ms_total, launch_ms=launch_ms, status=st, clocks=clk, moments=mom, start=start)


def _mixed_error_sample(wl, n_steps, n_cells=256):
    """Error of the mixed path against the FP64 oracle on a seeded sample of cells: the mixed
    library path and the oracle run on exactly those cells from the same start and host-made
    pressures (outside any timed region; cells are independent, so the sample is the full
    computation for them).  The FP64 kernel's own error on the same sample is reported beside it."""
    import torch

    import oracle
    from paper_2511_21031_gb300 import pab
    cells = np.sort(np.random.default_rng(12).choice(wl.n_cells, min(n_cells, wl.n_cells), replace=False))
    sub = wl.subset(cells)
    kw = dict(s_lognormal=sub.s, R0ref=sub.R0ref, span_K=sub.span_K, alpha0=sub.alpha0)
    sm = pab.Solver(sub.n_cells, sub.n_bins, precision="mixed", **kw)
    sd = pab.Solver(sub.n_cells, sub.n_bins, precision="fp64", **kw)
    mm = torch.empty((pab.N_MOMENTS, sub.n_cells), dtype=torch.float64, device="cuda")
    md = torch.empty_like(mm)
    P = oracle.Params(**sub.fluid)
    R0o, wo = oracle.bins(sub.n_bins, sub.R0ref, sub.s, sub.span_K)
    Ro = np.repeat(R0o[:, None], sub.n_cells, axis=1).copy()
    Vo = np.zeros_like(Ro)
    ho = np.zeros(Ro.shape, dtype=np.float32)
    for n in range(n_steps):
        ph = sub.pressure_step(n)
        p = torch.as_tensor(ph, device="cuda")
        sm.step(p, sub.dt, moments=mm)
        sd.step(p, sub.dt, moments=md)
        oracle.step(P, R0o, ph, sub.dt, Ro, Vo, ho)
    om = oracle.moments(P, R0o, wo, np.full(sub.n_cells, oracle.equilibrium_nb(sub.alpha0, R0o, wo)), Ro, Vo)
    Rm, Vm, _ = sm.get_state()
    Rd, Vd, _ = sd.get_state()
    g, d = mm.cpu().numpy(), md.cpu().numpy()
    Rm, Vm, Rd, Vd = Rm.cpu().numpy(), Vm.cpu().numpy(), Rd.cpu().numpy(), Vd.cpu().numpy()
    v_floor = 1e-3 * math.sqrt(sub.fluid["p0"] / sub.fluid["rho"])
    out = _mixed_errors(g, om, Rm, Vm, Ro, Vo, wo, v_floor)
    out["fp64_kernel"] = {k: v for k, v in _mixed_errors(d, om, Rd, Vd, Ro, Vo, wo, v_floor).items()
                          if k in ("R", "alpha", "R2Rdot")}
    out["sample"] = f"{sub.n_cells} seeded cells x {sub.n_bins} bins x {n_steps} steps, against the oracle"
    sm.close()
    sd.close()
    return out


def _mixed_errors(g, o, Rm, Vm, Rd, Vd, w, v_floor):
    """Error of every mixed output against the FP64 one: R and the positive moments relative,
    Rdot against max(|Rdot|, v_floor), the signed sums (<R^2 Rdot>, S_alpha) against the sum of
    their absolute terms plus the floor, and <R^3 Rdot^2>/<R^3> against max(|value|, v_floor^2)."""
    w = np.asarray(w)[:, None]
    scale = np.sum(w * Rd * Rd * (np.abs(Vd) + v_floor), axis=0)

    def rel(a, b):
        return float(np.max(np.abs(a - b) / np.abs(b)))
    return {"R": rel(Rm, Rd),
            "Rdot": float(np.max(np.abs(Vm - Vd) / np.maximum(np.abs(Vd), v_floor))),
            "alpha": rel(g[1], o[1]), "R3": rel(g[2], o[2]),
            "R2Rdot": float(np.max(np.abs(g[3] - o[3]) / scale)),
            "S_alpha": float(np.max(np.abs(g[4] - o[4]) / (3.0 * o[1] * scale / o[2]))),
            "R3pbw_over_R3": rel(g[5], o[5]),
            "R3Rdot2_over_R3": float(np.max(np.abs(g[6] - o[6]) / np.maximum(np.abs(o[6]), v_floor ** 2)))}


TRANSFER_PV = 2338.0  # saturated vapour pressure of water at 20 C


def _bench_transfer(args, stream, dev, fp64_value):
    """The 128^3 x 31 FP64 workload with the contents of pab_transfer.h (gas and
    vapour with heat and mass transfer at the wall, p_v of water at 20 C). Its
    parity with the oracle is tests/test_gpu_transfer.py."""
    import torch

    from paper_2511_21031_gb300 import pab
    wl = make_workload("grid128", 0, args.edge)
    total = args.warmup + args.steps
    sol = pab.Solver(wl.n_cells, wl.n_bins, s_lognormal=wl.s, R0ref=wl.R0ref, span_K=wl.span_K,
                     alpha0=wl.alpha0, gas_mode=pab.PAB_GAS_TRANSFER, pv=TRANSFER_PV)
    with torch.cuda.stream(stream):
        ps = [wl.pressure_step(n, xp=torch, device=dev) for n in range(total)]
    torch.cuda.synchronize()
    r = _time_steps(sol, wl, ps, args, stream)
    sol.close()
    del ps
    torch.cuda.synchronize()
    bs = wl.n_cells * wl.n_bins * args.steps
    return {"workload": wl.name.replace("fp64", "transfer"),
            "label": "contents with heat and mass transfer (FP64)", "precision": "fp64",
            "value": bs / (r["ms_total"] * 1e-3), "unit": "bin-steps/s",
            "ms_per_step": r["ms_total"] / args.steps,
            "latency_ms": {"p50": float(np.percentile(r["launch_ms"], 50)),
                           "p99": float(np.percentile(r["launch_ms"], 99))},
            "trials_per_bin_step": r["status"]["n_attempts"] / bs, "status_flags": r["status"]["flags"],
            "vs_polytropic_fp64": (bs / (r["ms_total"] * 1e-3)) / fp64_value,
            "parity": "tests/test_gpu_transfer.py (against the oracle)"}


def _bench_batched(args, stream, dev, n_instances=512, insts=None, name=None):
    """512 independent instances (edge U{16..96}, Nb in {11,21,31,51}, amplitude
    U(0.3,1.5) p0, s U(0.2,0.7)) in one persistent mixed-precision launch per
    step, replayed from a CUDA graph, launch shape from the autotuner.  Given
    `insts` (instances sharing one forcing frequency and step), those instead."""
    import torch

    from paper_2511_21031_gb300 import autotune
    from paper_2511_21031_gb300.batch import Batch
    if insts is None:
        insts = workloads.batched_instances(n=n_instances)
    if getattr(args, "batch_launch", None):
        # profiling aid: a fixed launch shape instead of the autotuner's
        w_, c_, g_ = args.batch_launch
        tune = {"block_warps": w_, "ctas_per_sm": c_, "bins_per_grab": g_, "cached": False,
                "candidates": 0, "fixed": True}
    else:
        tune = autotune.tune_batch(insts, precision="mixed")
    bins = sum(w.n_cells * w.n_bins for w in insts)
    cells = sum(w.n_cells for w in insts)
    b = Batch(max_slots=len(insts), precision="mixed", capacity_bins=bins, max_bins=51)
    b.set_launch(tune["block_warps"], tune["ctas_per_sm"], tune["bins_per_grab"])
    total = args.warmup + args.steps
    # one pressure field per step for all instances, generated on the device (outside timing)
    theta = torch.empty(cells, dtype=torch.float64, device=dev)
    amp = torch.empty(cells, dtype=torch.float64, device=dev)
    offs, o = [], 0
    for w in insts:
        theta[o:o + w.n_cells] = torch.as_tensor(w.theta, device=dev)
        amp[o:o + w.n_cells] = w.amp
        offs.append(o)
        o += w.n_cells
    p0 = insts[0].fluid["p0"]
    om = 2.0 * math.pi * insts[0].freq
    ps = [p0 + p0 * amp * torch.sin(theta + om * (n + 0.5) * insts[0].dt) for n in range(total)]
    del theta, amp
    mom = torch.empty(7 * cells, dtype=torch.float64, device=dev)
    slots = []
    for w, off in zip(insts, offs):
        s_ = b.admit(w.n_cells, w.n_bins, s_lognormal=w.s, R0ref=w.R0ref, span_K=w.span_K,
                     alpha0=w.alpha0, **w.fluid)
        slots.append((s_, w, off))

    def bind(n):
        for s_, w, off in slots:
            b.bind(s_, ps[n][off:off + w.n_cells], w.dt,
                   moments=mom[7 * off:7 * (off + w.n_cells)].view(7, w.n_cells))
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        for n in range(args.warmup):
            bind(n)
            b.step(graph=True, stream=stream)
    torch.cuda.synchronize()
    attempts0 = sum(b.status(s_, stream=stream)["n_attempts"] for s_, _, _ in slots)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            bind(args.warmup + k)   # host-side pointer update only
            ev[k][0].record(stream)
            b.step(graph=True, stream=stream)
            ev[k][1].record(stream)
    torch.cuda.synchronize()
    ms = [a.elapsed_time(c) for a, c in ev]
    st = [b.status(s_, stream=stream) for s_, _, _ in slots]
    n_att = sum(x["n_attempts"] for x in st)
    n64 = sum(x["n_fp64"] for x in st)
    flags = 0
    for x in st:
        flags |= x["flags"]
    b.close()
    del ps, mom
    torch.cuda.synchronize()
    return {"workload": name or f"batched {len(insts)} instances", "label": "batched mixed (graph)",
            "precision": "mixed", "instances": len(insts), "cells": cells, "bins": bins,
            "value": bins * args.steps / (sum(ms) * 1e-3), "unit": "bin-steps/s",
            "ms_per_step": sum(ms) / args.steps,
            "latency_ms": {"p50": float(np.percentile(ms, 50)), "p99": float(np.percentile(ms, 99))},
            "trials_per_bin_step": n_att / (bins * args.steps),
            "fp64_trial_fraction": n64 / max(1, n_att), "status_flags": flags,
            "launch": {"block_warps": tune["block_warps"], "ctas_per_sm": tune["ctas_per_sm"],
                       "bins_per_grab": tune["bins_per_grab"], "autotuned": True,
                       "cached": tune.get("cached", False), "candidates": tune.get("candidates"),
                       "sample_best_ms": tune.get("ms"), "sample_worst_ms": tune.get("worst_ms")},
            "warmup_attempts": attempts0}


def _bench_serving(args, n_requests=16, rate=200.0):
    """The first n_requests of the seeded Poisson stream (200 req/s; edge lognormal
    median 78.4 clipped to [32, 192]; Nb in {21, 31}; 200 flow steps each, mixed),
    served by continuous batching on the wall clock."""
    from paper_2511_21031_gb300 import autotune
    from paper_2511_21031_gb300.serve import ServingEngine
    reqs = workloads.request_stream(n=n_requests, rate=rate)
    tune = autotune.tune_batch([r.work for r in reqs], precision="mixed", sample=8)
    eng = ServingEngine(capacity_bins=2_000_000_000, max_slots=256,
                        launch=(tune["block_warps"], tune["ctas_per_sm"], tune["bins_per_grab"]))
    rep = eng.run(reqs, clock="wall")
    eng.close()
    offered = rate * float(np.mean([r.work.bins_total * r.work.n_steps for r in reqs]))
    return {"workload": f"serving {n_requests} requests at {rate:g} req/s", "label": "serving mixed",
            "precision": "mixed", "requests": n_requests,
            "value": rep["throughput_bin_steps_per_s"], "unit": "bin-steps/s",
            "gpu_value": rep["gpu_throughput_bin_steps_per_s"],
            "latency_s": rep["latency_s"], "concurrency": rep["concurrency"],
            "iterations": rep["iterations"], "elapsed_s": rep["elapsed_s"],
            "offered_bin_steps_per_s": offered, "status_flags": rep["flags"],
            "launch": {"block_warps": tune["block_warps"], "ctas_per_sm": tune["ctas_per_sm"],
                       "bins_per_grab": tune["bins_per_grab"], "autotuned": True}}


def _bench_serving_sweep(args, rates, n_requests):
    """The seeded Poisson request stream at several offered rates (n_requests each), served on the
    wall clock: per rate the p50/p99 latency, the throughput, the GPU's busy share and the mean
    concurrency, to place the knee between idle and saturated serving."""
    from paper_2511_21031_gb300 import autotune
    from paper_2511_21031_gb300.serve import ServingEngine
    out = []
    tune = None
    for rate in rates:
        reqs = workloads.request_stream(n=n_requests, rate=rate)
        if tune is None:
            tune = autotune.tune_batch([r.work for r in reqs], precision="mixed", sample=8)
        eng = ServingEngine(capacity_bins=2_000_000_000, max_slots=256,
                            launch=(tune["block_warps"], tune["ctas_per_sm"], tune["bins_per_grab"]))
        rep = eng.run(reqs, clock="wall")
        eng.close()
        out.append({"rate": rate, "requests": n_requests, "completed": rep["completed"],
                    "latency_s": rep["latency_s"], "throughput": rep["throughput_bin_steps_per_s"],
                    "gpu_busy": rep["gpu_busy_s"] / rep["elapsed_s"], "concurrency": rep["concurrency"],
                    "elapsed_s": rep["elapsed_s"], "flags": rep["flags"]})
    return {"workload": f"serving sweep, {n_requests} requests per rate", "label": "serving sweep mixed",
            "precision": "mixed", "unit": "bin-steps/s", "rates": out,
            "launch": {"block_warps": tune["block_warps"], "ctas_per_sm": tune["ctas_per_sm"],
                       "bins_per_grab": tune["bins_per_grab"], "autotuned": True}}


def _bench_latency_small(args, stream, dev, block_warps=0):
    """The 64-cell x Nb 21 workload (0.5 p0 at 100 kHz, 1000 flow steps of 1e-8 s, adaptive FP64)
    call by call: the latency the host sees per call through pab_bubble_step (device buffers; the
    call and a wait on its stream) and through pab_bubble_step_host (host buffers; the call copies
    the pressure in and the moments out and waits), each over the whole 1000-step run from
    equilibrium, with the kernel's own duration from CUDA events beside them."""
    import torch

    from paper_2511_21031_gb300 import pab
    wl = workloads.config_small()
    out = {"workload": wl.name, "label": "per-call latency, 64 cells x Nb 21 (FP64)", "precision": "fp64",
           "unit": "bin-steps/s", "steps": wl.n_steps}
    ph = [torch.as_tensor(wl.pressure_step(n)).pin_memory() for n in range(wl.n_steps)]
    pd = [x.to(dev) for x in ph]
    mh = torch.empty((pab.N_MOMENTS, wl.n_cells), dtype=torch.float64).pin_memory()
    md = torch.empty((pab.N_MOMENTS, wl.n_cells), dtype=torch.float64, device=dev)
    for api in ("pab_bubble_step", "pab_bubble_step_host"):
        sol = pab.Solver(wl.n_cells, wl.n_bins, s_lognormal=wl.s, R0ref=wl.R0ref, span_K=wl.span_K,
                         alpha0=wl.alpha0)
        if block_warps:
            sol.set_block_warps(block_warps)
        # a few calls to load the kernels and warm the driver, then a fresh state
        start = sol.get_state(stream=stream)
        for n in range(5):
            sol.step(pd[n], wl.dt, moments=md, stream=stream)
        sol.set_state(*start, stream=stream)
        torch.cuda.synchronize()
        host_ms, kern_ms = [], []
        evs = []
        for n in range(wl.n_steps):
            t0 = time.perf_counter()
            if api == "pab_bubble_step":
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                sol.step(pd[n], wl.dt, moments=md, stream=stream)
                e1.record(stream)
                stream.synchronize()
                evs.append((e0, e1))
            else:
                sol.step_host(ph[n], wl.dt, moments_host=mh, stream=stream)
            host_ms.append((time.perf_counter() - t0) * 1e3)
        kern_ms = [a.elapsed_time(b) for a, b in evs]
        st = sol.status(stream=stream)
        sol.close()
        bs = wl.n_cells * wl.n_bins * wl.n_steps
        out[api] = {"p50_ms": float(np.percentile(host_ms, 50)), "p99_ms": float(np.percentile(host_ms, 99)),
                    "mean_ms": float(np.mean(host_ms)), "value": bs / (sum(host_ms) * 1e-3),
                    "trials_per_bin_step": st["n_attempts"] / bs, "status_flags": st["flags"]}
        if kern_ms:
            out[api]["kernel_p50_ms"] = float(np.percentile(kern_ms, 50))
            out[api]["kernel_p99_ms"] = float(np.percentile(kern_ms, 99))
    out["value"] = out["pab_bubble_step"]["value"]
    out["block_warps"] = block_warps or "default"
    return out


def _bench_collapse(args, stream, dev, precision, sample_cells=64):
    """The collapse-stress workload (64^3 cells x Nb 31, s = 0.5; plane wave of 1.2 p0 at 21.4 kHz
    with 5 % seeded phase jitter; 5e-9 s flow steps) over one forcing period (10,000 steps) from
    equilibrium: every cell is driven into tension, grows and collapses once, so the window holds
    the regime of the paper's Ohl-type case (Sec. 5).  Every step launch is timed with CUDA events
    on its stream; the pressure fields are made on the device between chunks of steps, outside the
    events.  The errors of every output against the FP64 oracle come from seeded sample cells run
    through the oracle after the timed steps, on the pressures the GPU used."""
    import torch

    from paper_2511_21031_gb300 import pab
    wl = workloads.config_collapse(edge=args.collapse_edge, n_steps=args.collapse_steps)
    C, B = wl.n_cells, wl.n_bins
    cells = np.sort(np.random.default_rng(13).choice(C, min(sample_cells, C), replace=False))
    cells_d = torch.as_tensor(cells, device=dev)
    sol = pab.Solver(C, B, precision=precision, s_lognormal=wl.s, R0ref=wl.R0ref, span_K=wl.span_K,
                     alpha0=wl.alpha0)
    first = 0
    if getattr(args, "collapse_load", None):
        # profiling aid: continue from a state saved by --collapse-save (no oracle comparison)
        ck = torch.load(args.collapse_load)
        first = int(ck["steps"])
        sol.set_state(ck["R"].to(dev), ck["V"].to(dev), ck["h"].to(dev), stream=stream)
    mom = torch.empty((pab.N_MOMENTS, C), dtype=torch.float64, device=dev)
    p_sample = []
    launch_ms = []
    n_att = n64 = 0
    flags = 0
    chunk = max(8, min(250, int(2e9 // (8 * C))))   # about 2 GB of pressure fields at a time
    torch.cuda.synchronize()
    for c0 in range(first, first + wl.n_steps, chunk):
        n1 = min(first + wl.n_steps, c0 + chunk)
        with torch.cuda.stream(stream):
            ps = [wl.pressure_step(n, xp=torch, device=dev) for n in range(c0, n1)]
            p_sample.append(torch.stack([p.index_select(0, cells_d) for p in ps]).cpu())
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in ps]
        with torch.cuda.stream(stream):
            for p, (e0, e1) in zip(ps, evs):
                e0.record(stream)
                sol.step(p, wl.dt, moments=mom, stream=stream)
                e1.record(stream)
        st = sol.status(stream=stream)
        torch.cuda.synchronize()
        launch_ms += [a.elapsed_time(b) for a, b in evs]
        n_att += st["n_attempts"]
        n64 += st["n_fp64"]
        flags |= st["flags"]
        del ps
    R, V, hh = sol.get_state(stream=stream)
    torch.cuda.synchronize()
    if getattr(args, "collapse_save", None):
        torch.save({"R": R.cpu(), "V": V.cpu(), "h": hh.cpu(), "steps": first + wl.n_steps},
                   args.collapse_save)
    del hh
    gR = R[:, cells_d].cpu().numpy()
    gV = V[:, cells_d].cpu().numpy()
    gm = mom[:, cells_d].cpu().numpy()
    w = np.array(sol.w)
    sol.close()
    del R, V, mom
    torch.cuda.synchronize()
    bs = C * B * wl.n_steps
    total_ms = float(sum(launch_ms))
    out = {"workload": wl.name + ("_mixed" if precision == "mixed" else "_fp64"),
           "label": f"collapse stress, one period ({precision})", "precision": precision,
           "cells": C, "bins": B, "steps": wl.n_steps, "value": bs / (total_ms * 1e-3),
           "unit": "bin-steps/s", "ms_per_step": total_ms / wl.n_steps,
           "latency_ms": {"p50": float(np.percentile(launch_ms, 50)),
                          "p99": float(np.percentile(launch_ms, 99))},
           "trials_per_bin_step": n_att / bs, "fp64_trial_fraction": n64 / max(1, n_att),
           "status_flags": flags}
    if precision == "fp64":
        flops = bs * (out["trials_per_bin_step"] * FP64_FLOPS_PER_TRIAL + FP64_FLOPS_PER_BINSTEP)
        with_int = flops + bs * (out["trials_per_bin_step"] * FP64_INT_PIPE_FLOPS_PER_TRIAL
                                 + FP64_INT_PIPE_FLOPS_PER_BINSTEP)
        out["roofline"] = {"bound": "alu", "pipe": "fp64", "achieved": flops / (total_ms * 1e-3) / 1e12,
                           "peak": _fp64_peak_derived() / 1e12, "unit": "TFLOP/s",
                           "frac": flops / (total_ms * 1e-3) / _fp64_peak_derived(),
                           "achieved_with_int_pipe": with_int / (total_ms * 1e-3) / 1e12,
                           "int_pipe_flops_per_trial": FP64_INT_PIPE_FLOPS_PER_TRIAL,
                           "int_pipe_flops_per_binstep": FP64_INT_PIPE_FLOPS_PER_BINSTEP}
    else:
        out["roofline"] = _mixed_compute_roofline(out["value"], out["trials_per_bin_step"],
                                                  out["fp64_trial_fraction"])
    # the oracle on the sample cells, from equilibrium on the same pressures (outside any timing)
    try:
        if first:
            raise RuntimeError("continued from a saved state: no oracle comparison")
        import oracle
        sub = wl.subset(cells)
        P = oracle.Params(**sub.fluid)
        R0o, wo = oracle.bins(B, sub.R0ref, sub.s, sub.span_K)
        Ro = np.repeat(R0o[:, None], len(cells), axis=1).copy()
        Vo = np.zeros_like(Ro)
        ho = np.zeros(Ro.shape, dtype=np.float32)
        pall = torch.cat(p_sample).numpy()
        for n in range(wl.n_steps):
            oracle.step(P, R0o, np.ascontiguousarray(pall[n]), wl.dt, Ro, Vo, ho)
        nb = np.full(len(cells), oracle.equilibrium_nb(sub.alpha0, R0o, wo))
        om = oracle.moments(P, R0o, wo, nb, Ro, Vo)
        v_floor = 1e-3 * math.sqrt(sub.fluid["p0"] / sub.fluid["rho"])
        err = _mixed_errors(gm, om, gR, gV, Ro, Vo, wo, v_floor)
        err["sample"] = f"{len(cells)} seeded cells x {B} bins x {wl.n_steps} steps"
        err["min_R_over_R0"] = float(np.min(Ro / R0o[:, None]))
        out["error_vs_oracle"] = err
    except Exception as e:   # the line stands without its error sample
        out["error_vs_oracle"] = {"error": repr(e)[:200]}
    return out


# FP64-pipe instructions of the carrier-coupling kernels by their source, per cell and per
# (bin, cell): GB300 retires 2 per clock and SM.  set_conservative forms its products (the cube
# of each summed value and the rescale of each value) on the integer pipe, leaving an FMA per
# summed value and a reciprocal and an inverse square root per cell; with the five products in
# FP64 the pipe, not HBM, bounded it (0.43 of HBM).
CLOSURE_FP64_INSTR = {
    "mixture_pressure": (4.0, 0.0),
    "get_conservative": (0.0, 2.0),
    "set_conservative": (13.0, 1.0),
}
FP64_PIPE_INSTR_PER_CLK_PER_SM = 2.0
# Algorithmic HBM bytes of the carrier-coupling kernels (FP64): per cell and per (bin, cell).
CLOSURE_BYTES = {
    # alpha, <R^3 p_bw>/<R^3>, <R^3 Rdot^2>/<R^3> and p_l in, p out
    "mixture_pressure": (40.0, 0.0),
    # R and Rdot in, n_b R and n_b Rdot out (default n_b)
    "get_conservative": (0.0, 32.0),
    # alpha in and n_b out per cell; n_b R and n_b Rdot in, R and Rdot out per bin-cell
    "set_conservative": (16.0, 32.0),
}


def _bench_closure(args, stream, dev):
    """One Strang-split flow step of the carrier coupling (pab_closure.h) on the 128^3 x 31 FP64
    workload: the bubble half step at the flow step's start pressure, the mixture pressure from its
    moments (the carrier pressure standing in for the liquid pressure), the conservative variables
    out and back (the carrier transports n_b R_i and n_b Rdot_i, n_b recovered from alpha), and the
    second half step at the end pressure.  Each kernel group is timed with CUDA events."""
    import torch

    from paper_2511_21031_gb300 import pab
    wl = make_workload("grid128", 0, args.edge)
    C, B = wl.n_cells, wl.n_bins
    total = args.warmup + args.steps
    sol = pab.Solver(C, B, s_lognormal=wl.s, R0ref=wl.R0ref, span_K=wl.span_K, alpha0=wl.alpha0)
    with torch.cuda.stream(stream):
        ps = [wl.pressure_at(n * wl.dt, xp=torch, device=dev) for n in range(total + 1)]
        mom = torch.empty((pab.N_MOMENTS, C), dtype=torch.float64, device=dev)
        pmix = torch.empty(C, dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    names = ("half_1", "mixture_pressure", "get_conservative", "set_conservative", "half_2")

    def flow_step(n):
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(len(names) + 1)]
        with torch.cuda.stream(stream):
            evs[0].record(stream)
            sol.strang_half(ps[n], wl.dt, moments=mom, stream=stream)
            evs[1].record(stream)
            sol.mixture_pressure(mom, ps[n], out=pmix, stream=stream)
            evs[2].record(stream)
            qR, qV = sol.get_conservative(stream=stream)
            evs[3].record(stream)
            sol.set_conservative(mom[1], qR, qV, stream=stream)
            evs[4].record(stream)
            sol.strang_half(ps[n + 1], wl.dt, moments=mom, stream=stream)
            evs[5].record(stream)
        # qR and qV were allocated on `stream`: the caching allocator reuses their blocks only
        # for later work on that stream, ordered after this step
        return evs

    for n in range(args.warmup):
        flow_step(n)
    sol.status(stream=stream)
    torch.cuda.synchronize()
    timed = [flow_step(args.warmup + k) for k in range(args.steps)]
    torch.cuda.synchronize()
    ms = {k: 0.0 for k in names}
    for evs in timed:
        for i, k in enumerate(names):
            ms[k] += evs[i].elapsed_time(evs[i + 1])
    st = sol.status(stream=stream)
    sol.close()
    del ps, timed
    peak, src = _hbm_peak()
    kernels = {}
    pipe = FP64_PIPE_INSTR_PER_CLK_PER_SM * N_SM * SM_MAX_MHZ * 1e6
    for k, (per_cell, per_bin_cell) in CLOSURE_BYTES.items():
        per_step_ms = ms[k] / args.steps
        gbs = (per_cell * C + per_bin_cell * C * B) / (per_step_ms * 1e-3) / 1e9
        ic, ib = CLOSURE_FP64_INSTR[k]
        ips = (ic * C + ib * C * B) / (per_step_ms * 1e-3)
        kernels[k] = {"ms_per_step": per_step_ms, "algorithmic_gbs": gbs, "hbm_frac": gbs / peak,
                      "fp64_pipe_frac": ips / pipe,
                      "bound": "fp64" if ips / pipe > gbs / peak else "hbm"}
    total_ms = sum(ms.values())
    bs = C * B * args.steps
    return {"workload": wl.name.replace("fp64", "strang"), "label": "Strang-split flow step with the closure (FP64)",
            "precision": "fp64", "value": bs / (total_ms * 1e-3), "unit": "bin-steps/s",
            "ms_per_step": total_ms / args.steps,
            "half_steps_ms_per_step": (ms["half_1"] + ms["half_2"]) / args.steps,
            "closure_kernels": kernels, "hbm_peak_gbs": peak, "hbm_peak_source": src,
            "trials_per_bin_step": st["n_attempts"] / bs, "status_flags": st["flags"],
            "parity": "tests/test_gpu_closure.py (against the oracle)"}


def _bench_el(args, stream, dev):
    """Volume-averaged (EL) model: fixed bubbles (R0 = 10 um, alpha0 = 1e-3) in a
    128^3 grid of 75 um cells, each advanced under its cell's pressure (0.5 p0 at
    100 kHz, random phase per cell) and smeared into alpha and alpha_dot with the
    truncated Gaussian kernel, every step."""
    import torch

    from paper_2511_21031_gb300.el import BubbleCloud
    wl = workloads.bubble_cloud(edge=128, dx=75e-6, alpha0=1e-3)
    cl = BubbleCloud(wl.pos, wl.R0, wl.edge, wl.edge, wl.edge, wl.dx, **wl.fluid)
    total = args.warmup + args.steps
    ps = [wl.pressure_step(n, xp=torch, device=dev) for n in range(total)]
    a = torch.empty(wl.edge ** 3, dtype=torch.float64, device=dev)
    ad = torch.empty_like(a)
    with torch.cuda.stream(stream):
        for n in range(args.warmup):
            cl.step(ps[n], wl.dt, alpha=a, alpha_dot=ad, stream=stream)
    cl.status(stream=stream)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    s0 = torch.cuda.Event(enable_timing=True)
    s1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        e0.record(stream)
        for k in range(args.steps):
            cl.step(ps[args.warmup + k], wl.dt, alpha=a, alpha_dot=ad, stream=stream)
        e1.record(stream)
        s0.record(stream)
        for k in range(args.steps):
            cl.smear(a, ad, stream=stream)
        s1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    ms_smear = s0.elapsed_time(s1)
    st = cl.status(stream=stream)
    cl.close()
    del ps
    return {"workload": wl.name, "label": "EL bubbles + Gaussian smearing (FP64)", "precision": "fp64",
            "bubbles": wl.n_bubbles, "cells": wl.edge ** 3,
            "value": wl.n_bubbles * args.steps / (ms * 1e-3), "unit": "bubble-steps/s",
            "ms_per_step": ms / args.steps, "smear_ms_per_step": ms_smear / args.steps,
            "trials_per_bubble_step": st["n_attempts"] / (wl.n_bubbles * args.steps),
            "status_flags": st["flags"]}


def _summary(line):
    """The line's headline figures in a few hundred characters (3 significant digits): the
    default line, the end-to-end figure, the FMA probe and each extra line's value with its
    distinguishing figures."""
    def g(x):
        return float(f"{x:.3g}") if isinstance(x, (int, float)) and x == x else x
    out = {"value": g(line["value"]), "frac": g(line["roofline"].get("frac")),
           "frac_meas": g(line["roofline"].get("frac_of_measured")), "e2e": g(line["e2e"]["value"])}
    fma = line.get("fma_probe") or {}
    if "fp64_tflops" in fma:
        out["fma_tflops"] = [g(fma["fp64_tflops"]), g(fma["fp32_tflops"])]
    for v in line.get("variants", []):
        key = v.get("workload", "?")
        if "error" in v:
            out[key] = "error"
            continue
        e = {"v": g(v.get("value"))}
        if "trials_per_bin_step" in v:
            e["tr"] = g(v["trials_per_bin_step"])
        if v.get("fp64_trial_fraction"):
            e["f64"] = g(v["fp64_trial_fraction"])
        if v.get("vs_single_instance_same_work") is not None:
            e["vs1"] = g(v["vs_single_instance_same_work"])
        r = v.get("roofline") or {}
        for k_src, k_dst in (("frac", "frac"), ("fp64_frac", "f64frac"), ("fp32_frac", "f32frac")):
            if r.get(k_src) is not None:
                e[k_dst] = g(r[k_src])
        eo = v.get("error_vs_oracle") or v.get("error_vs_fp64_kernel") or {}
        if "alpha" in eo:
            e["err_a"] = g(eo["alpha"])
            e["err_R"] = g(eo["R"])
        if "pab_bubble_step" in v:
            e = {"dev_p50_p99_ms": [g(v["pab_bubble_step"]["p50_ms"]), g(v["pab_bubble_step"]["p99_ms"])],
                 "host_p50_p99_ms": [g(v["pab_bubble_step_host"]["p50_ms"]),
                                     g(v["pab_bubble_step_host"]["p99_ms"])]}
        if "latency_s" in v:
            e["p50_p99_s"] = [g(v["latency_s"]["p50"]), g(v["latency_s"]["p99"])]
        if "rates" in v:
            e = {str(x["rate"]): [g(x["latency_s"]["p50"]), g(x["latency_s"]["p99"]), g(x["gpu_busy"])]
                 for x in v["rates"]}
        out[key] = e
    return out


def run_ours(args):
    import torch

    from paper_2511_21031_gb300 import pab
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    wl = make_workload(args.workload, rank, args.edge)
    precision = args.precision or wl.precision

    # cpu baseline first, on rank 0 only, before any heavy GPU work
    cpu = cpu_baseline(wl, seconds=args.cpu_seconds) if (rank == 0 and ws == 1 and args.cpu_seconds > 0) else None

    stream = torch.cuda.Stream()
    total = args.warmup + args.steps
    with torch.cuda.stream(stream):
        solver = pab.Solver(wl.n_cells, wl.n_bins, precision=precision, s_lognormal=wl.s,
                            R0ref=wl.R0ref, span_K=wl.span_K, alpha0=wl.alpha0)
        if args.block_warps:
            solver.set_block_warps(args.block_warps)
        ps = [wl.pressure_step(n, xp=torch, device=dev) for n in range(total)]
        solver.moments()  # one reduce-only launch (profiled for its per-bin cost)
    torch.cuda.synchronize()
    dev_index = torch.cuda.current_device()
    res = _time_steps(solver, wl, ps, args, stream,
                      clocks=ClockSampler(dev_index, ClockSampler.device_uuid(dev_index)),
                      keep_start=True)
    if "trace" in res:
        if rank == 0:
            print(json.dumps({"trace_trials": res["trace"], "bin_steps_per_launch": wl.n_cells * wl.n_bins,
                              "workload": wl.name, "precision": precision}), flush=True)
        solver.close()
        return 0
    ms_total, launch_ms, st, clk = res["ms_total"], res["launch_ms"], res["status"], res["clocks"]

    # end to end through the host-buffer C-ABI entry points (pinned host memory), over the
    # same steps from the same state as the timed region: the pipelined call (the input copy
    # of step k+1 and the output copy of step k overlap the steps; two host buffer sets),
    # then the synchronous call for reference
    n_e2e = args.steps
    ph = [ps[args.warmup + k].cpu().pin_memory() for k in range(n_e2e)]
    mh = [torch.empty((pab.N_MOMENTS, wl.n_cells), dtype=torch.float64).pin_memory() for _ in range(2)]
    solver.step_host_async(ph[0], wl.dt, moments_host=mh[0], stream=stream)  # warm the pipeline
    solver.host_wait()

    def e2e_run(pipelined):
        solver.set_state(*res["start"], stream=stream)
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        t0 = time.perf_counter()
        for k in range(n_e2e):
            if pipelined:
                solver.step_host_async(ph[k], wl.dt, moments_host=mh[k % 2], stream=stream)
            else:
                solver.step_host(ph[k], wl.dt, moments_host=mh[0], stream=stream)
        solver.host_wait()
        return pdist.max_over_ranks(time.perf_counter() - t0, device=dev)

    e2e_s = e2e_run(True)
    e2e_sync_s = e2e_run(False)
    solver.status(stream=stream)
    solver.close()
    del ps

    bin_steps = wl.n_cells * wl.n_bins * args.steps
    value = pdist.weak_scaling_value(bin_steps, ms_total, ws)
    trials_per_binstep = st["n_attempts"] / bin_steps
    avg_launch_s = statistics.mean(launch_ms) * 1e-3
    sm_mhz = clk["sm_mhz"] if clk else SM_MAX_MHZ
    if precision == "fp64":
        flops_per_launch = wl.n_cells * wl.n_bins * (trials_per_binstep * FP64_FLOPS_PER_TRIAL
                                                     + FP64_FLOPS_PER_BINSTEP)
        peak = NOMINAL_FP64_FLOPS_PER_CLK_PER_SM * N_SM * SM_MAX_MHZ * 1e6
        roof = {"bound": "alu", "achieved": flops_per_launch / avg_launch_s / 1e12,
                "peak": peak / 1e12, "unit": "TFLOP/s",
                "frac": flops_per_launch / avg_launch_s / peak,
                "traffic": FP64_DRAM_BYTES_PER_BINSTEP * wl.n_cells * wl.n_bins,
                "fp64_pipe_active_ncu": FP64_PIPE_ACTIVE_NCU,
                "pipe": "fp64", "peak_source": "derived: 4 FP64 flop/clk/SM x 152 SMs x 2070 MHz",
                "frac_at_measured_clock": flops_per_launch / avg_launch_s
                / (NOMINAL_FP64_FLOPS_PER_CLK_PER_SM * N_SM * sm_mhz * 1e6),
                # with the operations the integer pipe forms in place of FP64 instructions,
                # counted as those instructions would be (context: no FP64 pipe executes them)
                "achieved_with_int_pipe": (flops_per_launch + wl.n_cells * wl.n_bins
                                           * (trials_per_binstep * FP64_INT_PIPE_FLOPS_PER_TRIAL
                                              + FP64_INT_PIPE_FLOPS_PER_BINSTEP)) / avg_launch_s / 1e12,
                "int_pipe_flops_per_trial": FP64_INT_PIPE_FLOPS_PER_TRIAL,
                "int_pipe_flops_per_binstep": FP64_INT_PIPE_FLOPS_PER_BINSTEP}
    else:
        roof = {"bound": "alu", "achieved": None, "peak": None, "unit": "TFLOP/s", "frac": None,
                "traffic": None, "pipe": "fp64+fp32"}

    variants = []
    if args.variants and args.mixed and ws == 1:
        for name, vwl in (("grid128 mixed", wl), ("grid256 mixed", make_workload("grid256_mixed", rank))):
            vs = pab.Solver(vwl.n_cells, vwl.n_bins, precision="mixed", s_lognormal=vwl.s,
                            R0ref=vwl.R0ref, span_K=vwl.span_K, alpha0=vwl.alpha0)
            with torch.cuda.stream(stream):
                vps = [vwl.pressure_step(n, xp=torch, device=dev) for n in range(total)]
            torch.cuda.synchronize()
            r = _time_steps(vs, vwl, vps, args, stream)
            vbs = vwl.n_cells * vwl.n_bins * args.steps
            variants.append({
                "workload": vwl.name.replace("_fp64", "_mixed").replace("_mixed_mixed", "_mixed"),
                "label": name, "precision": "mixed",
                "value": vbs / (r["ms_total"] * 1e-3), "unit": "bin-steps/s",
                "ms_per_step": r["ms_total"] / args.steps,
                "latency_ms": {"p50": float(np.percentile(r["launch_ms"], 50)),
                               "p99": float(np.percentile(r["launch_ms"], 99))},
                "trials_per_bin_step": r["status"]["n_attempts"] / vbs,
                "fp64_trial_fraction": r["status"]["n_fp64"] / max(1, r["status"]["n_attempts"]),
                "speedup_vs_fp64_grid128": (vbs / (r["ms_total"] * 1e-3)) / value,
                "error_vs_oracle": _mixed_error_sample(vwl, min(total, 40)),
                "roofline": _mixed_compute_roofline(
                    vbs / (r["ms_total"] * 1e-3), r["status"]["n_attempts"] / vbs,
                    r["status"]["n_fp64"] / max(1, r["status"]["n_attempts"])),
            })
            vs.close()
            del vps
            torch.cuda.synchronize()

    def extra(name, fn):
        # a failed extra line must not cost the bench its result: it is recorded instead
        try:
            variants.append(fn())
        except Exception as e:
            entry = {"workload": name, "error": repr(e)[:300]}
            try:
                torch.cuda.synchronize()
            except Exception as e2:    # a sticky CUDA error: recorded, the line still prints
                entry["sync_error"] = repr(e2)[:300]
            variants.append(entry)

    def batched():
        bv = _bench_batched(args, stream, dev, n_instances=args.batch_instances)
        bv["speedup_vs_fp64_grid128"] = bv["value"] / value
        bv["roofline"] = _mixed_compute_roofline(bv["value"], bv["trials_per_bin_step"],
                                                 bv["fp64_trial_fraction"], batched=True)
        return bv

    def batched_slices():
        # the batch on exactly the single-instance mixed line's work: the 128^3 grid cut into
        # 512 instances of 16^3 cells, so the ratio of the two rates is the batch's own cost
        n = 512 if wl.n_cells % 512 == 0 else 1
        insts = workloads.sliced_instances(wl, n)
        bv = _bench_batched(args, stream, dev, insts=insts,
                            name=f"batched {n} slices of {wl.name.replace('_fp64', '_mixed')}")
        single = next((v for v in variants if v.get("label") == "grid128 mixed"
                       and "value" in v), None)
        bv["vs_single_instance_same_work"] = bv["value"] / single["value"] if single else None
        bv["roofline"] = _mixed_compute_roofline(bv["value"], bv["trials_per_bin_step"],
                                                 bv["fp64_trial_fraction"], batched=True)
        return bv

    if args.variants and args.transfer and ws == 1:
        extra("transfer", lambda: _bench_transfer(args, stream, dev, value))
    if args.variants and args.batched and ws == 1:
        extra("batched", batched)
        extra("batched slices", batched_slices)
    if args.variants and args.el and ws == 1:
        extra("el", lambda: _bench_el(args, stream, dev))
    if args.variants and args.closure and ws == 1:
        extra("strang closure", lambda: _bench_closure(args, stream, dev))
    if args.variants and args.serving and ws == 1:
        extra("serving", lambda: _bench_serving(args))
    if args.variants and args.collapse and ws == 1:
        if args.collapse_precision in ("both", "fp64"):
            extra("collapse fp64", lambda: _bench_collapse(args, stream, dev, "fp64"))
        if args.collapse_precision in ("both", "mixed"):
            extra("collapse mixed", lambda: _bench_collapse(args, stream, dev, "mixed"))
    if args.variants and args.latency and ws == 1:
        extra("latency small", lambda: _bench_latency_small(args, stream, dev))
    if args.variants and args.serving and args.serving_sweep and ws == 1:
        extra("serving sweep", lambda: _bench_serving_sweep(args, args.sweep_rates, args.sweep_requests))

    fma = None
    if args.peak_probe:
        # dependent-FMA throughput on every SM, FP64 and FP32 (measured beside the derived peaks)
        try:
            sink = torch.empty(N_SM * 16 * 256, dtype=torch.float64, device=dev)
            sp = int(stream.cuda_stream)
            pab.pab_peak_fma(pab.PAB_FP64, N_SM * 16, 256, 200, sink.data_ptr(), sp)   # warm
            ms, n = pab.pab_peak_fma(pab.PAB_FP64, N_SM * 16, 256, 2000, sink.data_ptr(), sp)
            ms32, n32 = pab.pab_peak_fma(pab.PAB_MIXED, N_SM * 16, 256, 20000, sink.data_ptr(), sp)
            fma = {"fp64_tflops": 2 * n / (ms * 1e-3) / 1e12, "fp32_tflops": 2 * n32 / (ms32 * 1e-3) / 1e12,
                   "fp64_derived_tflops": _fp64_peak_derived() / 1e12,
                   "fp32_derived_tflops": _fp32_peak_derived() / 1e12,
                   "how": "pab_peak_fma: 8 dependent FMA chains per thread, 2432 CTAs of 256 threads"}
            del sink
        except Exception as e:
            fma = {"error": repr(e)[:200]}
    if fma and "fp64_tflops" in fma and roof.get("achieved"):
        roof["peak_measured"] = fma["fp64_tflops"]
        roof["frac_of_measured"] = roof["achieved"] / fma["fp64_tflops"]
        roof["peak_measured_source"] = "pab_peak_fma in this run (fma_probe)"
    for v in variants:
        r = v.get("roofline") if isinstance(v, dict) else None
        if not (r and fma and "fp64_tflops" in fma):
            continue
        if r.get("pipe") == "fp64" and r.get("achieved"):
            r["frac_of_measured"] = r["achieved"] / fma["fp64_tflops"]
        if r.get("fp64_tflops") is not None:
            r["fp64_frac_of_measured"] = r["fp64_tflops"] / fma["fp64_tflops"]
            r["fp32_frac_of_measured"] = r["fp32_tflops"] / fma["fp32_tflops"]

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "bin-steps/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if precision == "fp64" else "f32+f64", "data": "synthetic",
            "config": {"workload": wl.name, "cells": wl.n_cells, "bins": wl.n_bins, "s": wl.s,
                       "dt": wl.dt, "forcing": f"{wl.amp} p0 at {wl.freq:g} Hz", "precision": precision,
                       "stepper": "adaptive SSP-RK3(2) tol 1e-4",
                       "l2": "no flush: the state (20 B per bin-step) is larger than L2",
                       "parallelism": f"{ws} independent blocks (weak)", "seed": wl.seed},
            "gpu_launches": args.steps,
            "latency_ms": {"p50": float(np.percentile(launch_ms, 50)),
                           "p99": float(np.percentile(launch_ms, 99))},
            "trials_per_bin_step": trials_per_binstep,
            "status_flags": st["flags"],
            "roofline": roof,
            "e2e": {"value": wl.n_cells * wl.n_bins * n_e2e * ws / e2e_s, "unit": "bin-steps/s",
                    "h2d_bytes_per_step": wl.n_cells * 8, "d2h_bytes_per_step": 7 * wl.n_cells * 8,
                    "api": "pab_bubble_step_host_async (2 in flight) + pab_host_wait",
                    "steps": n_e2e, "work": "the timed steps again, from the state they started from",
                    "sync_value": wl.n_cells * wl.n_bins * n_e2e * ws / e2e_sync_s},
            "clocks": clk,
            "cpu_baseline": cpu,
        }
        if variants:
            line["variants"] = variants
        if fma:
            line["fma_probe"] = fma
        line["summary"] = _summary(line)   # last, so that a record keeping the line's tail keeps it
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=("ours", "reference"))
    ap.add_argument("--workload", default="grid128")
    ap.add_argument("--precision", default=None, choices=(None, "fp64", "mixed"))
    ap.add_argument("--block-warps", type=int, default=0)
    ap.add_argument("--edge", type=int, default=0, help="grid edge override (profiling runs)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-peak-probe", dest="peak_probe", action="store_false",
                    help="skip the FP64/FP32 FMA-throughput probe")
    ap.add_argument("--no-collapse", dest="collapse", action="store_false",
                    help="skip the collapse-stress lines (64^3 x 31, 21.4 kHz, one period)")
    ap.add_argument("--collapse-edge", type=int, default=64)
    ap.add_argument("--collapse-steps", type=int, default=10000)
    ap.add_argument("--collapse-precision", default="both", choices=("both", "fp64", "mixed"))
    ap.add_argument("--collapse-save", default=None,
                    help="profiling aid: save the collapse line's final state to this file")
    ap.add_argument("--collapse-load", default=None,
                    help="profiling aid: start the collapse line from a saved state")
    ap.add_argument("--no-latency", dest="latency", action="store_false",
                    help="skip the per-call latency line of the 64-cell workload")
    ap.add_argument("--no-serving-sweep", dest="serving_sweep", action="store_false",
                    help="skip the serving rate sweep (about 75 s of wall time; --no-serving skips it too)")
    ap.add_argument("--sweep-rates", type=float, nargs="+", default=[2.0, 3.5, 5.0],
                    help="offered request rates of the sweep: below, near and above saturation")
    ap.add_argument("--sweep-requests", type=int, default=64)
    ap.add_argument("--no-variants", dest="variants", action="store_false",
                    help="skip the mixed-precision and batched lines")
    ap.add_argument("--no-batched", dest="batched", action="store_false",
                    help="skip the 512-instance batched line")
    ap.add_argument("--no-serving", dest="serving", action="store_false",
                    help="skip the continuous-batching serving line")
    ap.add_argument("--no-transfer", dest="transfer", action="store_false",
                    help="skip the heat-and-mass-transfer contents line")
    ap.add_argument("--no-closure", dest="closure", action="store_false",
                    help="skip the Strang-split flow step with the carrier-coupling kernels")
    ap.add_argument("--no-el", dest="el", action="store_false",
                    help="skip the volume-averaged (EL) line")
    ap.add_argument("--no-mixed", dest="mixed", action="store_false",
                    help="skip the single-instance mixed-precision lines")
    ap.add_argument("--trace-trials", action="store_true",
                    help="profiling aid: print the trials of every step launch (no timing)")
    ap.add_argument("--batch-launch", type=int, nargs=3, default=None, metavar=("WARPS", "CTAS_PER_SM", "GRAB"),
                    help="profiling aid: the batched line's launch shape, instead of the autotuner's")
    ap.add_argument("--batch-instances", type=int, default=512,
                    help="instances of the batched line (profiling runs use fewer)")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
