"""Host-side contract of bench.py that needs no GPU: the reference arm's JSON
line (the oracle timed on the host cores), the roofline helpers of the mixed
and batched lines with and without a measured peak, and the warm-up floor."""
import builtins
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_line_with_the_contract_keys():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "3"], capture_output=True, text=True, cwd=ROOT,
                       timeout=600, env=dict(os.environ, OMP_NUM_THREADS="4"))
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [x for x in r.stdout.splitlines() if x.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 1 and d["warmup"] == 3
    assert d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["cpu_baseline"]["cores"] == 4 and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert d["config"]["workload"].startswith("grid128")


def test_warmup_below_three_is_refused():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "2"], capture_output=True, text=True, cwd=ROOT,
                       timeout=300)
    assert r.returncode != 0 and "warmup" in (r.stderr + r.stdout)


def _bench():
    sys.path.insert(0, ROOT)
    import bench
    return bench


@pytest.mark.parametrize("batched", [False, True])
def test_mixed_roofline_object(batched):
    bench = _bench()
    d = bench._mixed_roofline(2.0e10, batched=batched)
    per = bench.BATCH_DRAM_BYTES_PER_BINSTEP if batched else bench.MIXED_DRAM_BYTES_PER_BINSTEP
    assert d["bound"] == "issue"
    assert d["achieved_hbm_gbs"] == pytest.approx(per * 20.0)
    assert d["hbm_frac"] == pytest.approx(d["achieved_hbm_gbs"] / d["hbm_peak_gbs"])
    assert 0.0 < d["issue_active_ncu"] <= 1.0 and 0.0 < d["fp64_pipe_active_ncu"] <= 1.0
    assert os.path.exists(os.path.join(ROOT, d["counters"]))
    assert isinstance(d["counters_build"], str) and d["counters_build"]


def test_hbm_peak_falls_back_when_no_measurement_is_there(monkeypatch):
    bench = _bench()
    real_open = builtins.open

    def no_peaks(path, *a, **k):
        if str(path).endswith("MEASURED_PEAKS.json"):
            raise OSError("absent")
        return real_open(path, *a, **k)

    monkeypatch.setattr(builtins, "open", no_peaks)
    peak, src = bench._hbm_peak()
    assert peak == bench.HBM_FALLBACK_GBS and "fallback" in src


def test_clock_summary_of_nvidia_smi_samples():
    """The samples of the bench's own GPU (by UUID, else by index) give the median SM clock, the
    maximum and every throttle reason seen active ("Not Active" is not); other GPUs' samples and
    malformed lines are ignored, and no samples give None."""
    bench = _bench()
    na, a = "Not Active", "Active"
    U0, U3 = "GPU-aaaa0000-0000-0000-0000-000000000000", "GPU-bbbb3333-3333-3333-3333-333333333333"
    lines = [
        f"0, {U0}, 2070, 2070, 900.1, 0x0000000000000000, {na}, {na}, {na}, {na}",
        f"3, {U3}, 1500, 2070, 1390.5, 0x0000000000000008, {a}, {na}, {na}, {na}",
        f"0, {U0}, 1980, 2070, 1390.5, 0x0000000000000004, {na}, {na}, {na}, {a}",
        "garbage",
        f"0, {U0}, [N/A], 2070, 1000.0, 0x0, {na}, {na}, {na}, {na}",
        f"3, {U3}, 1400, 2070, 1390.5, 0x0000000000000008, {a}, {na}, {na}, {na}",
        f"0, {U0}, 2040, 2070, 1200.0, 0x0000000000000000, {na}, {na}, {na}, {na}",
    ]
    # torch's device 0 is nvidia-smi's GPU 3 (UUID without the GPU- prefix, as torch prints it)
    d = bench.ClockSampler.summarise(lines, 0, U3[4:])
    assert d["matched_by"] == "uuid" and d["gpu"] == U3 and d["samples"] == 2
    assert d["sm_mhz"] == 1450.0 and d["reasons"] == ["hw_slowdown"]
    # UUID unknown or not listed: the index decides, as nvidia-smi numbers them
    for u in (None, "GPU-ffff"):
        d = bench.ClockSampler.summarise(lines, 0, u)
        assert d == {"sm_mhz": 2040.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3,
                     "gpu": "index 0", "matched_by": "index"}
    assert bench.ClockSampler.summarise(lines, 5, None) is None
    assert bench.ClockSampler.summarise([], 0) is None and bench.ClockSampler.summarise(["x"], 0) is None


def test_mixed_error_report_covers_every_output():
    """The bench's mixed-against-FP64 error: zero for equal outputs, the planted relative error
    for each output, and the floors where a value passes through zero."""
    import numpy as np
    bench = _bench()
    g = np.random.Generator(np.random.PCG64(5))
    B, C, vf = 5, 7, 1e-2
    w = g.uniform(0.1, 1.0, B)
    w /= w.sum()
    Rd = g.uniform(5e-6, 2e-5, (B, C))
    Vd = g.normal(0.0, 1.0, (B, C))
    o = np.abs(g.normal(1.0, 0.1, (7, C)))
    o[3] = g.normal(0.0, 1e-10, C)           # signed sums
    o[4] = g.normal(0.0, 1e3, C)
    e0 = bench._mixed_errors(o.copy(), o, Rd.copy(), Vd.copy(), Rd, Vd, w, vf)
    keys = {"R", "Rdot", "alpha", "R3", "R2Rdot", "S_alpha", "R3pbw_over_R3", "R3Rdot2_over_R3"}
    assert set(e0) == keys and all(v == 0.0 for v in e0.values())
    eps = 1e-7
    e = bench._mixed_errors(o * (1 + eps), o, Rd * (1 + eps), Vd * (1 + eps), Rd, Vd, w, vf)
    for k in ("R", "alpha", "R3", "R3pbw_over_R3"):
        assert e[k] == pytest.approx(eps, rel=1e-6), k
    assert 0.0 < e["Rdot"] <= eps * (1 + 1e-6)
    assert 0.0 < e["R2Rdot"] < eps and 0.0 < e["S_alpha"] and e["R3Rdot2_over_R3"] <= eps * (1 + 1e-6)


def test_closure_line_times_each_kernel_group(monkeypatch):
    """The Strang-split closure line on the CPU with a fake solver whose calls advance a fake
    event clock by known amounts: per-group times, the flow-step rate and each closure kernel's
    algorithmic bandwidth come out of that clock, and set_conservative gets alpha from row 1."""
    import contextlib
    import types

    import torch
    from paper_2511_21031_gb300 import pab
    bench = _bench()
    clock = [0.0]
    cost = {"strang_half": 4.0, "mixture_pressure": 1.0, "get_conservative": 2.0, "set_conservative": 3.0}

    class FakeSolver:
        def __init__(self, C, B, **kw):
            self.C, self.B = C, B

        def strang_half(self, p, dt, moments=None, stream=None):
            assert p.shape == (self.C,) and moments.shape == (pab.N_MOMENTS, self.C)
            clock[0] += cost["strang_half"]

        def mixture_pressure(self, m, p_l, out=None, stream=None):
            clock[0] += cost["mixture_pressure"]

        def get_conservative(self, stream=None):
            clock[0] += cost["get_conservative"]
            return torch.zeros((self.B, self.C)), torch.zeros((self.B, self.C))

        def set_conservative(self, alpha, qR, qV, stream=None):
            assert alpha.shape == (self.C,) and qR.shape == (self.B, self.C)
            clock[0] += cost["set_conservative"]

        def status(self, stream=None):
            return {"n_attempts": 7, "flags": 0}

        def close(self):
            pass

    class FakeEvent:
        def __init__(self, enable_timing=False):
            self.t = None

        def record(self, stream=None):
            self.t = clock[0]

        def elapsed_time(self, other):
            return other.t - self.t

    monkeypatch.setattr(pab, "Solver", FakeSolver)
    monkeypatch.setattr(torch.cuda, "Event", FakeEvent)
    monkeypatch.setattr(torch.cuda, "stream", lambda s: contextlib.nullcontext())
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a: None)
    args = types.SimpleNamespace(edge=8, warmup=3, steps=2)
    d = bench._bench_closure(args, None, torch.device("cpu"))
    C, B = 8 ** 3, 31
    assert d["ms_per_step"] == pytest.approx(14.0) and d["half_steps_ms_per_step"] == pytest.approx(8.0)
    assert d["value"] == pytest.approx(C * B / 14e-3)
    k = d["closure_kernels"]
    assert k["mixture_pressure"]["ms_per_step"] == pytest.approx(1.0)
    assert k["mixture_pressure"]["algorithmic_gbs"] == pytest.approx(40.0 * C / 1e-3 / 1e9)
    assert k["get_conservative"]["algorithmic_gbs"] == pytest.approx(32.0 * C * B / 2e-3 / 1e9)
    assert k["set_conservative"]["algorithmic_gbs"] == pytest.approx((16.0 * C + 32.0 * C * B) / 3e-3 / 1e9)
    assert k["set_conservative"]["hbm_frac"] == pytest.approx(k["set_conservative"]["algorithmic_gbs"] / d["hbm_peak_gbs"])
    pipe = 2.0 * 152 * 2070e6
    assert k["set_conservative"]["fp64_pipe_frac"] == pytest.approx((13.0 * C + 1.0 * C * B) / 3e-3 / pipe)
    assert k["get_conservative"]["fp64_pipe_frac"] == pytest.approx(2.0 * C * B / 2e-3 / pipe)
    assert d["status_flags"] == 0 and d["workload"].endswith("strang")


def test_mixed_compute_roofline_applies_the_flop_fit(monkeypatch):
    """FP32 and FP64 flops per second from the fitted flops per trial and per bin-step: FP32
    trials carry the FP32 and the FP64 bookkeeping of a trial, collapse trials the FP64 trial's."""
    bench = _bench()
    fit = {"fp32_per_trial": 100.0, "fp64_per_trial": 20.0, "fp64_per_fp64_trial": 130.0,
           "fp32_per_binstep": 10.0, "fp64_per_binstep": 5.0, "source": "test"}
    monkeypatch.setattr(bench, "MIXED_FLOPS", fit)
    d = bench._mixed_compute_roofline(1e10, 1.5, 0.1)
    t32, t64 = 1.5 * 0.9, 1.5 * 0.1
    assert d["fp32_tflops"] == pytest.approx(1e10 * (t32 * 100.0 + 10.0) / 1e12)
    assert d["fp64_tflops"] == pytest.approx(1e10 * (t32 * 20.0 + t64 * 130.0 + 5.0) / 1e12)
    assert d["fp32_frac"] == pytest.approx(d["fp32_tflops"] * 1e12 / bench._fp32_peak_derived())
    assert d["fp64_frac"] == pytest.approx(d["fp64_tflops"] * 1e12 / bench._fp64_peak_derived())
    monkeypatch.setattr(bench, "MIXED_FLOPS", None)
    assert bench._mixed_compute_roofline(1e10, 1.5, 0.1)["fp64_frac"] is None


def test_summary_keeps_every_line_within_the_recorded_tail():
    """The summary closes the JSON line and names every extra line's value, so a record that
    keeps only the line's last 1500 characters keeps the headline figures of every line."""
    bench = _bench()
    lat = {"p50_ms": 0.05, "p99_ms": 0.07}
    line = {"value": 4.2e9, "roofline": {"frac": 0.65, "frac_of_measured": 0.77},
            "e2e": {"value": 4.1e9}, "fma_probe": {"fp64_tflops": 1.05, "fp32_tflops": 70.1},
            "variants": [
                {"workload": f"w{i}", "value": 1.23456e9 * (i + 1), "trials_per_bin_step": 1.05,
                 "fp64_trial_fraction": 0.011, "roofline": {"fp64_frac": 0.5, "fp32_frac": 0.05},
                 "error_vs_oracle": {"alpha": 1e-7, "R": 3e-5}} for i in range(8)]
            + [{"workload": "lat", "value": 1.0, "pab_bubble_step": lat, "pab_bubble_step_host": lat},
               {"workload": "bad", "error": "RuntimeError('x')"}]}
    s = bench._summary(line)
    assert s["value"] == 4.2e9 and s["frac_meas"] == 0.77 and s["fma_tflops"] == [1.05, 70.1]
    assert s["w3"]["v"] == 4.94e9 and s["w0"]["f64"] == 0.011 and s["w0"]["err_a"] == 1e-7
    assert s["lat"]["dev_p50_p99_ms"] == [0.05, 0.07] and s["bad"] == "error"
    assert len(json.dumps({"summary": s})) < 1500
