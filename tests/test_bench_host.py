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
