"""The JSON line bench.py prints (the contract its callers parse): the
reference arm on the CPU (a small mesh, the oracle timed as it stands) and the
default arm on the GPU (a small cube), each as a subprocess."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_bench(*args, timeout=600):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT,
                       capture_output=True, text=True, timeout=timeout)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.strip().splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    return json.loads(lines[0])


def common_keys(d):
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "e2e"):
        assert k in d, k
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["unit"] == "G pairs/s" and d["higher_is_better"] is True
    assert d["config"]["workload"].startswith("cube-")
    assert d["e2e"]["value"] > 0 and d["e2e"]["unit"] == d["unit"]


def test_reference_arm_line():
    d = run_bench("--impl", "reference", "--mesh", "4", "--targets", "512", "--steps", "1",
                  "--warmup", "0")
    common_keys(d)
    assert d["impl"] == "reference" and d["dtype"] == "f64"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0


@pytest.mark.gpu
def test_default_arm_line():
    d = run_bench("--mesh", "8", "--targets", "4096", "--steps", "3", "--warmup", "3", "--no-solve",
                  "--no-cpu-baseline", "--no-compensated", "--no-trunc", "--no-fp32-compare")
    common_keys(d)
    assert d["n_gpus"] == 1 and d["steps"] == 3 and d["warmup"] == 3
    roof = d["roofline"]
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in roof, k
    assert roof["frac"] == pytest.approx(roof["achieved"] / roof["peak"])
    assert 0 < roof["frac"] < 1.5
    assert d["gpu_launches"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] > 0 and d["e2e"]["d2h_bytes_per_step"] > 0
    assert "sm_mhz" in d["clocks"] and "reasons" in d["clocks"]
    # pairs per step over the measured time
    pairs = d["config"]["pairs_per_step"]
    assert d["value"] == pytest.approx(pairs / (d["ms_per_step"] * 1e-3) / 1e9, rel=1e-6)
