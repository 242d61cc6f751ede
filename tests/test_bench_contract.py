"""The JSON line of bench.py: the reference arm (the oracle on the host
cores, no GPU) and, marked gpu, the GB300 arm's main line."""
import json
import math
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(args, timeout):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args],
                       capture_output=True, text=True, timeout=timeout, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    return json.loads(lines[0])


def _common(line):
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config"):
        assert k in line, k
    assert line["unit"] == "photons/s" and line["higher_is_better"] is True
    assert line["scaling"] == "weak" and line["data"] == "synthetic"
    assert line["config"]["workload"] == "rich1_meshed_1000_pion_tracks"
    assert line["value"] > 0 and line["ms_per_step"] > 0


def test_reference_arm_line():
    """--impl reference times the oracle on the host cores on the same
    workload, with its cpu_baseline and a host-only e2e of the same value."""
    line = _run(["--impl", "reference", "--steps", "1", "--warmup", "1"], timeout=600)
    _common(line)
    assert line["impl"] == "reference" and line["dtype"] == "f64"
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "photons/s",
                           "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    ph = line["config"]["photons_per_step"]
    assert 3.0e5 < ph < 4.0e5
    assert line["value"] == pytest.approx(ph / (line["ms_per_step"] / 1e3), rel=1e-6)


@pytest.mark.gpu
def test_gb300_arm_main_line():
    """The GB300 arm without the extra legs: rate from the timed steps, the
    roofline's fraction as achieved over peak for the slower of its FP32 and
    L2 bounds, the clock record and the launch count."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    line = _run(["--steps", "4", "--warmup", "3", "--no-extras"], timeout=900)
    _common(line)
    assert line["n_gpus"] == 1 and line["steps"] == 4 and line["warmup"] == 3
    assert line["dtype"] == "f32"
    assert line["value"] == pytest.approx(
        line["config"]["photons_per_step"] / (line["ms_per_step"] / 1e3), rel=0.01)
    assert line["gpu_launches"] == 4 * 4
    r = line["roofline"]
    assert r["bound"] in ("l2", "fp32") and r["unit"] in ("GB/s", "TFLOP/s")
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"], rel=1e-9)
    b = r["bounds"]
    assert set(b) >= {"fp32", "l2", "l2_outside_smem", "alu_minmax", "mufu", "hbm"}
    slower = "l2" if b["l2"]["frac"] >= b["fp32"]["frac"] else "fp32"
    assert r["bound"] == slower
    for v in b.values():
        assert v["frac"] == pytest.approx(v["achieved"] / v["peak"], rel=1e-9)
        assert math.isfinite(v["photons_per_s_bound"])
    assert 0.0 < r["frac"] < 1.5
    assert r["kernel_ms"] > 0 and r["kernel_ms"] < line["ms_per_step"]
    assert "sm_mhz" in line["clocks"] and "reasons" in line["clocks"]
