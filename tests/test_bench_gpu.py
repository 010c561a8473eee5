"""bench.py keeps its JSON-line contract: one line with the metric, the
device-timed value, the roofline of the dominant kernel, end-to-end figures
through host buffers, the launch count and the clocks sampled while timing."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bench_json_line_contract():
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--workload", "ring-2^25-f64", "--steps", "2",
                        "--warmup", "3", "--no-cpu-baseline"], capture_output=True, text=True, cwd=ROOT, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "roofline", "e2e", "gpu_launches", "clocks"):
        assert k in d, k
    assert d["unit"] == "GLUP/s" and d["value"] > 0 and d["warmup"] >= 3
    assert isinstance(d["clocks"], dict) and "sm_max_mhz" in d["clocks"]   # None when the run was shorter than a sample
    rf = d["roofline"]
    assert rf["bound"] == "alu" and rf["achieved"] > 0 and rf["fp64_unit_peak"] > 0
    assert rf["emul_share_of_32"] == d["config"]["emul_share_of_32"]
    e = d["e2e"]
    assert e["value"] > 0 and e["h2d_bytes_per_step"] == e["d2h_bytes_per_step"] == 8 * (1 << 25)
    # copies run beside the other context's steps, never instead of them
    assert e["value"] <= 1.1 * d["value"] and e["contexts_agree_bitwise"] is True
    assert d["gpu_launches"] > 0
    # the plain one-step-per-launch kernel on the same ring, beside the headline
    pl = d["plain"]
    assert pl["form"] == "plain" and pl["value"] > 0 and pl["launches_per_step"] == 20
    assert 0 < pl["hbm"]["frac"] < 1.2 and 0 < pl["fp64_unit"]["frac"] < 1.2
    assert abs(pl["headline_over_plain"] - d["value"] / pl["value"]) < 1e-9
