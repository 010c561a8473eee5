"""bench.py --impl reference: the CPU oracle timed on the host, one JSON line in
the same contract as the GPU arm (CPU only: no device is touched)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run(*extra, env=None):
    e = dict(os.environ, **(env or {}))
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", *extra],
                       capture_output=True, text=True, cwd=ROOT, timeout=300, env=e)
    assert p.returncode == 0, p.stderr[-2000:]
    return [json.loads(l) for l in p.stdout.splitlines() if l.startswith("{")]


@pytest.mark.parametrize("workload", ["ring-4000-f64", "batch-256-f64"])
def test_reference_line(workload):
    (d,) = run("--workload", workload, "--steps", "1", "--warmup", "3")
    assert d["impl"] == "reference" and d["unit"] == "GLUP/s" and d["value"] > 0
    assert d["steps"] == 1 and d["warmup"] == 3 and d["ms_per_step"] > 1000   # one ~2 s sample
    assert d["config"]["workload"] == workload and d["higher_is_better"] is True
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "GLUP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_config_matches_the_gpu_arm_keys():
    (d,) = run("--steps", "1", "--warmup", "3")
    c = d["config"]
    assert (c["workload"], c["N"], c["nt"], c["k"]) == ("ring-2^28-f64", 1 << 28, 1000, 0.25)


def test_other_ranks_stay_silent():
    assert run("--workload", "ring-4000-f64", "--steps", "1", env={"RANK": "1", "WORLD_SIZE": "2"}) == []


def test_cpu_report_runs_the_paper_shaped_configurations_in_full():
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--cpu-report"], capture_output=True,
                       text=True, cwd=ROOT, timeout=300)
    assert p.returncode == 0, p.stderr[-2000:]
    (d,) = [json.loads(l)["cpu_report"] for l in p.stdout.splitlines() if l.startswith("{")]
    assert d["C0_oracle"]["N"] == 10**6 and d["C0_oracle"]["nt"] == 1000 and d["C0_oracle"]["glups"] > 0
    assert d["C1_oracle"]["N"] == 4000 and d["C1_oracle"]["nt"] == 100
    assert {r["threads"] for r in d["C0_threaded"]} >= {2, 20, 40}
