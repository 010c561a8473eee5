"""Host check of the integer-pipe binary64 routines (csrc/dp_emul.cuh) against
the host's IEEE 754 arithmetic (CPU only; the routines compile for the host).

Covers random magnitudes, near-cancellation, exponent differences 0..70, exact
ties, power-of-two and general multipliers, whole Eq. 2 chains, and raw random
bit patterns (where exceptional operands must be flagged, never computed
wrongly)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_integer_binary64_matches_host_ieee(tmp_path):
    exe = tmp_path / "emul_check"
    subprocess.check_call(["g++", "-O2", "-ffp-contract=off", "-std=c++17", "-o", str(exe),
                           os.path.join(ROOT, "tests", "emul_check.cpp"), "-lm"])
    p = subprocess.run([str(exe), "300000"], capture_output=True, text=True)
    assert p.returncode == 0, p.stdout + p.stderr
    lines = dict(l.split(" ", 1) for l in p.stdout.strip().splitlines() if " mismatches=" in l)
    for cat in ("add", "mul", "eq2", "raw", "edge"):
        assert cat in lines and lines[cat].startswith("mismatches=0"), p.stdout
    # ordinary finite data never leaves the routines' domain
    for cat in ("add", "mul", "eq2", "edge"):
        assert " bad=0 " in " " + lines[cat] + " ", p.stdout
