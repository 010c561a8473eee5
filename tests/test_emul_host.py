"""Host check of the integer-pipe binary64 routines (csrc/dp_emul.cuh) against
the host's IEEE 754 arithmetic (CPU only; the routines compile for the host).

Packed form: random magnitudes, near-cancellation, exponent differences 0..70,
exact ties, power-of-two and general multipliers, whole Eq. 2 chains, and raw
random bit patterns (where exceptional operands must be flagged, never computed
wrongly).  Unpacked form (whole tiles): the same single-operation cases with
exponent differences up to 560 and exact cancellation to +0, and T-step rings
(T = 1..12; smooth, random, integer-valued and mixed-magnitude data, data at the
input screen's lower bound; power-of-two, general and negative r) compared
step by step with IEEE binary64."""
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
    for cat in ("add", "mul", "eq2", "raw", "edge", "addx", "mulx", "edgex", "tile"):
        assert cat in lines and lines[cat].startswith("mismatches=0"), p.stdout
    # ordinary finite data never leaves the routines' domain (packed form), and
    # every constructed tile passes the unpacked form's screen
    for cat in ("add", "mul", "eq2", "edge", "tile"):
        assert " bad=0 " in " " + lines[cat] + " ", p.stdout
