"""The host check of the integer-pipe binary64 routines catches planted
mistakes (CPU only).  Each mutant is a copy of csrc/dp_emul.cuh with one
plausible mistake in code the host and the GPU share (rounding constants, the
sticky bit, the exponent bias, the product's rounding position, the input
screen's bounds); tests/emul_check.cpp built against the copy must report
mismatches against the host's IEEE arithmetic, or inputs that the screen let
through and that then left the routines' domain."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "paper_2307_01117_gb300", "csrc", "dp_emul.cuh")
CHECK = os.path.join(ROOT, "tests", "emul_check.cpp")

# (name, text in dp_emul.cuh, planted replacement)
MUTANTS = [
    ("rounding ties away from even", "const int64_t q = (Sn + 255 + ((Sn >> 9) & 1)) & ~(int64_t)511;",
     "const int64_t q = (Sn + 256) & ~(int64_t)511;"),
    ("sticky bit dropped (host path)", "  B |= (int64_t)(((uint64_t)B << shc) != (uint64_t)Bs);  // sticky\n#endif",
     "#endif"),
    ("exponent bias off by one in pack", "const uint64_t v = ((uint64_t)(x.e + 1081) << 52) + mag;",
     "const uint64_t v = ((uint64_t)(x.e + 1082) << 52) + mag;"),
    ("product rounded one place low", "const int64_t half_m1 = top ? 127 : 63;", "const int64_t half_m1 = top ? 63 : 31;"),
    ("normalised one place low", "r.e = p >= 0 ? eb + p - 59 : kZeroE;", "r.e = p >= 0 ? eb + p - 60 : kZeroE;"),
    ("screen admits values too small", "lo = 53 + T * shrink + 3;", "lo = 1;"),
]


def run_check(header_text, tmp_path):
    (tmp_path / "tests").mkdir()
    (tmp_path / "paper_2307_01117_gb300" / "csrc").mkdir(parents=True)
    (tmp_path / "paper_2307_01117_gb300" / "csrc" / "dp_emul.cuh").write_text(header_text)
    shutil.copy(CHECK, tmp_path / "tests" / "emul_check.cpp")
    exe = tmp_path / "emul_check"
    subprocess.check_call(["g++", "-O2", "-ffp-contract=off", "-std=c++17", "-o", str(exe),
                           str(tmp_path / "tests" / "emul_check.cpp"), "-lm"])
    p = subprocess.run([str(exe), "100000"], capture_output=True, text=True, timeout=300)
    lines = dict(l.split(" ", 1) for l in p.stdout.strip().splitlines() if " mismatches=" in l)
    return p.returncode, lines


pytestmark = pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(name, old, new, tmp_path):
    text = open(HDR).read()
    assert text.count(old) == 1, name
    rc, lines = run_check(text.replace(old, new), tmp_path)
    mism = {k: int(v.split()[0].split("=")[1]) for k, v in lines.items()}
    bad_tiles = int(lines.get("tile", "mismatches=0 bad=0").split()[1].split("=")[1]) if "tile" in lines else 0
    assert rc != 0 or any(mism.values()) or bad_tiles, f"no category catches: {name}: {lines}"
