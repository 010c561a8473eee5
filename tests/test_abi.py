"""The C ABI library loads and exports every entry point include/heat.h declares
(CPU only: argument validation and static strings, no device work)."""
import ctypes
import os
import re

import pytest

from paper_2307_01117_gb300 import heat as H

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for hdr in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not hdr.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", hdr)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(heat_[a-z0-9_]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2307_01117_gb300 import build
    build.build()
    return H.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("heat_create", "heat_set", "heat_get", "heat_run", "heat_destroy", "heat_strerror", "heat_sum"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    assert set(declared_functions()) <= set(H._PROTOS)


def test_strerror_is_static_text(lib):
    assert H.heat_strerror(H.HEAT_OK) == "ok"
    assert "wait" in H.heat_strerror(H.HEAT_ETIMEOUT)
    assert H.heat_strerror(12345) == "unknown status"


@pytest.mark.parametrize("args", [
    (0, 1, 0.5, 1.0, 1.0, 0),            # nx < 1
    (10, 0, 0.5, 1.0, 1.0, 0),           # np < 1
    (2**62, 4, 0.5, 1.0, 1.0, 0),        # N overflows int64
    (10, 2, float("nan"), 1.0, 1.0, 0),  # non-finite k
    (10, 2, 0.5, float("inf"), 1.0, 0),  # non-finite dt
    (10, 2, 0.5, 1.0, 0.0, 0),           # dx == 0
    (10, 2, 0.5, 1.0, 1.0, 7),           # unknown dtype
    (10, 2, 1e300, 1e300, 1e-300, 0),    # r overflows
])
def test_create_rejects_bad_arguments_before_any_device_work(lib, args):
    h = ctypes.c_void_p(123)
    rc = lib.heat_create(ctypes.byref(h), *args)
    assert rc == H.HEAT_EINVAL
    assert h.value is None


def test_null_context_is_einval(lib):
    assert lib.heat_run(None, 1) == H.HEAT_EINVAL
    assert lib.heat_sync(None) == H.HEAT_EINVAL
    assert lib.heat_set_form(None, 0, 0) == H.HEAT_EINVAL
    lib.heat_destroy(None)  # no-op


def test_plain_c_client_compiles_links_and_runs(lib, tmp_path):
    """The header is plain C99 and the library links from C (tests/abi_c_client.c)."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("needs gcc")
    libdir = os.path.dirname(H.lib()._name)
    exe = tmp_path / "abi_c_client"
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic",
                           "-I", os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "abi_c_client.c"),
                           "-L", libdir, "-lheat", f"-Wl,-rpath,{libdir}", "-lm", "-o", str(exe)])
    p = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert p.returncode == 0 and "c client ok" in p.stdout, p.stdout + p.stderr
