"""CPU checks of the C ABI: the library builds, loads without a GPU, and
exports every function include/mpgb.h declares (no compute calls)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INCLUDE = os.path.join(ROOT, "include")


def declared_functions():
    names = set()
    for h in sorted(os.listdir(INCLUDE)):
        if h.endswith(".h"):
            src = open(os.path.join(INCLUDE, h)).read()
            names |= set(re.findall(r"MPGB_API\s+[\w\s\*]+?\b(mp_\w+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    from paper_0809_1833_gb300 import build
    return build.build()


def test_header_declares_api():
    names = declared_functions()
    for must in ("mp_plan_create", "mp_plan_destroy", "mp_recover", "mp_recover_batched",
                 "mp_status_string", "mp_last_error_message"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT\s+(mp_\w+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    # nothing undeclared leaks out
    assert exported <= set(declared_functions()), exported - set(declared_functions())


def test_loads_without_gpu_and_binding_covers_header(libpath):
    L = ctypes.CDLL(libpath)
    for n in declared_functions():
        assert hasattr(L, n)
    from paper_0809_1833_gb300 import binding as B
    assert set(B.SIGNATURES) == set(declared_functions())


def test_status_strings(libpath):
    from paper_0809_1833_gb300 import binding as B
    assert B.status_name(B.MP_OK) == "MP_OK"
    assert B.status_name(B.MP_ERR_TIMEOUT) == "MP_ERR_TIMEOUT"
    assert B.status_name(12345) == "MP_UNKNOWN_STATUS"


def test_null_arguments_rejected_on_host(libpath):
    """Argument checks happen before any CUDA call."""
    from paper_0809_1833_gb300 import binding as B
    L = B.lib()
    assert L.mp_plan_create(None, None, None, None) == B.MP_ERR_INVALID
    h = ctypes.c_void_p()
    d = B.mp_plan_desc(0, 5, 0, 0, 0, 0)
    assert L.mp_plan_create(ctypes.byref(h), ctypes.byref(d), ctypes.c_void_p(16), None) == B.MP_ERR_INVALID
    assert "N and M" in B.last_error()
    d = B.mp_plan_desc(4, 5, 7, 0, 0, 0)
    assert L.mp_plan_create(ctypes.byref(h), ctypes.byref(d), ctypes.c_void_p(16), None) == B.MP_ERR_INVALID
    assert L.mp_recover(None, None, None, None, None, None, None) == B.MP_ERR_INVALID
    assert L.mp_plan_destroy(None) == B.MP_OK


def test_header_compiles_as_c(tmp_path):
    c = tmp_path / "t.c"
    incs = "".join(f'#include "{h}"\n' for h in sorted(os.listdir(INCLUDE)) if h.endswith(".h"))
    c.write_text(incs + "int main(void){mp_result r; (void)r; return (int)sizeof(mp_plan_desc) == 0;}\n")
    p = subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                        "-c", str(c), "-o", str(tmp_path / "t.o")], capture_output=True, text=True)
    assert p.returncode == 0, p.stderr


def header_enum_values():
    """Every `MP_NAME = value` enumerator the headers declare."""
    vals = {}
    for h in sorted(os.listdir(INCLUDE)):
        if h.endswith(".h"):
            src = open(os.path.join(INCLUDE, h)).read()
            src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)   # comments mention values in prose
            src = re.sub(r"//[^\n]*", " ", src)
            for name, v in re.findall(r"\b(MP_[A-Z0-9_]+)\s*=\s*(-?\d+)", src):
                vals[name] = int(v)
    return vals


def test_binding_constants_match_header():
    """The binding's option, query, precision, stop-reason and status
    numbers are the header's (a renumbered or added enumerator must reach
    both sides)."""
    from paper_0809_1833_gb300 import binding as B
    hdr = header_enum_values()
    assert {"MP_OPT_BATCH_GRAM", "MP_OPT_BATCH_GRAM_BELOW", "MP_Q_BATCH_GRAM_BELOW", "MP_PREC_BF16"} <= set(hdr)
    checked = 0
    for name, v in hdr.items():
        if hasattr(B, name):
            assert getattr(B, name) == v, (name, getattr(B, name), v)
            checked += 1
    assert checked >= 40, checked
