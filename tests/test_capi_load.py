"""The C-ABI library builds for sm_103a, loads, and exports every function that
include/gbtraffic.h declares (no device calls: runs without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(sim_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("sim_create", "sim_route", "sim_step", "sim_read_state", "sim_destroy"):
        assert must in names


def test_library_loads_and_exports_every_declared_symbol():
    from paper_1807_01148_gb300 import build
    so = build.build()
    lib = ctypes.CDLL(so)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, f"not exported: {missing}"


def test_binding_covers_the_exports():
    from paper_1807_01148_gb300 import gbtraffic
    assert set(gbtraffic.EXPORTS) <= set(declared_functions())
