"""The C-ABI library builds for sm_103a, loads, and exports every entry point include/osam.h declares
(no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

from paper_2511_20687_gb300 import build_lib, osam

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            names += re.findall(r"^OSAM_API\s+[\w\s\*]+?\b(\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    build_lib.build()
    lib = ctypes.CDLL(build_lib.LIB)
    names = declared_symbols()
    assert "schwarz_init" in names and "opinf_fit" in names and len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert set(osam.EXPORTED) == set(names)


def test_binding_loads():
    build_lib.build()
    L = osam.load()
    assert L.osam_last_error(None) is not None
