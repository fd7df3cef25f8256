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


def test_product_path_never_touches_the_oracle():
    """The library sources and the Python package import, link or name no part of oracle/ (the
    oracle is test infrastructure; only tests, smoke() and bench.py's CPU legs use it), and the CUDA
    sources include nothing from it."""
    import re
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    pkg = os.path.join(root, "paper_2511_20687_gb300")
    for dirpath, _, files in os.walk(pkg):
        if "_build" in dirpath or "__pycache__" in dirpath:
            continue
        for f in files:
            if not f.endswith((".py", ".cu", ".cuh", ".h", ".c", ".cpp")):
                continue
            text = open(os.path.join(dirpath, f)).read()
            assert not re.search(r"^\s*(from\s+oracle|import\s+oracle)", text, re.M), f
            assert "osam_oracle" not in text and "liboracle" not in text, f
    header = open(os.path.join(root, "include", "osam.h")).read()
    assert "oracle" not in header


def test_oracle_shares_no_code_with_the_library():
    """The oracle includes only the C standard library and imports neither the package nor its
    binding; the seeded workload generators reach it as plain arrays, not imports."""
    import re
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    c_src = open(os.path.join(root, "oracle", "osam_oracle.c")).read()
    includes = re.findall(r'#include\s*[<"]([^>"]+)[>"]', c_src)
    assert includes and all(i in ("math.h", "stdint.h", "stdlib.h", "string.h", "stdio.h") for i in includes), includes
    for f in ("fit.py", "oracle.py"):
        text = open(os.path.join(root, "oracle", f)).read()
        assert not re.search(r"^\s*(from|import)\s+paper_2511_20687_gb300", text, re.M), f
        assert "libosam" not in text, f
