"""The C-ABI library builds, loads and exports every entry point include/asd.h declares
(no compute calls: runs without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "asd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_ \*]*?\b(asd_[a-z0-9_]+)\s*\(", src, re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    from paper_2308_07487_gb300 import build
    so = build.build()
    lib = ctypes.CDLL(so)
    names = declared_functions()
    assert "asd_pair_corr" in names and "asd_thermalize" in names and "asd_ll_integrate" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, f"not exported: {missing}"


def test_binding_declares_the_same_entry_points():
    from paper_2308_07487_gb300 import asd
    assert set(asd.exported_symbols()) == set(declared_functions())


def test_status_strings():
    from paper_2308_07487_gb300 import asd
    assert asd.strerror(0) == "ok"
    assert asd.strerror(-1).startswith("invalid argument")
