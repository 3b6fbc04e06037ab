"""The C ABI library loads and exports every entry point include/cpm.h
declares, and the Python binding carries the same names.  No compute call is
made (this runs without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "cpm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:cpm_status|void|const char\*|int64_t)\s+(\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_hot_path_calls():
    names = declared_functions()
    for n in ("cpm_band_build", "cpm_apply", "oras_setup", "oras_apply", "cpm_solve", "cpm_solve_adjoint"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2110_06322_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_uses_the_c_names():
    from paper_2110_06322_gb300 import cpm
    assert sorted(cpm.EXPORTED) == declared_functions()
