"""The C-ABI library builds for sm_103a, loads without a GPU and exports every entry point
include/lasto_poisson.h declares (no compute calls here)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "lasto_poisson.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lasto_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_core_boundary():
    names = _declared()
    for core in ("lasto_poisson_create", "lasto_poisson_solve", "lasto_poisson_destroy", "lasto_poisson_last_error"):
        assert core in names


def test_library_exports_every_declared_symbol():
    from paper_0806_1723_gb300 import binding, build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(binding.EXPORTS) == _declared()
