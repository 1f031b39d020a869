"""The C-ABI library loads and exports every entry point include/kifmm.h
declares (no compute calls: runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            names += re.findall(r"^\s*(?:kifmm_status|const char \*)\s*(kifmm_\w+)\s*\(", src, re.M)
    return sorted(set(names))


def test_header_declares_entry_points():
    names = _declared()
    for n in ("kifmm_plan_create", "kifmm_set_sources", "kifmm_evaluate", "kifmm_clump_reduce", "kifmm_backward"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2512_09478_gb300 import build as B
    lib_path = B.build()
    lib = ctypes.CDLL(lib_path)
    for n in _declared():
        assert hasattr(lib, n), n


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_2512_09478_gb300 import kifmm
    with pytest.raises(FileNotFoundError):
        kifmm._LIB = None
        kifmm.load(str(tmp_path / "missing.so"))
    kifmm._LIB = None
