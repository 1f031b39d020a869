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


def test_lr_stride_closed_forms():
    """Eq. 2, S ~ sqrt(k_DEM / k_LR), rounded down and at least 1 (host-only
    entry point: runs without a GPU)."""
    from paper_2512_09478_gb300 import build as B, kifmm
    B.build()
    kifmm._LIB = None
    from paper_2512_09478_gb300 import lr_stride, KifmmError
    assert lr_stride(1e6, 1.0) == 1000            # exact square
    assert lr_stride(4.0e8, 1.0e2) == 2000
    assert lr_stride(99.0, 1.0) == 9              # sqrt(99) = 9.95: rounded down
    assert lr_stride(1.0, 1.0) == 1
    assert lr_stride(1.0, 1e3) == 1               # long-range stiffer than contacts
    assert lr_stride(2.5e9, 0.1) == 158113        # floor(sqrt(2.5e10)) = 158113.88...
    # scale invariance: only the ratio matters
    assert lr_stride(3.0e12, 7.0e3) == lr_stride(3.0e6, 7.0e-3)
    for bad in ((0.0, 1.0), (1.0, 0.0), (-1.0, 1.0), (float("nan"), 1.0), (1.0, float("inf"))):
        with pytest.raises(KifmmError) as e:
            lr_stride(*bad)
        assert e.value.code == 1
