"""The C-ABI library loads and exports every entry point include/kifmm.h
declares (no compute calls: runs without a GPU)."""
import ctypes
import os
import re

import numpy as np
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


def test_host_side_argument_checks():
    """Argument errors are reported before any CUDA call, so they hold without
    a GPU: plan descriptors out of range, null plans and pointers, a skin
    outside [0, 1], unknown list kinds, and the status strings."""
    import ctypes as C
    from paper_2512_09478_gb300 import build as B, kifmm
    lib = C.CDLL(B.build())
    kifmm._LIB = None
    P = C.c_void_p
    lib.kifmm_plan_create.argtypes = [C.POINTER(kifmm.PlanDesc), C.POINTER(P)]
    lib.kifmm_status_string.restype = C.c_char_p
    lib.kifmm_status_string.argtypes = [C.c_int]

    def desc(**kw):
        d = dict(p=6, leaf_cap=64, max_depth=20, precision=kifmm.PRECISIONS["mixed_fp16"], coef=1.0,
                 n_max=1000, n_systems_max=1, dtype=0, pinv_eps=0.0, autotune=0, direct_max=0, m2l_eps=0.0)
        d.update(kw)
        return kifmm.PlanDesc(**d)

    bad = [dict(p=1), dict(p=11), dict(leaf_cap=0), dict(max_depth=0), dict(max_depth=21), dict(precision=7),
           dict(n_max=0), dict(n_systems_max=0), dict(dtype=2), dict(pinv_eps=-1.0), dict(pinv_eps=1.0),
           dict(m2l_eps=-1e-5), dict(m2l_eps=1.0), dict(m2l_eps=float("nan")),
           dict(m2l_eps=1e-5, precision=kifmm.PRECISIONS["fp32"]),
           dict(m2l_eps=1e-5, precision=kifmm.PRECISIONS["fp64"]), dict(reuse_lists=2), dict(reuse_lists=-1)]
    for kw in bad:
        h = P()
        d = desc(**kw)
        assert lib.kifmm_plan_create(C.byref(d), C.byref(h)) == 1, kw
        assert not h.value
    assert lib.kifmm_plan_create(None, None) == 1
    null = P()
    buf = (C.c_double * 8)()
    for name, args in [("kifmm_plan_destroy", [null]),
                       ("kifmm_evaluate", [null, None, None, None, None]),
                       ("kifmm_update_sources", [null, buf, buf, None]),
                       ("kifmm_refresh_sources", [null, buf, buf, C.c_double(0.05), None, None]),
                       ("kifmm_backward", [null, buf, buf, None, None, None]),
                       ("kifmm_get_device_status", [null, None]),
                       ("kifmm_profile_enable", [null, 1]),
                       ("kifmm_tree_info", [null, None]),
                       ("kifmm_copy_list", [null, 0, buf, None]),
                       ("kifmm_set_m2l_tuning", [null, 2, 1, 4]),
                       ("kifmm_set_m2l_wait_bound", [null, C.c_int64(1)])]:
        assert getattr(lib, name)(*args) == 1, name
    names = {k: lib.kifmm_status_string(k).decode() for k in range(7)}
    assert names[0] == "ok" and names[1] == "invalid argument" and names[6] == "call out of order"
    assert len(set(names.values())) == 7
    assert lib.kifmm_status_string(99).decode() == "unknown status"


def test_far_image_operator_matches_the_oracle():
    """The library's host-side far-image operator (C++, FP64) against the
    oracle's own (numpy): the same definition, written twice, at p = 3 and 4
    and two cell sides; it also scales as 1 / cell (the kernel's degree)."""
    from paper_2512_09478_gb300 import build as B, kifmm
    from oracle import oracle as O
    B.build()
    kifmm._LIB = None
    for p in (3, 4):
        for L in (1.0, 2.5):
            T = kifmm.far_image_operator(p, L)
            To = O.far_image_operator(p, L)
            assert np.abs(T - To).max() <= 1e-12 * np.abs(To).max(), (p, L)
    T1, T3 = kifmm.far_image_operator(4, 1.0), kifmm.far_image_operator(4, 3.0)
    assert np.abs(T3 - T1 / 3.0).max() <= 1e-12 * np.abs(T1).max()
    from paper_2512_09478_gb300 import KifmmError
    for bad in ((1, 1.0), (4, 0.0), (4, float("inf"))):
        with pytest.raises(KifmmError):
            kifmm.far_image_operator(*bad)
