"""The C-ABI library builds, loads and exports every symbol the header
declares (no GPU needed: nothing here calls into CUDA)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "wt.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(wt_[A-Za-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2605_13987_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("wt_create", "wt_add_columns", "wt_fit", "wt_relax", "wt_extend", "wt_sample_H", "wt_eq1",
                 "wt_last_error", "wt_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_the_header(lib):
    from paper_2605_13987_gb300 import _binding
    assert set(declared_functions()) == set(_binding.SIGNATURES)
    _binding.load_library()


def test_null_handle_calls_fail_cleanly(lib):
    """Entry points reject a NULL context without touching the GPU."""
    from paper_2605_13987_gb300 import _binding as B
    L = B.load_library()
    assert L.wt_fit(None, None, None) == B.WT_ERR_ARG
    assert L.wt_relax(None, None, 0) == B.WT_ERR_ARG
    assert L.wt_extend(None, 0, None, 0, None) == B.WT_ERR_ARG
    L.wt_destroy(None)


def test_grid_checks_come_before_any_cuda_call(lib):
    """wt_create rejects a non-mirror z boundary and odd lateral sizes on the host."""
    from paper_2605_13987_gb300 import _binding as B
    L = B.load_library()
    ctx = ctypes.c_void_p()
    g = B.wt_grid(55e-6, 55e-6, 100e-6, 8, 8, 16, 5.7, 1)
    assert L.wt_create(ctypes.byref(ctx), ctypes.byref(g), 0) == B.WT_ERR_UNSUPPORTED
    assert ctx.value is None
    g = B.wt_grid(55e-6, 55e-6, 100e-6, 9, 8, 16, 5.7, B.WT_Z_MIRROR)
    assert L.wt_create(ctypes.byref(ctx), ctypes.byref(g), 0) == B.WT_ERR_ARG


def undocumented_prototypes(text):
    """Prototypes whose block of contiguous lines (typedefs, macros, other
    prototypes of a group) does not start right below a comment."""
    lines = text.splitlines()
    proto = re.compile(r"^(wt_status|const char\*|void)\s+(wt_[A-Za-z_0-9]+)\s*\(")
    bad = []
    for k, line in enumerate(lines):
        m = proto.match(line)
        if not m:
            continue
        j = k - 1
        while j >= 0 and lines[j].strip() and not lines[j].strip().endswith("*/"):
            j -= 1
        if j < 0 or not lines[j].strip():
            bad.append(m.group(2))
    return bad


def test_undocumented_prototypes_are_found():
    assert undocumented_prototypes("/* doc */\nwt_status wt_a(int x);\n\nint y;\nwt_status wt_b(int y);\n") == ["wt_b"]
    assert undocumented_prototypes("/* doc */\ntypedef struct {\n    int a;\n} t;\nwt_status wt_c(t* x);\n") == []


def test_every_entry_point_is_documented():
    """Each prototype (or group of prototypes) of the header sits directly
    below a comment that states what the call computes."""
    assert not undocumented_prototypes(open(HEADER).read())
