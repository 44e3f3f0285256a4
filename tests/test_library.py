"""The C-ABI library builds, loads and exports every symbol include/dbl.h
declares (no GPU needed: nothing here computes)."""
import os
import re

import pytest

import paper_2101_09441_gb300 as dbl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(dbl\w+)\s*\(", src)
    return sorted(set(n for n in names if not n.endswith("_fn")))


@pytest.fixture(scope="module")
def lib():
    dbl.build()
    return dbl.lib()


def test_every_declared_symbol_is_exported(lib):
    declared = _declared()
    assert "dbl_build" in declared and "dbl_query" in declared
    for name in declared:
        assert hasattr(lib, name), name


def test_binding_lists_match_header():
    assert set(dbl.EXPORTS) <= set(_declared())


def test_default_options_and_errors_without_gpu(lib):
    import ctypes
    opt = dbl._Options()
    lib.dbl_default_options(ctypes.byref(opt))
    assert opt.team == 1 and opt.bfs_words == 16 and opt.flags == 0
    # invalid arguments are rejected before any device work
    h = ctypes.c_void_p()
    assert lib.dbl_build(None, None, 64, None, None, 64, None, None, ctypes.byref(h)) == dbl.DBL_ERR_INVALID
    g = dbl._Graph(10, 0, 0, 0)
    assert lib.dbl_build(ctypes.byref(g), None, 64, None, None, 64, None, None, ctypes.byref(h)) == dbl.DBL_ERR_INVALID
    assert b"row_ptr" in lib.dbl_last_error(None)
    assert lib.dbl_query(None, None, None, 0, None, None, None) == dbl.DBL_ERR_INVALID


def test_option_checks_without_gpu(lib):
    """Options are validated before any device work: Table 3 ranking rule,
    leaf threshold, vertex capacity, team width; the newer entry points reject
    a NULL handle."""
    import ctypes
    g = dbl._Graph(10, 0, 16, 0)  # row_ptr is never dereferenced before the checks below
    h = ctypes.c_void_p()
    for field, value in (("landmark_rule", 4), ("landmark_rule", -1), ("leaf_r", -1),
                         ("vertex_capacity", 1 << 31), ("team", 3)):
        opt = dbl._Options()
        lib.dbl_default_options(ctypes.byref(opt))
        setattr(opt, field, value)
        st = lib.dbl_build(ctypes.byref(g), None, 64, None, None, 64, ctypes.byref(opt), None, ctypes.byref(h))
        assert st == dbl.DBL_ERR_INVALID, (field, value, st)
        assert not h.value
    first = ctypes.c_int32(0)
    assert lib.dbl_add_vertices(None, 1, ctypes.byref(first), None) == dbl.DBL_ERR_INVALID
    assert lib.dbl_set_schedule(None, 1, 1, 0) == dbl.DBL_ERR_INVALID
    assert lib.dbl_mlp_sync(None, None) == dbl.DBL_ERR_INVALID


def test_kernels_compiled_for_sm103a():
    from paper_2101_09441_gb300 import native_build
    assert "arch=compute_103a,code=sm_103a" in native_build.ARCH
