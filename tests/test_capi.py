"""Host-side checks of the C ABI: the library loads, exports every entry point
that include/st.h declares, and rejects bad arguments before touching a GPU."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1908_06097_gb300 import build, st

    build.build()
    return st.load()


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(st_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 18
    for n in names:
        assert hasattr(lib, n), n


def test_binding_lists_every_export():
    from paper_1908_06097_gb300 import st

    assert set(st.EXPORTS) <= set(declared_functions())


def test_argument_errors_without_gpu(lib):
    from paper_1908_06097_gb300 import st

    h = ctypes.c_void_p()
    assert lib.st_plan_create(None, 10, st._Grid(0, 11), 1, None) == st.ST_ERR_ARG
    assert lib.st_plan_create(ctypes.byref(h), 0, st._Grid(0, 1), 1, None) == st.ST_ERR_ARG
    assert "T=0" in st.last_error()
    assert lib.st_plan_create(ctypes.byref(h), 10, st._Grid(0, 5), 1, None) == st.ST_ERR_ARG
    assert "N >= T+1" in st.last_error()
    assert lib.st_plan_create(ctypes.byref(h), 10, st._Grid(1, 3), 1, None) == st.ST_ERR_ARG
    assert lib.st_plan_create(ctypes.byref(h), 10, st._Grid(7, 11), 1, None) == st.ST_ERR_ARG
    assert lib.st_plan_create(ctypes.byref(h), 10, st._Grid(0, 11), 0, None) == st.ST_ERR_ARG
    bad = st._Opts(9, 1.0, 0, None)
    assert lib.st_plan_create(ctypes.byref(h), 10, st._Grid(0, 11), 1, ctypes.byref(bad)) == st.ST_ERR_ARG
    neg = st._Opts(0, -1.0, 0, None)
    assert lib.st_plan_create(ctypes.byref(h), 10, st._Grid(0, 11), 1, ctypes.byref(neg)) == st.ST_ERR_ARG
    assert h.value is None
    # NULL plans are rejected by every call; destroy is NULL-safe
    for name in ["st_inv_transform", "st_dir_transform", "st_inv_adjoint", "st_dir_adjoint"]:
        assert getattr(lib, name)(None, None, None, None) == st.ST_ERR_ARG
    assert lib.st_inv_transform_uv(None, None, None, None, None, None) == st.ST_ERR_ARG
    assert lib.st_plan_destroy(None) == st.ST_OK
    assert lib.st_group_destroy(None) == st.ST_OK
    assert lib.st_sync_status(None) == st.ST_ERR_ARG
    assert lib.st_group_create(ctypes.byref(h), None, 0) == st.ST_ERR_ARG


def test_missing_library_fails_loudly(tmp_path):
    from paper_1908_06097_gb300 import st

    with pytest.raises(ImportError):
        st.load(str(tmp_path / "nope.so"))
