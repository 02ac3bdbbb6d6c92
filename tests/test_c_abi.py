"""The C-ABI library loads (no GPU needed) and exports every entry point
that include/*.h declares; the Python binding declares the same names."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(pot3d_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1709_01126_gb300 import _build

    path = _build.build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    names = declared_functions()
    for n in ("pot3d_plan", "pot3d_solve", "pot3d_field", "pot3d_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    from paper_1709_01126_gb300 import pot3d

    assert set(pot3d.EXPORTS) == set(declared_functions())


def test_strerror_and_errors_without_gpu(lib):
    lib.pot3d_strerror.restype = ctypes.c_char_p
    assert lib.pot3d_strerror(0) == b"ok"
    assert b"breakdown" in lib.pot3d_strerror(-5)
    # a NULL plan is rejected before any CUDA call
    lib.pot3d_solve.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                                ctypes.c_void_p, ctypes.c_void_p]
    assert lib.pot3d_solve(None, None, 1e-10, None, None) == -1
    assert lib.pot3d_last_error() == -1


def test_selftest_wait_validates_before_any_cuda_call(lib):
    lib.pot3d_selftest_wait.argtypes = [ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p]
    st = ctypes.c_int(7)
    for limit in (0.0, -1.0, 11.0, float("nan")):
        assert lib.pot3d_selftest_wait(limit, ctypes.byref(st), None) == -1
    assert lib.pot3d_selftest_wait(0.1, None, None) == -1
    assert st.value == 7
