"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every symbol the header declares, and the pure-host entry points (defaults,
status strings, workspace queries, argument validation) behave."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1905_09539_gb300 import _lib
    if not os.path.exists(_lib.LIB_PATH):
        from paper_1905_09539_gb300 import build
        build.build()
    return _lib.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "tsylv.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b((?:g?tsylv)_[a-z_]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 12
    for name in names:
        assert hasattr(lib, name), name
    from paper_1905_09539_gb300 import _lib
    assert set(_lib.EXPORTS) <= set(names)


def test_defaults_and_status(lib):
    from paper_1905_09539_gb300 import _lib
    o = _lib.default_opts()
    assert o.precision == 0 and o.use_graph == 1 and abs(o.tol - 1e-12) < 1e-20 and o.max_refine == 10
    for s in range(0, 7):
        assert len(_lib.status_string(s)) > 0
    assert "argument" in _lib.status_string(-3)


def test_workspace_queries(lib):
    from paper_1905_09539_gb300 import _lib
    o = _lib.default_opts()
    n = (ctypes.c_int64 * 3)(64, 64, 64)
    w = lib.tsylv_workspace_bytes(3, n, 0, ctypes.byref(o))
    wg = lib.tsylv_workspace_bytes(3, n, 1, ctypes.byref(o))
    assert w >= 64 ** 3 * 8 and wg > w
    assert lib.tsylv_workspace_bytes(0, n, 0, ctypes.byref(o)) == 0
    bad = (ctypes.c_int64 * 3)(64, 0, 64)
    assert lib.tsylv_workspace_bytes(3, bad, 0, ctypes.byref(o)) == 0


def test_argument_validation_without_gpu(lib):
    from paper_1905_09539_gb300 import _lib
    o = _lib.default_opts()
    n = (ctypes.c_int64 * 2)(4, 4)
    P = ctypes.c_void_p
    null2 = (P * 2)(None, None)
    # d out of range -> -1, before any CUDA call
    assert lib.tsylv_solve(0, n, null2, None, None, None, 0, ctypes.byref(o), None, None) == -1
    assert lib.tsylv_solve(5, n, null2, None, None, None, 0, ctypes.byref(o), None, None) == -1
    bad = (ctypes.c_int64 * 2)(4, -1)
    assert lib.tsylv_solve(2, bad, null2, None, None, None, 0, ctypes.byref(o), None, None) == -2
    assert lib.tsylv_solve(2, n, None, None, None, None, 0, ctypes.byref(o), None, None) == -3
    assert lib.tsylv_solve(2, n, null2, None, None, None, 0, ctypes.byref(o), None, None) == -3
    fake = (P * 2)(16, 16)
    assert lib.tsylv_solve(2, n, fake, None, None, None, 0, ctypes.byref(o), None, None) == -4
    assert lib.gtsylv_solve(2, n, fake, None, None, None, None, 0, ctypes.byref(o), None, None) == -4
    assert lib.tsylv_solve(2, n, fake, P(16), P(16), P(17), 1 << 30, ctypes.byref(o), None, None) == -6
    assert lib.tsylv_solve(2, n, fake, P(16), P(16), P(256), 16, ctypes.byref(o), None, None) == -7
