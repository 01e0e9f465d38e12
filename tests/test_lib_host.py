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
    return sorted(set(re.findall(r"\b((?:z?g?tsylv|gsylvten)_[a-z_]+)\s*\(", src)))


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
    assert o.wait_ms == 2000
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
    assert lib.tsylv_solve(6, n, null2, None, None, None, 0, ctypes.byref(o), None, None) == -1
    bad = (ctypes.c_int64 * 2)(4, -1)
    assert lib.tsylv_solve(2, bad, null2, None, None, None, 0, ctypes.byref(o), None, None) == -2
    assert lib.tsylv_solve(2, n, None, None, None, None, 0, ctypes.byref(o), None, None) == -3
    assert lib.tsylv_solve(2, n, null2, None, None, None, 0, ctypes.byref(o), None, None) == -3
    fake = (P * 2)(16, 16)
    assert lib.tsylv_solve(2, n, fake, None, None, None, 0, ctypes.byref(o), None, None) == -4
    assert lib.gtsylv_solve(2, n, fake, None, None, None, None, 0, ctypes.byref(o), None, None) == -4
    assert lib.tsylv_solve(2, n, fake, P(16), P(16), P(17), 1 << 30, ctypes.byref(o), None, None) == -6
    assert lib.tsylv_solve(2, n, fake, P(16), P(16), P(256), 16, ctypes.byref(o), None, None) == -7


def test_option_validation_without_gpu(lib):
    """Out-of-range options are refused with -8 (the opts argument) before any
    CUDA call; every documented value passes validation."""
    from paper_1905_09539_gb300 import _lib
    n = (ctypes.c_int64 * 2)(4, 4)
    P = ctypes.c_void_p
    fake = (P * 2)(16, 16)
    wb = 1 << 30

    def st(**kw):
        o = _lib.default_opts(**kw)
        return lib.tsylv_solve(2, n, fake, P(16), P(16), P(256), wb, ctypes.byref(o), None, None)

    for kw in ({"fuse_step": 4}, {"fuse_step": -1}, {"schedule": 2}, {"partition": 2}, {"resid_update": 2},
               {"precision": 9}, {"tol": 0.0}, {"split": -1}, {"max_refine": -1}, {"residual": 7},
               {"wait_ms": 0}, {"wait_ms": 600001}, {"nmin": -2}, {"fp64_update": 3}, {"fp64_update": -1}):
        assert st(**kw) == -8, kw
    for kw in ({"host_io": 1}, {"fuse_step": 1}, {"nmin": 17}, {"nmin": 1}, {"fp64_update": 2, "schedule": 1},
               {"precision": _lib.TSYLV_TF32_REFINED, "schedule": 1},
               {"precision": _lib.TSYLV_BF16_REFINED, "schedule": 1}, {"precision": _lib.TSYLV_DF64, "schedule": 1},
               {"precision": _lib.TSYLV_DF64, "fp64_update": 2}):
        assert st(**kw) == _lib.TSYLV_EUNSUPPORTED, kw
    assert st(precision=5) == -8


def test_noalloc_option_validation_without_gpu(lib):
    """tsylv_solve_noalloc checks its options as tsylv_solve does (-6, its
    opts argument, for a field out of range; TSYLV_EUNSUPPORTED for host_io or
    an nmin above the tile extent), refuses any precision but FP64 with -6, and
    event timing and autotuning (nmin -1) with TSYLV_EUNSUPPORTED -- all before
    any CUDA call."""
    from paper_1905_09539_gb300 import _lib
    n = (ctypes.c_int64 * 2)(4, 4)
    P = ctypes.c_void_p
    fake = (P * 2)(16, 16)

    def st(**kw):
        o = _lib.default_opts(**kw)
        return lib.tsylv_solve_noalloc(2, n, fake, P(16), P(16), ctypes.byref(o), None, None)

    for kw in ({"fuse_step": 4}, {"schedule": 2}, {"partition": 2}, {"resid_update": 2}, {"precision": 9},
               {"tol": 0.0}, {"split": -1}, {"max_refine": -1}, {"residual": 7}, {"timing": 2},
               {"wait_ms": 0}, {"precision": _lib.TSYLV_FP32_REFINED}):
        assert st(**kw) == -6, kw
    for kw in ({"host_io": 1}, {"nmin": 17}, {"nmin": -1}, {"timing": 1}):
        assert st(**kw) == _lib.TSYLV_EUNSUPPORTED, kw
    bad = (ctypes.c_int64 * 2)(4, 0)
    assert lib.tsylv_solve_noalloc(2, bad, fake, P(16), P(16), None, None, None) == -2
    assert lib.tsylv_solve_noalloc(6, n, fake, P(16), P(16), None, None, None) == -1
    assert lib.tsylv_solve_noalloc(2, n, None, P(16), P(16), None, None, None) == -3


def test_selftest_argument_check_without_gpu(lib):
    """The wait-timeout diagnostic refuses a limit outside 1 ms .. 10 s before any CUDA call."""
    assert lib.tsylv_selftest_wait_timeout(0, None) == -1
    assert lib.tsylv_selftest_wait_timeout(999_999, None) == -1
    assert lib.tsylv_selftest_wait_timeout(10_000_000_001, None) == -1


def test_transform_validation_without_gpu(lib):
    """tsylv_transform: bad arguments are refused with -i before any CUDA call."""
    P = ctypes.c_void_p
    n = (ctypes.c_int64 * 2)(4, 5)
    M = (P * 2)(16, 16)
    wb = lib.tsylv_transform_workspace_bytes(2, n)
    assert wb >= 4 * 5 * 8
    assert lib.tsylv_transform_workspace_bytes(0, n) == 0
    bad = (ctypes.c_int64 * 2)(4, 0)
    assert lib.tsylv_transform_workspace_bytes(2, bad) == 0
    assert lib.tsylv_transform(0, n, M, None, P(16), P(16), P(256), wb, None) == -1
    assert lib.tsylv_transform(2, bad, M, None, P(16), P(16), P(256), wb, None) == -2
    assert lib.tsylv_transform(2, n, None, None, P(16), P(16), P(256), wb, None) == -3
    assert lib.tsylv_transform(2, n, M, None, None, P(16), P(256), wb, None) == -5
    assert lib.tsylv_transform(2, n, M, None, P(16), None, P(256), wb, None) == -6
    assert lib.tsylv_transform(2, n, M, None, P(16), P(16), P(257), wb, None) == -7
    assert lib.tsylv_transform(2, n, M, None, P(16), P(16), P(256), wb - 1, None) == -8


def test_backward_workspace_and_validation(lib):
    from paper_1905_09539_gb300 import _lib
    o = _lib.default_opts()
    n = (ctypes.c_int64 * 3)(20, 16, 12)
    N = 20 * 16 * 12
    ws = lib.tsylv_workspace_bytes(3, n, 0, ctypes.byref(o))
    wb = lib.tsylv_backward_workspace_bytes(3, n, 0, ctypes.byref(o))
    wbg = lib.tsylv_backward_workspace_bytes(3, n, 1, ctypes.byref(o))
    assert wb >= ws + N * 8           # transposed solve + Lambda
    assert wbg >= wb + 2 * N * 8      # + two mode-product temporaries
    P = ctypes.c_void_p
    fake = (P * 3)(16, 16, 16)
    assert lib.tsylv_backward(0, n, fake, None, P(16), P(16), None, None, None, P(256), 1 << 30,
                              ctypes.byref(o), None, None) == -1
    assert lib.tsylv_backward(3, n, None, None, P(16), P(16), None, None, None, P(256), 1 << 30,
                              ctypes.byref(o), None, None) == -3
    assert lib.tsylv_backward(3, n, fake, None, None, P(16), None, None, None, P(256), 1 << 30,
                              ctypes.byref(o), None, None) == -5
    assert lib.tsylv_backward(3, n, fake, None, P(16), None, None, None, None, P(256), 1 << 30,
                              ctypes.byref(o), None, None) == -6
    assert lib.tsylv_backward(3, n, fake, None, P(16), P(16), None, None, None, P(257), 1 << 30,
                              ctypes.byref(o), None, None) == -10
    assert lib.tsylv_backward(3, n, fake, None, P(16), P(16), None, None, None, P(256), 16,
                              ctypes.byref(o), None, None) == -11


def test_batched_workspace_and_validation(lib):
    from paper_1905_09539_gb300 import _lib
    o = _lib.default_opts()
    count = 3
    d = (ctypes.c_int * count)(3, 3, 2)
    n = (ctypes.c_int64 * 8)(8, 48, 20, 33, 9, 17, 40, 40)
    w = lib.tsylv_batched_workspace_bytes(count, d, n, 0, ctypes.byref(o))
    wg = lib.tsylv_batched_workspace_bytes(count, d, n, 1, ctypes.byref(o))
    N = 8 * 48 * 20 + 33 * 9 * 17 + 40 * 40
    assert w >= N * 8 and wg > w
    bad = (ctypes.c_int64 * 8)(8, 48, 0, 33, 9, 17, 40, 40)
    assert lib.tsylv_batched_workspace_bytes(count, d, bad, 0, ctypes.byref(o)) == 0
    o32 = _lib.default_opts(precision=_lib.TSYLV_FP32_REFINED)
    # the refined batch needs one order d for all equations
    assert lib.tsylv_batched_workspace_bytes(count, d, n, 0, ctypes.byref(o32)) == 0
    d3 = (ctypes.c_int * 2)(3, 3)
    n3 = (ctypes.c_int64 * 6)(8, 48, 20, 33, 9, 17)
    o8 = _lib.default_opts(nmin=8)  # FP64 with the tile shape fixed (no tuning over smaller cutoffs)
    assert lib.tsylv_batched_workspace_bytes(2, d3, n3, 0, ctypes.byref(o32)) > \
        lib.tsylv_batched_workspace_bytes(2, d3, n3, 0, ctypes.byref(o8))
    # the default FP64 batch tunes the tile shape: its bound covers the smallest cutoff
    assert lib.tsylv_batched_workspace_bytes(2, d3, n3, 0, ctypes.byref(o)) > \
        lib.tsylv_batched_workspace_bytes(2, d3, n3, 0, ctypes.byref(o8))
    P = ctypes.c_void_p
    offA = (ctypes.c_int64 * 8)(*range(8))
    offX = (ctypes.c_int64 * 3)(0, 1, 2)
    per = (ctypes.c_int * count)()
    args = lambda **kw: [kw.get("count", count), kw.get("d", d), kw.get("n", n), kw.get("offA", offA),
                         kw.get("offX", offX), kw.get("A", P(256)), None, kw.get("B", P(256)),
                         kw.get("X", P(256)), kw.get("work", P(256)), kw.get("wb", 1 << 40), ctypes.byref(o), per,
                         None, None]
    assert lib.tsylv_solve_batched(*args(count=0)) == -1
    assert lib.tsylv_solve_batched(*args(d=None)) == -2
    assert lib.tsylv_solve_batched(*args(n=bad)) == -3
    assert lib.tsylv_solve_batched(*args(offA=None)) == -4
    assert lib.tsylv_solve_batched(*args(offX=None)) == -5
    assert lib.tsylv_solve_batched(*args(A=None)) == -6
    assert lib.tsylv_solve_batched(*args(B=None)) == -8
    assert lib.tsylv_solve_batched(*args(X=None)) == -9
    assert lib.tsylv_solve_batched(*args(work=P(300))) == -10
    assert lib.tsylv_solve_batched(*args(wb=16)) == -11


def test_generalized_d5_unsupported_without_gpu(lib):
    """The generalized form is built for d <= 4: a d = 5 call returns
    TSYLV_EUNSUPPORTED before any CUDA call (the Laplace form takes d = 5)."""
    from paper_1905_09539_gb300 import _lib
    n = (ctypes.c_int64 * 5)(4, 4, 4, 4, 4)
    P = ctypes.c_void_p
    fake = (P * 5)(16, 16, 16, 16, 16)
    o = _lib.default_opts()
    assert lib.gtsylv_solve(5, n, fake, fake, P(16), P(16), P(256), 1 << 30, ctypes.byref(o), None, None) == \
        _lib.TSYLV_EUNSUPPORTED
    assert lib.tsylv_workspace_bytes(5, n, 0, ctypes.byref(o)) > 4 ** 5 * 8


def test_two_term_validation_without_gpu(lib):
    """gsylvten_solve (Eq. (3.1)): bad arguments give -i, orders outside 2..4,
    precisions other than FP64, the wavefront schedule and autotuning give
    TSYLV_EUNSUPPORTED -- all before any CUDA call."""
    from paper_1905_09539_gb300 import _lib
    P = ctypes.c_void_p
    n = (ctypes.c_int64 * 3)(8, 8, 8)
    fake = (P * 3)(16, 16, 16)
    o = _lib.default_opts()
    wb = lib.gsylvten_workspace_bytes(3, n, ctypes.byref(o))
    assert wb > 8 ** 3 * 8
    assert lib.gsylvten_workspace_bytes(1, n, ctypes.byref(o)) == 0
    assert lib.gsylvten_solve(0, n, fake, P(16), P(16), P(16), P(256), wb, ctypes.byref(o), None, None) == -1
    assert lib.gsylvten_solve(3, n, None, P(16), P(16), P(16), P(256), wb, ctypes.byref(o), None, None) == -3
    assert lib.gsylvten_solve(3, n, fake, None, P(16), P(16), P(256), wb, ctypes.byref(o), None, None) == -4
    assert lib.gsylvten_solve(3, n, fake, P(16), None, P(16), P(256), wb, ctypes.byref(o), None, None) == -5
    assert lib.gsylvten_solve(3, n, fake, P(16), P(16), None, P(256), wb, ctypes.byref(o), None, None) == -6
    assert lib.gsylvten_solve(3, n, fake, P(16), P(16), P(16), P(257), wb, ctypes.byref(o), None, None) == -7
    assert lib.gsylvten_solve(3, n, fake, P(16), P(16), P(16), P(256), 16, ctypes.byref(o), None, None) == -8
    n1 = (ctypes.c_int64 * 1)(8)
    assert lib.gsylvten_solve(1, n1, fake, P(16), P(16), P(16), P(256), wb, ctypes.byref(o), None, None) == \
        _lib.TSYLV_EUNSUPPORTED
    for kw in ({"precision": _lib.TSYLV_FP32_REFINED}, {"schedule": 1}, {"nmin": -1}):
        ok = _lib.default_opts(**kw)
        assert lib.gsylvten_solve(3, n, fake, P(16), P(16), P(16), P(256), wb, ctypes.byref(ok), None, None) == \
            _lib.TSYLV_EUNSUPPORTED, kw
    bad = _lib.default_opts(wait_ms=0)
    assert lib.gsylvten_solve(3, n, fake, P(16), P(16), P(16), P(256), wb, ctypes.byref(bad), None, None) == -9


def test_complex_validation_without_gpu(lib):
    """ztsylv_solve / zgtsylv_solve: bad arguments give -i, d = 5, precisions
    other than FP64, the wavefront schedule and autotuning give
    TSYLV_EUNSUPPORTED -- all before any CUDA call."""
    from paper_1905_09539_gb300 import _lib
    P = ctypes.c_void_p
    n = (ctypes.c_int64 * 3)(8, 8, 8)
    fake = (P * 3)(16, 16, 16)
    o = _lib.default_opts()
    w = lib.ztsylv_workspace_bytes(3, n, 0, ctypes.byref(o))
    wg = lib.ztsylv_workspace_bytes(3, n, 1, ctypes.byref(o))
    assert w >= 8 ** 3 * 16 and wg > w
    assert w > lib.tsylv_workspace_bytes(3, n, 0, ctypes.byref(o))
    assert lib.ztsylv_workspace_bytes(0, n, 0, ctypes.byref(o)) == 0
    z = lib.ztsylv_solve
    zg = lib.zgtsylv_solve
    assert z(0, n, fake, P(16), P(16), P(256), w, ctypes.byref(o), None, None) == -1
    assert z(3, n, None, P(16), P(16), P(256), w, ctypes.byref(o), None, None) == -3
    assert z(3, n, fake, None, P(16), P(256), w, ctypes.byref(o), None, None) == -4
    assert z(3, n, fake, P(16), None, P(256), w, ctypes.byref(o), None, None) == -5
    assert z(3, n, fake, P(16), P(16), P(257), w, ctypes.byref(o), None, None) == -6
    assert z(3, n, fake, P(16), P(16), P(256), 16, ctypes.byref(o), None, None) == -7
    assert zg(3, n, fake, None, P(16), P(16), P(256), wg, ctypes.byref(o), None, None) == -4
    assert zg(3, n, fake, fake, None, P(16), P(256), wg, ctypes.byref(o), None, None) == -5
    assert zg(3, n, fake, fake, P(16), P(16), P(256), w if w < wg else 16, ctypes.byref(o), None, None) == -8
    n5 = (ctypes.c_int64 * 5)(4, 4, 4, 4, 4)
    f5 = (P * 5)(16, 16, 16, 16, 16)
    assert z(5, n5, f5, P(16), P(16), P(256), 1 << 30, ctypes.byref(o), None, None) == _lib.TSYLV_EUNSUPPORTED
    for kw in ({"precision": _lib.TSYLV_FP32_REFINED}, {"schedule": 1}, {"nmin": -1}):
        ok = _lib.default_opts(**kw)
        assert z(3, n, fake, P(16), P(16), P(256), 1 << 30, ctypes.byref(ok), None, None) == \
            _lib.TSYLV_EUNSUPPORTED, kw
    bad = _lib.default_opts(wait_ms=0)
    assert z(3, n, fake, P(16), P(16), P(256), 1 << 30, ctypes.byref(bad), None, None) == -8
    dm = _lib.default_opts(fp64_update=2)
    assert z(3, n, fake, P(16), P(16), P(256), 1 << 30, ctypes.byref(dm), None, None) == _lib.TSYLV_EUNSUPPORTED


def test_plan_validation_without_gpu(lib):
    """tsylv_plan_create / tsylv_plan_execute: bad arguments give -i and the
    requests a plan does not serve give TSYLV_EUNSUPPORTED, all before any
    CUDA call; destroying a null plan is a no-op."""
    from paper_1905_09539_gb300 import _lib
    P = ctypes.c_void_p
    n = (ctypes.c_int64 * 3)(8, 8, 8)
    fake = (P * 3)(16, 16, 16)
    o = _lib.default_opts()
    wb = lib.tsylv_workspace_bytes(3, n, 0, ctypes.byref(o))
    h = P()
    cr = lambda *a: lib.tsylv_plan_create(*a)
    assert cr(None, 3, n, fake, None, 0, P(256), wb, ctypes.byref(o), None) == -1
    assert cr(ctypes.byref(h), 0, n, fake, None, 0, P(256), wb, ctypes.byref(o), None) == -2
    bad = (ctypes.c_int64 * 3)(8, 0, 8)
    assert cr(ctypes.byref(h), 3, bad, fake, None, 0, P(256), wb, ctypes.byref(o), None) == -3
    assert cr(ctypes.byref(h), 3, n, None, None, 0, P(256), wb, ctypes.byref(o), None) == -4
    holes = (P * 3)(16, None, 16)
    assert cr(ctypes.byref(h), 3, n, fake, holes, 0, P(256), wb, ctypes.byref(o), None) == -5
    assert cr(ctypes.byref(h), 3, n, fake, None, 2, P(256), wb, ctypes.byref(o), None) == -6
    assert cr(ctypes.byref(h), 3, n, fake, None, 0, P(257), wb, ctypes.byref(o), None) == -7
    assert cr(ctypes.byref(h), 3, n, fake, None, 0, P(256), 16, ctypes.byref(o), None) == -8
    badopt = _lib.default_opts(wait_ms=0)
    assert cr(ctypes.byref(h), 3, n, fake, None, 0, P(256), wb, ctypes.byref(badopt), None) == -9
    for kw in ({"precision": _lib.TSYLV_FP32_REFINED}, {"nmin": -1}, {"timing": 1}, {"fp64_update": 2, "schedule": 1},
               {"precision": _lib.TSYLV_DF64, "schedule": 1}):
        ok = _lib.default_opts(**kw)
        assert cr(ctypes.byref(h), 3, n, fake, None, 0, P(256), 1 << 30, ctypes.byref(ok), None) == \
            _lib.TSYLV_EUNSUPPORTED, kw
    assert not h.value
    assert lib.tsylv_plan_execute(None, P(16), P(16), P(256), wb, None, None) == -1
    lib.tsylv_plan_destroy(None)
