"""GPU test of tsylv_solve_noalloc, the entry point for callers that cannot
allocate device memory when they solve (their own allocator owns the device,
or cudaMalloc's latency and synchronisation are not acceptable in their loop).

Every call goes through the C ABI.  Each problem is solved twice in a row by
the entry point, and both results are compared with that of tsylv_solve (the
workspace-based entry point) on the same inputs, within the FP64 parity
tolerance of the other GPU tests.  A call that leaves an error status in the
shared array (a singular problem) is followed by a good call, which must
return TSYLV_OK and the right solution.  The file sorts last so that a run
stopping at the first failure has run every other test before it; it passes
alone and after the others.
"""
import ctypes

import numpy as np
import pytest

import synthetic

pytestmark = pytest.mark.gpu
TOL = 1e-11


def _dev(a):
    import torch
    a = np.asfortranarray(a, dtype=np.float64)
    t = torch.from_numpy(a)
    out = torch.empty_strided(t.shape, t.stride(), dtype=torch.float64, device="cuda")
    out.copy_(t)
    return out


def _host(t):
    return np.asfortranarray(t.detach().cpu().numpy())


def _call_noalloc(lib, A, B, X, stream):
    d = B.dim()
    n = (ctypes.c_int64 * d)(*B.shape)
    pa = (ctypes.c_void_p * d)(*[a.data_ptr() for a in A])
    from paper_1905_09539_gb300 import _lib
    info = _lib.Info()
    st = lib.tsylv_solve_noalloc(d, n, pa, B.data_ptr(), X.data_ptr(), None, ctypes.byref(info),
                                 ctypes.c_void_p(stream.cuda_stream))
    return st, info


def _close(Xn, Xr):
    return (np.linalg.norm(Xn - Xr) / np.linalg.norm(Xr) <= TOL and
            np.max(np.abs(Xn - Xr)) / np.max(np.abs(Xr)) <= TOL)


def test_noalloc_matches_workspace_solve_twice():
    import torch
    import paper_1905_09539_gb300 as ts
    from paper_1905_09539_gb300 import _lib
    lib = _lib.load()
    stream = torch.cuda.current_stream()
    for seed, shape in ((21, (40, 33, 24)), (22, (64, 64, 64))):
        p = synthetic.problem(seed, shape, force_blocks=[[n // 2 - 1] for n in shape])
        A = [_dev(a) for a in p["A"]]
        B = _dev(p["B"])
        X_ref, st = ts.tsylv_solve(A, B)
        assert st == 0
        Xr = _host(X_ref)
        for _ in range(2):  # the second call finds the first call's contents in the array
            X = ts.empty_fortran(shape, B.device)
            X.fill_(float("nan"))
            st, info = _call_noalloc(lib, A, B, X, stream)
            assert st == 0, _lib.last_error()
            assert info.tiles > 0
            assert _close(_host(X), Xr)


def test_noalloc_good_call_after_failing_call():
    """A singular problem leaves TSYLV_ESINGULAR in the shared status word;
    the next call clears it and solves its own problem correctly."""
    import torch
    import paper_1905_09539_gb300 as ts
    from paper_1905_09539_gb300 import _lib
    lib = _lib.load()
    stream = torch.cuda.current_stream()
    shape = (24, 20, 16)
    p = synthetic.problem(5, shape)
    As = [np.triu(a.copy()) for a in p["A"]]
    for a in As:
        np.fill_diagonal(a, 1.0)
    As[0][0, 0] = -2.0  # a_1,00 + a_2,jj + a_3,kk = 0 for every (j, k)
    Bs = _dev(p["B"])
    X = ts.empty_fortran(shape, Bs.device)
    st, _ = _call_noalloc(lib, [_dev(a) for a in As], Bs, X, stream)
    assert st == _lib.TSYLV_ESINGULAR
    q = synthetic.problem(6, shape, force_blocks=[[7], [9], [3]])
    A = [_dev(a) for a in q["A"]]
    B = _dev(q["B"])
    X_ref, st = ts.tsylv_solve(A, B)
    assert st == 0
    X = ts.empty_fortran(shape, B.device)
    st, _ = _call_noalloc(lib, A, B, X, stream)
    assert st == _lib.TSYLV_OK, _lib.last_error()
    assert _close(_host(X), _host(X_ref))


def test_noalloc_rejects_oversized_problem():
    import torch
    from paper_1905_09539_gb300 import _lib
    lib = _lib.load()
    stream = torch.cuda.current_stream()
    d = 3
    n = (ctypes.c_int64 * d)(256, 256, 256)
    fake = ctypes.c_void_p(256)
    pa = (ctypes.c_void_p * d)(256, 256, 256)
    st = lib.tsylv_solve_noalloc(d, n, pa, fake, fake, None, None, ctypes.c_void_p(stream.cuda_stream))
    assert st == _lib.TSYLV_ESCRATCH
    assert "32 MiB" in _lib.last_error()
