"""GB300-native solver for triangular tensor Sylvester equations.

Thin Python binding over the C ABI of ``include/tsylv.h``: it only marshals
torch CUDA tensors (device memory, streams) into pointers; every step of the
solve runs in the library's sm_103a kernels.  There is no CPU path: if
``libtsylv.so`` has not been built, every call raises.

Tensor convention: a tensor argument has the mathematical shape
``(n_1, ..., n_d)`` and column-major memory (mode 1 fastest, the index map
Eq. (2.1) of Chen & Kressner); matrices are ``(n, n)`` column-major.  Use
:func:`fortran` to obtain that layout from any tensor.  Inputs in another
layout are copied into it first (marshalling only).
"""
import ctypes

import torch

from . import _lib
from ._lib import (TSYLV_BF16_REFINED, TSYLV_FP32_REFINED, TSYLV_FP64, TSYLV_RESID_DF64, TSYLV_RESID_FP64,
                   TSYLV_TF32_REFINED, TSYLV_DF64, Info, Opts, default_opts, load, status_string)

__all__ = ["tsylv_solve", "gtsylv_solve", "gsylvten_solve", "ztsylv_solve", "tsylv_solve_transposed", "gtsylv_solve_transposed",
           "tsylv_residual", "tsylv_backward", "tsylv_solve_batched", "BatchPools", "solve", "fortran", "TsylvError",
           "Opts", "Info", "default_opts", "TSYLV_FP64", "TSYLV_FP32_REFINED", "TSYLV_TF32_REFINED",
           "TSYLV_BF16_REFINED", "TSYLV_DF64", "TSYLV_RESID_DF64", "TSYLV_RESID_FP64", "workspace", "solve_general",
           "reduce_coefficients", "transform", "selftest_wait_timeout", "empty_fortran", "SolvePlan"]


class TsylvError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        msg = "%s: status %d (%s)" % (where, status, status_string(status))
        if status == _lib.TSYLV_ECUDA:
            msg += ": " + _lib.last_error()
        super().__init__(msg)


def is_fortran(t):
    d = t.dim()
    exp = 1
    for k in range(d):
        if t.shape[k] != 1 and t.stride(k) != exp:
            return False
        exp *= t.shape[k]
    return True


def fortran(t, dtype=torch.float64):
    """Same values, column-major memory (mode 1 fastest), float64, on t's device."""
    t = t.to(dtype)
    if is_fortran(t):
        return t
    d = t.dim()
    perm = list(range(d))[::-1]
    return t.permute(*perm).contiguous().permute(*perm)


def empty_fortran(shape, device, dtype=torch.float64):
    d = len(shape)
    perm = list(range(d))[::-1]
    return torch.empty(tuple(shape[::-1]), device=device, dtype=dtype).permute(*perm)


_ws = {}


def workspace(nbytes, device):
    """Grow-only device workspace (allocated by PyTorch, reused across calls)."""
    dev = torch.device(device)
    key = (dev.type, dev.index if dev.index is not None else torch.cuda.current_device())
    buf = _ws.get(key)
    if buf is None or buf.numel() < nbytes:
        buf = torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=dev)
        _ws[key] = buf
    return buf


def _check_cuda(*ts):
    for t in ts:
        if t is not None and not t.is_cuda:
            raise ValueError("expected CUDA tensors (the solver runs on the GPU only)")


def _mats(ms):
    ms = [fortran(m) for m in ms]
    arr = (ctypes.c_void_p * len(ms))(*[m.data_ptr() for m in ms])
    return ms, arr


def _dims(shape):
    return (ctypes.c_int64 * len(shape))(*[int(s) for s in shape])


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _opts(opts, kw):
    if opts is None:
        opts = default_opts(**kw)
    elif kw:
        for k, v in kw.items():
            setattr(opts, k, v)
    return opts


def _solve(fn, ws_fn, gen, transposed, A, C, B, X, opts, check, stream, info, kw):
    lib = load()
    _check_cuda(B, *A, *(C or []))
    o = _opts(opts, kw)
    B = fortran(B)
    d = B.dim()
    if X is None:
        X = empty_fortran(B.shape, B.device)
    elif not is_fortran(X) or X.dtype != torch.float64:
        raise ValueError("X must be a float64 column-major tensor (see fortran())")
    A_, pa = _mats(A)
    pc = None
    if gen:
        C_, pc = _mats(C)
    n = _dims(B.shape)
    nbytes = ws_fn(d, n, 1 if gen else 0, ctypes.byref(o))
    if nbytes == 0:
        raise ValueError("invalid problem shape %s" % (tuple(B.shape),))
    work = workspace(nbytes, B.device)
    inf = info if info is not None else Info()
    args = [d, n, pa] + ([pc] if gen else []) + [B.data_ptr(), X.data_ptr(), work.data_ptr(), work.numel(),
                                                 ctypes.byref(o), ctypes.byref(inf), _stream(stream)]
    st = fn(*args)
    if check and st != 0:
        raise TsylvError(st, fn.__name__)
    return X, st


def tsylv_solve(A, B, X=None, *, opts=None, check=True, stream=None, info=None, **kw):
    """X with sum_mu X x_mu A_mu = B (Eq. (2.2)); returns (X, status)."""
    lib = load()
    return _solve(lib.tsylv_solve, lib.tsylv_workspace_bytes, False, False, A, None, B, X, opts, check, stream,
                  info, kw)


def gtsylv_solve(A, C, B, X=None, *, opts=None, check=True, stream=None, info=None, **kw):
    """X with sum_mu X x_mu A_mu x_{eta != mu} C_eta = B; returns (X, status)."""
    lib = load()
    return _solve(lib.gtsylv_solve, lib.tsylv_workspace_bytes, True, False, A, C, B, X, opts, check, stream,
                  info, kw)


def gsylvten_solve(A, C, B, X=None, *, opts=None, check=True, stream=None, info=None, **kw):
    """X with X x_1 A_1 + X x_1 C x_2 A_2 ... x_d A_d = B (the paper's two-term
    form, Eq. (3.1)); C is one n_1 x n_1 upper triangular matrix.  Returns (X, status)."""
    lib = load()
    _check_cuda(B, C, *A)
    o = _opts(opts, kw)
    B = fortran(B)
    d = B.dim()
    if X is None:
        X = empty_fortran(B.shape, B.device)
    elif not is_fortran(X) or X.dtype != torch.float64:
        raise ValueError("X must be a float64 column-major tensor (see fortran())")
    A_, pa = _mats(A)
    C_ = fortran(C)
    n = _dims(B.shape)
    nbytes = lib.gsylvten_workspace_bytes(d, n, ctypes.byref(o))
    if nbytes == 0:
        raise ValueError("gsylvten_solve: invalid or unsupported shape %s (d = 2..4)" % (tuple(B.shape),))
    work = workspace(nbytes, B.device)
    inf = info if info is not None else Info()
    st = lib.gsylvten_solve(d, n, pa, C_.data_ptr(), B.data_ptr(), X.data_ptr(), work.data_ptr(), work.numel(),
                            ctypes.byref(o), ctypes.byref(inf), _stream(stream))
    if check and st != 0:
        raise TsylvError(st, "gsylvten_solve")
    return X, st


def ztsylv_solve(A, B, C=None, X=None, *, opts=None, check=True, stream=None, info=None, **kw):
    """Complex-triangular variant: X with sum_mu X x_mu A_mu = B (C None) or
    sum_mu X x_mu A_mu x_{eta != mu} C_eta = B, every tensor and matrix
    complex128 (A_mu, C_mu upper triangular).  Returns (X, status)."""
    lib = load()
    _check_cuda(B, *A, *(C or []))
    o = _opts(opts, kw)
    z = torch.complex128
    B = fortran(B, z)
    d = B.dim()
    if X is None:
        X = empty_fortran(B.shape, B.device, z)
    elif not is_fortran(X) or X.dtype != z:
        raise ValueError("X must be a complex128 column-major tensor")
    ms = [fortran(a, z) for a in A]
    pa = (ctypes.c_void_p * d)(*[m.data_ptr() for m in ms])
    gen = C is not None
    if gen:
        cs = [fortran(c, z) for c in C]
        pc = (ctypes.c_void_p * d)(*[m.data_ptr() for m in cs])
    n = _dims(B.shape)
    nbytes = lib.ztsylv_workspace_bytes(d, n, 1 if gen else 0, ctypes.byref(o))
    if nbytes == 0:
        raise ValueError("ztsylv_solve: invalid or unsupported shape %s (d = 1..4)" % (tuple(B.shape),))
    work = workspace(nbytes, B.device)
    inf = info if info is not None else Info()
    tail = [B.data_ptr(), X.data_ptr(), work.data_ptr(), work.numel(), ctypes.byref(o), ctypes.byref(inf),
            _stream(stream)]
    st = lib.zgtsylv_solve(d, n, pa, pc, *tail) if gen else lib.ztsylv_solve(d, n, pa, *tail)
    if check and st != 0:
        raise TsylvError(st, "ztsylv_solve")
    return X, st


class SolvePlan:
    """Repeated FP64 solves with fixed coefficients (tsylv_plan_*): the 2x2
    structure of the A_mu is read once here; solve() only enqueues work on
    the stream (no host synchronisation) and returns X and a device int32
    tensor that receives the execution's status code.  The coefficient
    tensors must stay alive (and keep their 2x2 structure) while the plan is
    used; their values may change between executions."""

    def __init__(self, A, C=None, *, transposed=False, opts=None, stream=None, **kw):
        lib = load()
        _check_cuda(*A, *(C or []))
        self._o = _opts(opts, kw)
        self._A, pa = _mats(A)
        self._C, pc = (None, None) if C is None else _mats(C)
        self.d = len(A)
        self.shape = tuple(int(a.shape[0]) for a in self._A)
        self.device = self._A[0].device
        n = _dims(self.shape)
        nbytes = lib.tsylv_workspace_bytes(self.d, n, 1 if C is not None else 0, ctypes.byref(self._o))
        if nbytes == 0:
            raise ValueError("SolvePlan: invalid or unsupported shape %s" % (self.shape,))
        self._work = torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=self.device)
        h = ctypes.c_void_p()
        st = lib.tsylv_plan_create(ctypes.byref(h), self.d, n, pa, pc, 1 if transposed else 0,
                                   self._work.data_ptr(), self._work.numel(), ctypes.byref(self._o), _stream(stream))
        if st != 0:
            raise TsylvError(st, "tsylv_plan_create")
        self._h = h

    def solve(self, B, X=None, status=None, *, stream=None):
        """Enqueue one solve of B (column-major float64, the plan's shape)."""
        lib = load()
        B = fortran(B)
        if tuple(B.shape) != self.shape:
            raise ValueError("B must have the plan's shape %s" % (self.shape,))
        if X is None:
            X = empty_fortran(B.shape, B.device)
        if status is None:
            status = torch.zeros(1, dtype=torch.int32, device=B.device)
        st = lib.tsylv_plan_execute(self._h, B.data_ptr(), X.data_ptr(), self._work.data_ptr(), self._work.numel(),
                                    status.data_ptr(), _stream(stream))
        if st != 0:
            raise TsylvError(st, "tsylv_plan_execute")
        return X, status

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().tsylv_plan_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tsylv_solve_transposed(A, G, L=None, *, opts=None, check=True, stream=None, info=None, **kw):
    """L with A^T(L) = G for the Laplace-form operator; returns (L, status)."""
    lib = load()
    return _solve(lib.tsylv_solve_transposed, lib.tsylv_workspace_bytes, False, True, A, None, G, L, opts, check,
                  stream, info, kw)


def gtsylv_solve_transposed(A, C, G, L=None, *, opts=None, check=True, stream=None, info=None, **kw):
    """L with A^T(L) = G for the generalized operator; returns (L, status)."""
    lib = load()
    return _solve(lib.gtsylv_solve_transposed, lib.tsylv_workspace_bytes, True, True, A, C, G, L, opts, check,
                  stream, info, kw)


def tsylv_residual(A, B, X, C=None, R=None, *, opts=None, check=True, stream=None, **kw):
    """R = B - A(X) and the relative residual ||R|| / (||A|| ||X||)."""
    lib = load()
    _check_cuda(B, X, *A, *(C or []))
    o = _opts(opts, kw)
    B = fortran(B)
    X = fortran(X)
    if R is None:
        R = empty_fortran(B.shape, B.device)
    A_, pa = _mats(A)
    pc = None
    if C is not None:
        C_, pc = _mats(C)
    n = _dims(B.shape)
    d = B.dim()
    work = workspace(lib.tsylv_residual_workspace_bytes(d, n, 1 if C is not None else 0), B.device)
    rel = ctypes.c_double(-1.0)
    st = lib.tsylv_residual(d, n, pa, pc, B.data_ptr(), X.data_ptr(), R.data_ptr(), ctypes.byref(rel),
                            work.data_ptr(), work.numel(), ctypes.byref(o), _stream(stream))
    if check and st != 0:
        raise TsylvError(st, "tsylv_residual")
    return R, rel.value, st


def _out_buffer(t, shape, device, what):
    if tuple(t.shape) != tuple(shape) or t.dtype != torch.float64 or t.device != torch.device(device) or \
            not is_fortran(t):
        raise ValueError("tsylv_backward: out %s must be a column-major float64 tensor of shape %s on %s"
                         % (what, tuple(shape), device))
    return t


def tsylv_backward(A, X, dX, C=None, *, want_dB=True, want_dA=True, want_dC=True, opts=None, check=True,
                   stream=None, info=None, out=None, **kw):
    """(dB, dA list, dC list) of a scalar loss with gradient dX at the solution X.

    out: optional (dB, dA list, dC list) of column-major float64 device tensors
    to write the requested gradients into (entries for gradients not requested
    may be None), so that repeated calls allocate nothing."""
    lib = load()
    _check_cuda(X, dX, *A, *(C or []))
    o = _opts(opts, kw)
    X = fortran(X)
    dX = fortran(dX)
    d = X.dim()
    A_, pa = _mats(A)
    pc = None
    gen = C is not None
    if gen:
        C_, pc = _mats(C)
    oB, oA, oC = out if out is not None else (None, None, None)
    if want_dB:
        dB = _out_buffer(oB, X.shape, X.device, "dB") if oB is not None else empty_fortran(X.shape, X.device)
    else:
        dB = None
    if want_dA:
        dA = [_out_buffer(t, (m, m), X.device, "dA") for t, m in zip(oA, X.shape)] if oA is not None else \
            [empty_fortran((m, m), X.device) for m in X.shape]
    else:
        dA = None
    if gen and want_dC:
        dC = [_out_buffer(t, (m, m), X.device, "dC") for t, m in zip(oC, X.shape)] if oC is not None else \
            [empty_fortran((m, m), X.device) for m in X.shape]
    else:
        dC = None
    pdA = (ctypes.c_void_p * d)(*[t.data_ptr() for t in dA]) if dA else None
    pdC = (ctypes.c_void_p * d)(*[t.data_ptr() for t in dC]) if dC else None
    n = _dims(X.shape)
    work = workspace(lib.tsylv_backward_workspace_bytes(d, n, 1 if gen else 0, ctypes.byref(o)), X.device)
    inf = info if info is not None else Info()
    st = lib.tsylv_backward(d, n, pa, pc, X.data_ptr(), dX.data_ptr(), dB.data_ptr() if dB is not None else None,
                            pdA, pdC, work.data_ptr(), work.numel(), ctypes.byref(o), ctypes.byref(inf),
                            _stream(stream))
    if check and st != 0:
        raise TsylvError(st, "tsylv_backward")
    return dB, dA, dC


def selftest_wait_timeout(timeout_s=0.05, stream=None):
    """Run the library's failure-path diagnostic (a solve whose first block is
    withheld, so that a bounded wait runs out); returns the status, which is
    TSYLV_ETIMEOUT when the path works."""
    lib = load()
    return lib.tsylv_selftest_wait_timeout(int(timeout_s * 1e9), _stream(stream))


from .autograd import solve  # noqa: E402
from .general import reduce_coefficients, solve_general, transform  # noqa: E402
from .batched import BatchPools, tsylv_solve_batched  # noqa: E402
