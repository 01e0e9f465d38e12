"""Equations with general (dense) coefficients: Alg. 1 and its counterpart
for the d-term form.

The coefficients are reduced on the host (LAPACK through scipy): real Schur
forms A_mu = U_mu T_mu U_mu^T for the Laplace form; for the d-term form the
real generalized Schur form of every pair, A_mu = Q_mu S_mu Z_mu^T,
C_mu = Q_mu T_mu Z_mu^T (QZ).  The right-hand side is transformed on the GPU,
B~ = B x_mu U_mu^T (Q_mu^T), the (quasi-)triangular equation is solved by
tsylv_solve / gtsylv_solve, and the solution is transformed back,
X = X~ x_mu U_mu (Z_mu).  Because  X x_mu Q S Z^T = ((X x_mu Z^T) x_mu S) x_mu Q,
the d-term operator of X equals the triangular operator of X~ = X x_all Z^T
followed by x_all Q, which gives the two transforms.
"""
import ctypes

import numpy as np
import torch

from . import _lib


def transform(X, M, trans=None, Y=None, stream=None):
    """Y = X x_1 op(M_1) ... x_d op(M_d) on the GPU (tsylv_transform);
    op(M) = M^T where trans[mu] is true; an entry None of M skips its mode."""
    from . import TsylvError, _check_cuda, _dims, _stream, empty_fortran, fortran, is_fortran, workspace
    lib = _lib.load()
    X = fortran(X)
    d = X.dim()
    _check_cuda(X, *[m for m in M if m is not None])
    if Y is None:
        Y = empty_fortran(X.shape, X.device)
    elif not is_fortran(Y) or Y.dtype != torch.float64:
        raise ValueError("Y must be a float64 column-major tensor")
    Ms = [fortran(m) if m is not None else None for m in M]
    pm = (ctypes.c_void_p * d)(*[m.data_ptr() if m is not None else None for m in Ms])
    tr = (ctypes.c_int * d)(*[1 if (trans is not None and trans[mu]) else 0 for mu in range(d)])
    n = _dims(X.shape)
    work = workspace(lib.tsylv_transform_workspace_bytes(d, n), X.device)
    st = lib.tsylv_transform(d, n, pm, tr, X.data_ptr(), Y.data_ptr(), work.data_ptr(), work.numel(), _stream(stream))
    if st != 0:
        raise TsylvError(st, "tsylv_transform")
    return Y


def reduce_coefficients(A, C=None, device=None):
    """Host reduction of general coefficients (numpy arrays): Laplace form
    (C None): [(T, U)] with A = U T U^T; d-term form: [(S, T, Q, Z)] with
    A = Q S Z^T, C = Q T Z^T.  With a device, the factors come back as
    column-major device tensors, ready to be reused by solve_general."""
    import scipy.linalg as sl
    if C is None:
        out = []
        for a in A:
            T, U = sl.schur(np.asarray(a, dtype=np.float64), output="real")
            out.append((np.asfortranarray(T), np.asfortranarray(U)))
    else:
        out = []
        for a, c in zip(A, C):
            S, T, Q, Z = sl.qz(np.asarray(a, dtype=np.float64), np.asarray(c, dtype=np.float64), output="real")
            out.append((np.asfortranarray(S), np.asfortranarray(T), np.asfortranarray(Q), np.asfortranarray(Z)))
    if device is not None:
        out = [tuple(_to_dev(m, device) for m in r) for r in out]
    return out


def _to_dev(m, dev):
    if isinstance(m, torch.Tensor):
        return m
    return torch.from_numpy(np.ascontiguousarray(np.asarray(m).T)).to(dev).T  # column-major copy


def solve_general(A, B, C=None, *, X=None, reduced=None, **kw):
    """X with sum_mu X x_mu A_mu (x_{eta != mu} C_eta) = B for general square
    coefficients (device tensors A, C; host reduction, GPU transforms and
    triangular solve).  X: optional column-major float64 output tensor (the
    transformed right-hand side, the triangular solve and the transform back
    all happen in it, so repeated calls reuse one buffer and its captured
    schedules).  reduced: the output of reduce_coefficients, to reuse a
    reduction.  Keyword arguments go to the triangular solve (precision, ...)."""
    from . import gtsylv_solve, tsylv_solve
    dev = B.device
    if reduced is None:
        reduced = reduce_coefficients([a.detach().cpu().numpy() for a in A],
                                      None if C is None else [c.detach().cpu().numpy() for c in C])

    def to_dev(m):
        return _to_dev(m, dev)

    if C is None:
        T = [to_dev(t) for t, _ in reduced]
        U = [to_dev(u) for _, u in reduced]
        Xt = transform(B, U, trans=[True] * len(U), Y=X)
        Xt, st = tsylv_solve(T, Xt, X=Xt, **kw)
        return transform(Xt, U, Y=Xt), st
    S = [to_dev(r[0]) for r in reduced]
    Tm = [to_dev(r[1]) for r in reduced]
    Q = [to_dev(r[2]) for r in reduced]
    Z = [to_dev(r[3]) for r in reduced]
    Xt = transform(B, Q, trans=[True] * len(Q), Y=X)
    Xt, st = gtsylv_solve(S, Tm, Xt, X=Xt, **kw)
    return transform(Xt, Z, Y=Xt), st
