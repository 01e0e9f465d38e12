"""Plain CPU FP64 oracle for the triangular tensor Sylvester equation.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; the solver package never imports it.

The arithmetic lives in ``tsylv_oracle.c`` (plain C, double precision, written
from Sec. 2.1 / Alg. 2 and Sec. 3.1 of Chen & Kressner); this module only
compiles it with gcc and marshals numpy arrays through ctypes.

Tensors are numpy arrays whose memory is column-major with mode 1 fastest
(the index map Eq. (2.1)); pass ``np.asfortranarray`` data of shape
``(n1, ..., nd)``.  Matrices are ``(n, n)`` Fortran-ordered arrays.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tsylv_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force=False):
    """Compile the oracle shared library with gcc (no CUDA involved)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        # -std=c11 keeps a * b + c unfused (ISO C contraction rules) on every host
        subprocess.check_call(["gcc", "-O3", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i64p = ctypes.POINTER(ctypes.c_int64)
        lib.orc_apply.argtypes = [ctypes.c_int, i64p, P, P, P, P, ctypes.c_int]
        lib.orc_backsub.argtypes = [ctypes.c_int, i64p, P, P, P, ctypes.c_int]
        lib.orc_recursive.argtypes = [ctypes.c_int, i64p, P, P, P, ctypes.c_int64, ctypes.c_int]
        lib.orc_grad.argtypes = [ctypes.c_int, i64p, P, P, P, P, P, P]
        lib.orc_check_structure.argtypes = [ctypes.c_int, i64p, P]
        for f in (lib.orc_apply, lib.orc_backsub, lib.orc_recursive, lib.orc_grad, lib.orc_check_structure):
            f.restype = ctypes.c_int
        _lib = lib
    return _lib


class OracleError(RuntimeError):
    pass


def _mats(ms):
    """Keep Fortran copies alive and return (list, pointer array)."""
    if ms is None:
        return None, None
    ms = [np.asfortranarray(m, dtype=np.float64) for m in ms]
    arr = (ctypes.c_void_p * len(ms))(*[m.ctypes.data for m in ms])
    return ms, arr


def _dims(X):
    n = (ctypes.c_int64 * X.ndim)(*X.shape)
    return X.ndim, n


def _check(rc, what):
    if rc != 0:
        raise OracleError("%s failed with status %d" % (what, rc))


def apply(A, X, C=None, transpose=False):
    """Y = A(X): sum_mu X x_mu A_mu (x_{eta != mu} C_eta); transpose -> A^T."""
    X = np.asfortranarray(X, dtype=np.float64)
    Y = np.zeros_like(X, order="F")
    A_, pa = _mats(A)
    C_, pc = _mats(C)
    d, n = _dims(X)
    _check(_load().orc_apply(d, n, pa, pc, X.ctypes.data, Y.ctypes.data, int(transpose)), "orc_apply")
    return Y


def solve_backsub(A, B, C=None, transpose=False):
    """O-A: element back-substitution over the coupled diagonal groups."""
    X = np.array(B, dtype=np.float64, order="F", copy=True)
    A_, pa = _mats(A)
    C_, pc = _mats(C)
    d, n = _dims(X)
    _check(_load().orc_backsub(d, n, pa, pc, X.ctypes.data, int(transpose)), "orc_backsub")
    return X


def solve_recursive(A, B, C=None, nmin=4, transpose=False):
    """O-B: Alg. 2 recursion (Laplace form) / its d-term generalized analogue;
    transpose=True solves A^T(X) = B with the reversed recursion order."""
    X = np.array(B, dtype=np.float64, order="F", copy=True)
    A_, pa = _mats(A)
    C_, pc = _mats(C)
    d, n = _dims(X)
    _check(_load().orc_recursive(d, n, pa, pc, X.ctypes.data, int(nmin), 1 if transpose else 0), "orc_recursive")
    return X


def grad(A, X, Lam, C=None, want_dC=True):
    """(dA list, dC list or None) of a scalar loss, given X and Lambda = A^{-T}(dL/dX)."""
    X = np.asfortranarray(X, dtype=np.float64)
    Lam = np.asfortranarray(Lam, dtype=np.float64)
    A_, pa = _mats(A)
    C_, pc = _mats(C)
    d, n = _dims(X)
    dA = [np.zeros((m, m), order="F") for m in X.shape]
    pdA = (ctypes.c_void_p * d)(*[g.ctypes.data for g in dA])
    dC = None
    pdC = None
    if C is not None and want_dC:
        dC = [np.zeros((m, m), order="F") for m in X.shape]
        pdC = (ctypes.c_void_p * d)(*[g.ctypes.data for g in dC])
    _check(_load().orc_grad(d, n, pa, pc, X.ctypes.data, Lam.ctypes.data, pdA, pdC), "orc_grad")
    return dA, dC


def solve_dense(A, B, C=None):
    """General (dense, not triangular) coefficients, small sizes only: the
    assembled operator of Eq. (1.4) -- sum over mu of the Kronecker product
    with A_mu in position mu (mode 1 rightmost, column-major vec) and the
    identity, or C_eta for the d-term form, in every other position -- solved
    by LAPACK (numpy.linalg.solve).  This is the plain definition of what
    Alg. 1 computes (Schur reduction, triangular solve, back-transformation)."""
    from functools import reduce
    d = len(A)
    shape = tuple(int(a.shape[0]) for a in A)
    N = int(np.prod(shape))
    M = np.zeros((N, N))
    for mu in range(d):
        facs = [np.asarray(A[eta], dtype=np.float64) if eta == mu else
                (np.eye(shape[eta]) if C is None else np.asarray(C[eta], dtype=np.float64)) for eta in range(d)]
        M += reduce(np.kron, facs[::-1])
    x = np.linalg.solve(M, np.asarray(B, dtype=np.float64).reshape(-1, order="F"))
    return np.asfortranarray(x.reshape(shape, order="F"))


def check_structure(A, shape):
    A_, pa = _mats(A)
    n = (ctypes.c_int64 * len(shape))(*shape)
    return _load().orc_check_structure(len(shape), n, pa)
