"""Plain CPU oracle of the complex-triangular variant (Sec. 2.4: every
coefficient reduced to complex Schur form, hence upper triangular; no 2x2
blocks): the Laplace form Eq. (2.2) and the d-term generalized form with
complex FP64 coefficients and tensors.

TEST INFRASTRUCTURE ONLY (imported by tests/), numpy complex128:

* apply(A, X, C): the operator by mode products (each term X x_mu A_mu, and
  for the d-term form x_{eta != mu} C_eta).
* assemble(A, C): the matrix of the operator (column-major vec, mode 1
  fastest: the Kronecker sums of Eq. (1.4)).
* solve_dense(A, B, C): the assembled system solved by LAPACK (small sizes).
* solve_recursive(A, B, C, nmin): Alg. 2 in the paper's order: split the
  largest mode (lowest on ties) at floor(m/2) -- triangular coefficients need
  no guard --, solve the trailing part, subtract its contribution through the
  off-diagonal coefficient block from the leading right-hand side (every term
  for the d-term form), solve the leading part; boxes of at most nmin per mode
  by the dense solve.
"""
from functools import reduce

import numpy as np


def _mode(X, M, mu):
    """X x_mu M: (X x_mu M)(.., i, ..) = sum_k M(i, k) X(.., k, ..)."""
    Y = np.tensordot(np.asarray(M), np.moveaxis(X, mu, 0), axes=(1, 0))
    return np.moveaxis(Y, 0, mu)


def _term(X, A, C, mu, block=None):
    """X x_mu A_mu (x_{eta != mu} C_eta for the d-term form); block replaces A_mu."""
    Y = _mode(X, A[mu] if block is None else block, mu)
    if C is not None:
        for eta in range(X.ndim):
            if eta != mu:
                Y = _mode(Y, C[eta], eta)
    return Y


def apply(A, X, C=None):
    X = np.asarray(X, dtype=np.complex128)
    return sum(_term(X, A, C, mu) for mu in range(X.ndim))


def assemble(A, C=None):
    d = len(A)
    n = [a.shape[0] for a in A]
    total = 0
    for mu in range(d):
        facs = [np.asarray(A[eta]) if eta == mu else (np.asarray(C[eta]) if C is not None else np.eye(n[eta]))
                for eta in range(d)]
        total = total + reduce(np.kron, facs[::-1])
    return total


def solve_dense(A, B, C=None):
    B = np.asarray(B, dtype=np.complex128)
    x = np.linalg.solve(assemble(A, C), B.reshape(-1, order="F"))
    return np.asfortranarray(x.reshape(B.shape, order="F"))


def _take(X, mu, lo, hi):
    sl = [slice(None)] * X.ndim
    sl[mu] = slice(lo, hi)
    return X[tuple(sl)]


def solve_recursive(A, B, C=None, nmin=4):
    B = np.asarray(B, dtype=np.complex128)
    A = [np.asarray(a, dtype=np.complex128) for a in A]
    C = None if C is None else [np.asarray(c, dtype=np.complex128) for c in C]
    n = list(B.shape)
    mu = int(np.argmax(n))  # lowest mode on ties
    m = n[mu]
    if m <= nmin:
        return solve_dense(A, B, C)
    k = m // 2
    cut = lambda M, lo, hi: [a if eta != mu else a[lo:hi, lo:hi] for eta, a in enumerate(M)]
    A11, A22 = cut(A, 0, k), cut(A, k, m)
    C11 = None if C is None else cut(C, 0, k)
    C22 = None if C is None else cut(C, k, m)
    X2 = solve_recursive(A22, _take(B, mu, k, m), C22, nmin)
    # Eq. (2.3a): B1 -= the terms of X2 through the off-diagonal blocks of mode mu
    B1 = np.array(_take(B, mu, 0, k))
    for term in range(len(A)):
        if C is None and term != mu:
            continue  # the Laplace form couples the two parts through A_mu only
        Y = X2
        for eta in range(len(A)):
            if eta == mu:
                M = (A if term == mu else C)[mu][:k, k:]
            elif C is None:
                continue
            else:
                M = A[eta] if eta == term else C[eta]
            Y = _mode(Y, M, eta)
        B1 -= Y
    X1 = solve_recursive(A11, B1, C11, nmin)
    return np.asfortranarray(np.concatenate([X1, X2], axis=mu))
