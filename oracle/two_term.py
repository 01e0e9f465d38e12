"""Plain CPU FP64 oracle for the paper's own generalized form (Sec. 3,
Eq. (3.1)):  X x_1 A_1 + X x_1 C x_2 A_2 x_3 ... x_d A_d = B,
with A_mu upper quasi-triangular and C upper triangular (after the reduction
of Alg. 4).  Its matrix is I x ... x I x A_1 + A_d x ... x A_2 x C (Eq. (1.5)).

TEST INFRASTRUCTURE ONLY (imported by tests/), numpy, small sizes:

* apply(A, C, X): the operator by mode products.
* assemble(A, C): the matrix Eq. (1.5) (column-major vec, mode 1 fastest).
* solve_dense(A, C, B): the assembled system solved by LAPACK.
* solve_recursive(A, C, B, nmin): the recursion of Sec. 3.1 (Alg. 5) in the
  paper's order: split the largest mode at floor(n/2), one further when the
  cut would separate a 2x2 block of A_mu; solve the trailing part; subtract
  its contribution from the leading right-hand side (case mu = 1: the A_1
  term and the C-chain term; case mu != 1: the chain with the off-diagonal
  block of A_mu in mode mu); solve the leading part with the updated
  right-hand side; small boxes by the dense solve.
"""
from functools import reduce

import numpy as np


def _mode(X, M, mu):
    """X x_mu M: (X x_mu M)(.., i, ..) = sum_k M(i, k) X(.., k, ..)."""
    Y = np.tensordot(np.asarray(M), np.moveaxis(X, mu, 0), axes=(1, 0))
    return np.moveaxis(Y, 0, mu)


def _chain(X, A, C, mu_block=None, block=None):
    """X x_1 C x_2 A_2 ... x_d A_d, with the factor of mode mu_block replaced by block."""
    d = X.ndim
    Y = X
    for mu in range(d):
        M = C if mu == 0 else A[mu]
        if mu == mu_block:
            M = block
        Y = _mode(Y, M, mu)
    return Y


def apply(A, C, X):
    X = np.asarray(X, dtype=np.float64)
    return _mode(X, A[0], 0) + _chain(X, A, C)


def assemble(A, C):
    d = len(A)
    n = [a.shape[0] for a in A]
    ident = [np.eye(m) for m in n]
    first = reduce(np.kron, [ident[mu] for mu in range(d - 1, 0, -1)] + [np.asarray(A[0])]) if d > 1 else \
        np.asarray(A[0], dtype=np.float64)
    second = reduce(np.kron, [np.asarray(A[mu]) for mu in range(d - 1, 0, -1)] + [np.asarray(C)]) if d > 1 else \
        np.asarray(C, dtype=np.float64)
    return first + second


def solve_dense(A, C, B):
    B = np.asarray(B, dtype=np.float64)
    x = np.linalg.solve(assemble(A, C), B.reshape(-1, order="F"))
    return np.asfortranarray(x.reshape(B.shape, order="F"))


def _take(X, mu, lo, hi):
    sl = [slice(None)] * X.ndim
    sl[mu] = slice(lo, hi)
    return X[tuple(sl)]


def solve_recursive(A, C, B, nmin=4):
    B = np.asarray(B, dtype=np.float64)
    A = [np.asarray(a, dtype=np.float64) for a in A]
    C = np.asarray(C, dtype=np.float64)
    n = list(B.shape)
    mu = int(np.argmax(n))  # lowest mode on ties
    m = n[mu]
    if m <= nmin:
        return solve_dense(A, C, B)
    k = m // 2
    if A[mu][k, k - 1] != 0.0:  # the cut would separate a 2x2 block
        k += 1
    if k >= m:
        k -= 2
    B1 = np.array(_take(B, mu, 0, k))
    B2 = _take(B, mu, k, m)
    A11 = [a if eta != mu else a[:k, :k] for eta, a in enumerate(A)]
    A22 = [a if eta != mu else a[k:, k:] for eta, a in enumerate(A)]
    if mu == 0:
        X2 = solve_recursive(A22, C[k:, k:], B2, nmin)
        B1 -= _mode(X2, A[0][:k, k:], 0) + _chain(X2, A, C[:k, k:])
        X1 = solve_recursive(A11, C[:k, :k], B1, nmin)
    else:
        X2 = solve_recursive(A22, C, B2, nmin)
        B1 -= _chain(X2, A, C, mu_block=mu, block=A[mu][:k, k:])
        X1 = solve_recursive(A11, C, B1, nmin)
    return np.asfortranarray(np.concatenate([X1, X2], axis=mu))
