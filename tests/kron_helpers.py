"""Dense Kronecker assembly used only by the oracle pins (small sizes).

vec() is column-major (mode 1 fastest, Eq. (2.1)); the operator of the
Laplace form is Eq. (1.4), sum_mu I x ... x A_mu x ... x I with mode d
leftmost; the d-term generalized form replaces each identity of term mu by C_eta.
"""
from functools import reduce

import numpy as np


def vec(X):
    return np.asarray(X).reshape(-1, order="F")


def unvec(v, shape):
    return np.asarray(v).reshape(shape, order="F")


def operator(A, C=None):
    d = len(A)
    N = int(np.prod([a.shape[0] for a in A]))
    M = np.zeros((N, N))
    for mu in range(d):
        facs = []
        for eta in range(d):
            if eta == mu:
                facs.append(A[eta])
            elif C is None:
                facs.append(np.eye(A[eta].shape[0]))
            else:
                facs.append(C[eta])
        # Kronecker order: mode d leftmost, mode 1 rightmost (Eq. (1.4))
        M += reduce(np.kron, facs[::-1])
    return M


def mode_product(X, M, mu):
    """Y = X x_mu M, i.e. Y_(mu) = M X_(mu)."""
    Xm = np.moveaxis(X, mu, 0)
    Y = np.tensordot(M, Xm, axes=(1, 0))
    return np.moveaxis(Y, 0, mu)
