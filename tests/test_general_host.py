"""General (dense) coefficients on the CPU: the dense oracle and the host
reduction of the package (Alg. 1's Schur / QZ step), pinned independently.

* solve_dense on (quasi-)triangular coefficients equals the C oracle's
  element back-substitution (independent code, Sec. 2.1).
* solve_dense's solution satisfies the equation evaluated by mode products
  (tensordot), not by the assembled matrix it was solved with.
* Reducing general coefficients on the host (real Schur / QZ), transforming
  the right-hand side by mode products, solving the triangular equation with
  the C oracle and transforming back reproduces solve_dense.
"""
import numpy as np
import pytest

import oracle
import synthetic
from tests.kron_helpers import mode_product


def _general(rng, n, shift=2.5):
    return np.asfortranarray(rng.standard_normal((n, n)) / np.sqrt(n) + shift * np.eye(n))


def _apply(A, X, C=None):
    d = len(A)
    out = np.zeros_like(X)
    for mu in range(d):
        Y = X
        for eta in range(d):
            if eta == mu:
                Y = mode_product(Y, A[eta], eta)
            elif C is not None:
                Y = mode_product(Y, C[eta], eta)
        out = out + Y
    return out


@pytest.mark.parametrize("gen", [False, True])
def test_dense_oracle_matches_backsub_on_triangular(gen):
    p = synthetic.problem(11, (6, 5, 4), generalized=gen, force_blocks=[[2], [1], []])
    Xo = oracle.solve_backsub(p["A"], p["B"], p["C"])
    Xd = oracle.solve_dense(p["A"], p["B"], p["C"])
    assert np.linalg.norm(Xd - Xo) <= 1e-12 * np.linalg.norm(Xo)


@pytest.mark.parametrize("gen", [False, True])
@pytest.mark.parametrize("shape", [(7, 6), (5, 4, 6), (3, 4, 3, 4)])
def test_dense_oracle_residual_by_mode_products(gen, shape):
    rng = np.random.default_rng(13)
    A = [_general(rng, n) for n in shape]
    C = [_general(rng, n, 2.0) for n in shape] if gen else None
    B = np.asfortranarray(rng.standard_normal(shape))
    X = oracle.solve_dense(A, B, C)
    R = B - _apply(A, X, C)
    assert np.linalg.norm(R) <= 1e-12 * np.linalg.norm(B)


@pytest.mark.parametrize("gen", [False, True])
def test_host_reduction_reproduces_dense_solve(gen):
    from paper_1905_09539_gb300.general import reduce_coefficients
    rng = np.random.default_rng(17)
    shape = (7, 5, 6)
    A = [_general(rng, n) for n in shape]
    C = [_general(rng, n, 2.0) for n in shape] if gen else None
    B = np.asfortranarray(rng.standard_normal(shape))
    red = reduce_coefficients(A, C)
    if not gen:
        Ts = [r[0] for r in red]
        U = [r[1] for r in red]
        for mu, (T, u) in enumerate(zip(Ts, U)):
            assert np.allclose(u @ T @ u.T, A[mu], atol=1e-13)
            assert np.all(np.tril(T, -2) == 0)
        Bt = B
        for mu in range(3):
            Bt = mode_product(Bt, U[mu].T, mu)
        Y = oracle.solve_backsub(Ts, np.asfortranarray(Bt))
        X = Y
        for mu in range(3):
            X = mode_product(X, U[mu], mu)
    else:
        S = [r[0] for r in red]
        T = [r[1] for r in red]
        Q = [r[2] for r in red]
        Z = [r[3] for r in red]
        for mu in range(3):
            assert np.allclose(Q[mu] @ S[mu] @ Z[mu].T, A[mu], atol=1e-13)
            assert np.allclose(Q[mu] @ T[mu] @ Z[mu].T, C[mu], atol=1e-13)
            assert np.all(np.tril(T[mu], -1) == 0)
        Bt = B
        for mu in range(3):
            Bt = mode_product(Bt, Q[mu].T, mu)
        Y = oracle.solve_backsub(S, np.asfortranarray(Bt), T)
        X = Y
        for mu in range(3):
            X = mode_product(X, Z[mu], mu)
    Xd = oracle.solve_dense(A, B, C)
    assert np.linalg.norm(X - Xd) <= 1e-11 * np.linalg.norm(Xd)
