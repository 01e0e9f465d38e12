"""Pins of the oracle of the paper's own generalized form (Sec. 3, Eq. (3.1)),
each independent of the code it checks:

* diagonal coefficients: the closed form x = b / (a1_i + c_i prod_{mu>=2} a_mu(j_mu));
* the operator by mode products equals the assembled matrix of Eq. (1.5);
* the recursion of Alg. 5 equals the dense assembled solve with 2x2 blocks
  forced across the split points (d = 2, 3, 4), and its residual, evaluated
  by mode products, is at rounding level;
* d = 2: the form is the generalized Sylvester equation A_1 X + C X A_2^T = B,
  the d-term form with (A_1, C) in mode 1 and (A_2, I) in mode 2 -- checked
  against the C oracle of that form;
* the shifted Kronecker case A_1 = -lambda I (Eq. (1.6)): the solution of
  (A_d x ... x A_2 x C - lambda I) vec(X) = vec(B).
"""
from functools import reduce

import numpy as np
import pytest

import oracle
import synthetic
from oracle import two_term


def _problem(seed, shape, force=None):
    p = synthetic.problem(seed, shape, generalized=True, force_blocks=force)
    return p["A"], p["C"][0], p["B"]


def test_closed_form_diagonal():
    rng = np.random.default_rng(1)
    shape = (5, 4, 3)
    a = [rng.uniform(1, 2, n) for n in shape]
    c = rng.uniform(1, 2, shape[0])
    A = [np.diag(v) for v in a]
    C = np.diag(c)
    B = rng.standard_normal(shape)
    i, j, k = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    Xc = B / (a[0][i] + c[i] * a[1][j] * a[2][k])
    for X in (two_term.solve_recursive(A, C, B, nmin=2), two_term.solve_dense(A, C, B)):
        assert np.max(np.abs(X - Xc) / np.abs(Xc)) <= 1e-14


@pytest.mark.parametrize("shape", [(6, 5), (4, 3, 5), (3, 4, 2, 3)])
def test_apply_equals_assembled(shape):
    A, C, _ = _problem(2, shape, force=[[1]] + [[]] * (len(shape) - 1))
    X = np.asfortranarray(np.random.default_rng(3).standard_normal(shape))
    y = two_term.assemble(A, C) @ X.reshape(-1, order="F")
    assert np.allclose(two_term.apply(A, C, X).reshape(-1, order="F"), y, rtol=0, atol=1e-13 * np.abs(y).max())


@pytest.mark.parametrize("shape", [(19, 13), (11, 9, 10), (7, 6, 5, 6)])
def test_recursion_equals_dense_solve(shape):
    force = [[n // 2 - 1] if n >= 6 else [] for n in shape]
    A, C, B = _problem(4, shape, force)
    Xr = two_term.solve_recursive(A, C, B, nmin=4)
    Xd = two_term.solve_dense(A, C, B)
    assert np.linalg.norm(Xr - Xd) <= 1e-12 * np.linalg.norm(Xd)
    R = B - two_term.apply(A, C, Xr)
    assert np.linalg.norm(R) <= 1e-13 * np.linalg.norm(B) * 10


def test_d2_is_the_generalized_sylvester_equation():
    shape = (17, 12)
    A, C, B = _problem(5, shape, force=[[7], [5]])
    X = two_term.solve_recursive(A, C, B, nmin=4)
    # the d-term form with (A_1, C) in mode 1 and (A_2, I) in mode 2
    Xo = oracle.solve_recursive(A, B, [C, np.asfortranarray(np.eye(shape[1]))], nmin=4)
    assert np.linalg.norm(X - Xo) <= 1e-12 * np.linalg.norm(Xo)


def test_shifted_kronecker_case():
    shape = (6, 5, 4)
    A, C, B = _problem(6, shape)
    lam = 0.75
    A = [np.asfortranarray(-lam * np.eye(shape[0]))] + list(A[1:])
    K = reduce(np.kron, [A[mu] for mu in range(len(shape) - 1, 0, -1)] + [C])
    x = np.linalg.solve(K - lam * np.eye(K.shape[0]), B.reshape(-1, order="F"))
    X = two_term.solve_recursive(A, C, B, nmin=4)
    assert np.linalg.norm(X.reshape(-1, order="F") - x) <= 1e-12 * np.linalg.norm(x)
