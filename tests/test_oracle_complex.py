"""Pins of the complex-triangular oracle (oracle/complex_tri.py) against facts
fixed by mathematics and by the already pinned real oracle.

A slip in it (a dropped term, a wrong sign, a conjugated or transposed
operand, the wrong off-diagonal block) fails one of:
  * closed form for diagonal complex coefficients
  * brute-force element sums of the operator (tiny shapes) against apply/assemble
  * textbook reductions: d = 1 complex triangular solve, d = 2 complex
    Sylvester equation (LAPACK's trsyl through scipy)
  * the complex-Schur route of a real quasi-triangular problem (Sec. 2.2 and
    Sec. 2.4: reduce every coefficient to complex Schur form, solve the
    triangular problem, transform back) against the real C oracle
  * the recursion (Alg. 2) agrees with the dense solve at every cutoff
"""
import itertools

import numpy as np
import pytest
import scipy.linalg as sla

import oracle
import synthetic
from oracle import complex_tri as ct

EPS = np.finfo(float).eps


@pytest.mark.parametrize("gen", [False, True])
@pytest.mark.parametrize("shape", [(7,), (6, 5), (5, 4, 6), (3, 4, 2, 5)])
def test_closed_form_diagonal(shape, gen):
    rng = np.random.default_rng(21)
    cz = lambda n: rng.uniform(1, 2, n) + 1j * rng.uniform(-1, 1, n)
    a = [cz(n) for n in shape]
    c = [cz(n) for n in shape]
    A = [np.diag(v) for v in a]
    C = [np.diag(v) for v in c] if gen else None
    B = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    ga = np.meshgrid(*a, indexing="ij")
    gc = np.meshgrid(*c, indexing="ij")
    den = 0
    for mu in range(len(shape)):
        t = ga[mu]
        if gen:
            for eta in range(len(shape)):
                if eta != mu:
                    t = t * gc[eta]
        den = den + t
    Xc = B / den
    for X in (ct.solve_dense(A, B, C), ct.solve_recursive(A, B, C, nmin=2)):
        assert np.max(np.abs(X - Xc) / np.abs(Xc)) <= 16 * EPS * len(shape)


def _brute_apply(A, X, C):
    """sum_mu X x_mu A_mu (x_{eta != mu} C_eta), one output entry at a time."""
    shape = X.shape
    d = len(shape)
    Y = np.zeros(shape, dtype=complex)
    for i in itertools.product(*[range(n) for n in shape]):
        acc = 0
        for j in itertools.product(*[range(n) for n in shape]):
            for mu in range(d):
                w = A[mu][i[mu], j[mu]]
                for eta in range(d):
                    if eta == mu:
                        continue
                    if C is None:
                        w = w * (1.0 if i[eta] == j[eta] else 0.0)
                    else:
                        w = w * C[eta][i[eta], j[eta]]
                acc += w * X[j]
        Y[i] = acc
    return Y


@pytest.mark.parametrize("gen", [False, True])
@pytest.mark.parametrize("shape", [(3,), (3, 2), (2, 3, 2), (2, 2, 2, 2)])
def test_operator_brute_force(shape, gen):
    p = synthetic.complex_problem(3, shape, generalized=gen)
    rng = np.random.default_rng(4)
    X = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    Yb = _brute_apply(p["A"], X, p["C"])
    assert np.allclose(ct.apply(p["A"], X, p["C"]), Yb, rtol=1e-14, atol=1e-14)
    Ym = (ct.assemble(p["A"], p["C"]) @ X.reshape(-1, order="F")).reshape(shape, order="F")
    assert np.allclose(Ym, Yb, rtol=1e-14, atol=1e-14)


def test_d1_triangular():
    p = synthetic.complex_problem(5, (23,))
    x = ct.solve_recursive(p["A"], p["B"], None, nmin=3)
    xs = sla.solve_triangular(p["A"][0], p["B"])
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= 1e-14


@pytest.mark.parametrize("gen", [False, True])
def test_d2_sylvester(gen):
    p = synthetic.complex_problem(6, (9, 7), generalized=gen)
    A1, A2 = p["A"]
    B = p["B"]
    if not gen:
        Xs = sla.solve_sylvester(A1, A2.T, B)  # A1 X + X A2^T = B
    else:
        C1, C2 = p["C"]
        # A1 X C2^T + C1 X A2^T = B  <=>  (C1^-1 A1) X + X (C2^-1 A2)^T = C1^-1 B C2^-T
        Xs = sla.solve_sylvester(np.linalg.solve(C1, A1), np.linalg.solve(C2, A2).T,
                                 np.linalg.solve(C1, np.linalg.solve(C2, B.T).T))
    for X in (ct.solve_dense(p["A"], B, p["C"]), ct.solve_recursive(p["A"], B, p["C"], nmin=2)):
        assert np.linalg.norm(X - Xs) / np.linalg.norm(Xs) <= 1e-12


@pytest.mark.parametrize("gen", [False, True])
@pytest.mark.parametrize("shape", [(7, 6), (6, 5, 7), (4, 5, 3, 4)])
def test_complex_schur_route_matches_real_oracle(shape, gen):
    p = synthetic.problem(11, shape, generalized=gen)
    A, C, B = p["A"], p["C"], p["B"]
    d = len(shape)
    if not gen:
        TU = [sla.schur(a, output="complex") for a in A]  # A = U T U^H
        T, S = [t for t, _ in TU], None
        Qh, Z = [u.conj().T for _, u in TU], [u for _, u in TU]
    else:
        T, S, Qh, Z = [], [], [], []
        for a, c in zip(A, C):
            AA, BB, Q, ZZ = sla.qz(a, c, output="complex")  # A = Q AA Z^H, C = Q BB Z^H
            T.append(AA)
            S.append(BB)
            Qh.append(Q.conj().T)
            Z.append(ZZ)
    Bt = B.astype(complex)
    for mu in range(d):
        Bt = ct._mode(Bt, Qh[mu], mu)
    Xt = ct.solve_recursive([np.triu(t) for t in T], Bt, None if S is None else [np.triu(s) for s in S], nmin=2)
    X = Xt
    for mu in range(d):
        X = ct._mode(X, Z[mu], mu)
    Xo = oracle.solve_recursive(A, B, C, nmin=2)
    assert np.max(np.abs(X.imag)) <= 1e-12 * np.max(np.abs(Xo))
    assert np.linalg.norm(X.real - Xo) / np.linalg.norm(Xo) <= 1e-12


@pytest.mark.parametrize("gen", [False, True])
@pytest.mark.parametrize("shape,nmins", [((13, 11, 9), (1, 2, 5, 13)), ((6, 5, 7, 4), (1, 3, 7)),
                                         ((40,), (1, 4, 40)), ((17, 9), (2, 8))])
def test_recursion_matches_dense(shape, nmins, gen):
    p = synthetic.complex_problem(12, shape, generalized=gen)
    Xd = ct.solve_dense(p["A"], p["B"], p["C"])
    for nmin in nmins:
        X = ct.solve_recursive(p["A"], p["B"], p["C"], nmin=nmin)
        assert np.linalg.norm(X - Xd) / np.linalg.norm(Xd) <= 1e-13, nmin
        R = p["B"] - ct.apply(p["A"], X, p["C"])
        assert np.linalg.norm(R) / np.linalg.norm(p["B"]) <= 1e-13


def test_trailing_box_is_decoupled():
    """With upper triangular coefficients the trailing box X[k:, k:, ...]
    solves the trailing sub-problem on its own: the fact the large GPU tests
    use to check sampled outputs."""
    p = synthetic.complex_problem(13, (12, 10, 9), generalized=True)
    X = ct.solve_recursive(p["A"], p["B"], p["C"], nmin=3)
    k = (5, 4, 6)
    sub = tuple(slice(kk, None) for kk in k)
    As = [a[kk:, kk:] for a, kk in zip(p["A"], k)]
    Cs = [c[kk:, kk:] for c, kk in zip(p["C"], k)]
    Xs = ct.solve_dense(As, p["B"][sub], Cs)
    assert np.linalg.norm(X[sub] - Xs) / np.linalg.norm(Xs) <= 1e-13
