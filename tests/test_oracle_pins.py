"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each pin is chosen so that a plausible slip in the oracle (a dropped term, a
wrong sign or index, a transposed operand, a cut 2x2 block) fails it:
  * closed form for diagonal coefficients (Eq. (2.2) with diagonal A_mu / C_mu)
  * LAPACK dense solve of the assembled Kronecker operator (Eq. (1.4))
  * textbook reductions: d = 1 triangular solve, d = 2 Sylvester (Eq. (1.1))
  * the complex-Schur route (Sec. 2.2: triangularize in complex arithmetic and
    drop the imaginary part) -- an algorithm without coupled 2x2 groups
  * C = I reduces the d-term form to the Laplace form
  * the two oracle routes (back-substitution, Alg. 2 recursion) agree
  * residual check of Sec. 2.4 and finite differences for the gradient
"""
import numpy as np
import pytest
import scipy.linalg as sla

import oracle
import synthetic
from tests.kron_helpers import mode_product, operator, unvec, vec

SHAPES = [(5,), (6, 5), (4, 5, 6), (3, 4, 3, 4), (2, 3, 2, 3, 2)]


def _prob(shape, gen, seed=0, force=None):
    return synthetic.problem(seed, shape, generalized=gen, force_blocks=force)


@pytest.mark.parametrize("gen", [False, True])
@pytest.mark.parametrize("shape", [(7,), (6, 5), (5, 4, 6), (3, 4, 2, 5), (3, 2, 4, 2, 3)])
def test_closed_form_diagonal(shape, gen):
    rng = np.random.default_rng(1)
    a = [rng.uniform(1, 2, n) for n in shape]
    c = [rng.uniform(1, 2, n) for n in shape]
    A = [np.diag(v) for v in a]
    C = [np.diag(v) for v in c] if gen else None
    B = np.asfortranarray(rng.standard_normal(shape))
    grids = np.meshgrid(*a, indexing="ij")
    if gen:
        cg = np.meshgrid(*c, indexing="ij")
        den = 0
        for mu in range(len(shape)):
            t = grids[mu].copy()
            for eta in range(len(shape)):
                if eta != mu:
                    t = t * cg[eta]
            den = den + t
    else:
        den = sum(grids)
    Xc = B / den
    for X in (oracle.solve_backsub(A, B, C), oracle.solve_recursive(A, B, C, nmin=2)):
        assert np.max(np.abs(X - Xc) / np.abs(Xc)) <= 4 * np.finfo(float).eps * len(shape)


def _split_points(n, nmin):
    """Split points the recursion visits in one mode (floor halving)."""
    pts = []

    def rec(lo, m):
        if m <= nmin:
            return
        k = m // 2
        pts.append(lo + k - 1)       # a 2x2 block starting here straddles the split
        rec(lo + k, m - k)
        rec(lo, k)
    rec(0, n)
    return pts


@pytest.mark.parametrize("gen", [False, True])
@pytest.mark.parametrize("shape", [(9,), (8, 7), (6, 6, 6), (4, 5, 6), (3, 4, 5, 6), (3, 4, 2, 3, 4)])
def test_dense_assembled_solve(shape, gen):
    # 2x2 blocks placed across split points, so the recursion's k+1 guard is exercised
    force = []
    for n in shape:
        pts = [p for p in _split_points(n, 2) if 0 <= p < n - 1]
        chosen, last = [], -3
        for p in sorted(pts):
            if p > last + 1:
                chosen.append(p)
                last = p + 1
        force.append(chosen)
    p = _prob(shape, gen, seed=3, force=force)
    A, C, B = p["A"], p["C"], p["B"]
    assert any(len(b) for b in p["blocks"])
    Xd = unvec(np.linalg.solve(operator(A, C), vec(B)), shape)
    for X in (oracle.solve_backsub(A, B, C),
              oracle.solve_recursive(A, B, C, nmin=2),
              oracle.solve_recursive(A, B, C, nmin=3)):
        assert np.linalg.norm(X - Xd) / np.linalg.norm(Xd) <= 1e-13


@pytest.mark.parametrize("gen", [False, True])
@pytest.mark.parametrize("shape", [(8, 6), (6, 6, 6), (7, 5, 6), (4, 4, 4, 4)])
def test_dense_solve_all_pairs(shape, gen):
    """Every index of every mode in a 2x2 block (one 1x1 block left in odd
    modes): nearly every unknown belongs to a coupled group of 2^d members,
    the perfect-shuffled diagonal blocks of Sec. 2.3 at their densest."""
    force = [list(range(0, n - 1, 2)) for n in shape]
    p = _prob(shape, gen, seed=5, force=force)
    A, C, B = p["A"], p["C"], p["B"]
    Xd = unvec(np.linalg.solve(operator(A, C), vec(B)), shape)
    for X in (oracle.solve_backsub(A, B, C),
              oracle.solve_recursive(A, B, C, nmin=2),
              oracle.solve_recursive(A, B, C, nmin=4)):
        assert np.linalg.norm(X - Xd) / np.linalg.norm(Xd) <= 1e-13


@pytest.mark.parametrize("shape", [(10, 8, 6), (9, 7)])
def test_dense_solve_real_schur(shape):
    """Coefficients that are real Schur forms of dense random matrices (the
    reduction of Alg. 1): 2x2 blocks wherever LAPACK's standardised form puts
    a complex pair, with unequal off-diagonal entries."""
    rng = np.random.default_rng(7)
    A = [np.asfortranarray(sla.schur(rng.standard_normal((n, n)) / np.sqrt(n) + 2.5 * np.eye(n),
                                     output="real")[0]) for n in shape]
    assert sum(int(np.count_nonzero(np.diag(a, -1))) for a in A) >= 2
    B = np.asfortranarray(rng.standard_normal(shape))
    Xd = unvec(np.linalg.solve(operator(A, None), vec(B)), shape)
    for X in (oracle.solve_backsub(A, B, None), oracle.solve_recursive(A, B, None, nmin=2)):
        assert np.linalg.norm(X - Xd) / np.linalg.norm(Xd) <= 1e-13


@pytest.mark.parametrize("gen", [False, True])
@pytest.mark.parametrize("shape", SHAPES)
def test_apply_matches_kron(shape, gen):
    p = _prob(shape, gen, seed=4)
    M = operator(p["A"], p["C"])
    Y = oracle.apply(p["A"], p["B"], p["C"])
    assert np.allclose(vec(Y), M @ vec(p["B"]), rtol=0, atol=1e-13 * np.abs(M).sum())
    YT = oracle.apply(p["A"], p["B"], p["C"], transpose=True)
    assert np.allclose(vec(YT), M.T @ vec(p["B"]), rtol=0, atol=1e-13 * np.abs(M).sum())


@pytest.mark.parametrize("gen", [False, True])
@pytest.mark.parametrize("shape", SHAPES)
def test_transposed_solve_matches_dense(shape, gen):
    p = _prob(shape, gen, seed=5)
    M = operator(p["A"], p["C"])
    Ld = unvec(np.linalg.solve(M.T, vec(p["B"])), shape)
    L = oracle.solve_backsub(p["A"], p["B"], p["C"], transpose=True)
    assert np.linalg.norm(L - Ld) / np.linalg.norm(Ld) <= 1e-13


@pytest.mark.parametrize("gen", [False, True])
@pytest.mark.parametrize("shape", SHAPES)
def test_transposed_recursion_matches_dense(shape, gen):
    """O-B on A^T (reversed recursion order) against LAPACK on the assembled M^T."""
    p = _prob(shape, gen, seed=6, force=[[n // 2 - 1] if n >= 4 else [] for n in shape])
    M = operator(p["A"], p["C"])
    Ld = unvec(np.linalg.solve(M.T, vec(p["B"])), shape)
    for nm in (2, 3, 5):
        L = oracle.solve_recursive(p["A"], p["B"], p["C"], nmin=nm, transpose=True)
        assert np.linalg.norm(L - Ld) / np.linalg.norm(Ld) <= 1e-13


def test_d1_triangular():
    rng = np.random.default_rng(7)
    A = np.triu(rng.standard_normal((12, 12))) + 3 * np.eye(12)
    b = rng.standard_normal(12)
    x = oracle.solve_backsub([A], b)
    assert np.allclose(x, sla.solve_triangular(A, b), rtol=1e-13, atol=0)


@pytest.mark.parametrize("gen", [False, True])
def test_d2_sylvester(gen):
    p = _prob((9, 7), gen, seed=8, force=[[2, 5], [3]])
    A1, A2 = p["A"]
    B = p["B"]
    if not gen:
        # Eq. (1.1): A1 X + X A2^T = B
        Xs = sla.solve_sylvester(A1, A2.T, B)
    else:
        # A1 X C2^T + C1 X A2^T = B  <=>  (C1^-1 A1) X + X (C2^-1 A2)^T = C1^-1 B C2^-T
        C1, C2 = p["C"]
        Xs = sla.solve_sylvester(np.linalg.solve(C1, A1), np.linalg.solve(C2, A2).T,
                                 np.linalg.solve(C1, np.linalg.solve(C2, B.T).T))
    for X in (oracle.solve_backsub(p["A"], B, p["C"]), oracle.solve_recursive(p["A"], B, p["C"], nmin=2)):
        assert np.linalg.norm(X - Xs) / np.linalg.norm(Xs) <= 1e-12


def _complex_triangular_solve(T, S, B):
    """Back-substitution for sum_mu X x_mu T_mu (x_eta S_eta) = B with upper
    triangular complex T_mu (S_mu), one unknown at a time (no coupled groups)."""
    shape = B.shape
    d = len(shape)
    X = np.zeros(shape, dtype=complex)
    for idx in reversed(list(np.ndindex(*shape))):
        # contributions of all later unknowns in the cone v >= idx
        sl = tuple(slice(i, None) for i in idx)
        sub = X[sl].copy()
        tot = 0
        diag = 0
        for mu in range(d):
            t = sub
            coef = 1.0
            for eta in range(d):
                M = T[eta] if eta == mu else (S[eta] if S is not None else None)
                if M is None:
                    continue
                row = M[idx[eta], idx[eta]:]
                t = np.tensordot(row, np.moveaxis(t, eta, 0), axes=(0, 0))
                t = np.expand_dims(t, 0)
                t = np.moveaxis(t, 0, eta)
                coef = coef * M[idx[eta], idx[eta]]
            if S is None:
                # Laplace: only the mode-mu line couples
                line = [0] * d
                row = T[mu][idx[mu], idx[mu]:]
                line_vals = np.moveaxis(sub, mu, 0)[(slice(None),) + (0,) * (d - 1)]
                tot += np.dot(row, line_vals)
            else:
                tot += t.reshape(-1)[0]
            diag += coef
        X[idx] = (B[idx] - tot) / diag
    return X


@pytest.mark.parametrize("gen", [False, True])
@pytest.mark.parametrize("shape", [(6, 5), (5, 4, 6), (3, 4, 3, 3)])
def test_complex_schur_route(shape, gen):
    p = _prob(shape, gen, seed=9)
    A, C, B = p["A"], p["C"], p["B"]
    d = len(shape)
    if not gen:
        # complex Schur A = U T U^H, X = Xt x_mu U_mu, Bt = B x_mu U_mu^H
        TU = [sla.schur(a, output="complex") for a in A]
        T = [t for t, _ in TU]
        U = [u for _, u in TU]
        S = None
        Qh = [u.conj().T for u in U]
        Z = U
    else:
        # complex QZ of (A_mu, C_mu): A = Q S Z^H, C = Q T Z^H
        T, S, Qh, Z = [], [], [], []
        for a, c in zip(A, C):
            AA, BB, Q, ZZ = sla.qz(a, c, output="complex")
            T.append(AA)
            S.append(BB)
            Qh.append(Q.conj().T)
            Z.append(ZZ)
    Bt = B.astype(complex)
    for mu in range(d):
        Bt = mode_product(Bt, Qh[mu], mu)
    Xt = _complex_triangular_solve(T, S, Bt)
    X = Xt
    for mu in range(d):
        X = mode_product(X, Z[mu], mu)
    assert np.max(np.abs(X.imag)) <= 1e-12 * np.max(np.abs(X.real))
    Xo = oracle.solve_recursive(A, B, C, nmin=2)
    assert np.linalg.norm(Xo - X.real) / np.linalg.norm(X.real) <= 1e-12


@pytest.mark.parametrize("shape", [(5, 4, 6), (3, 4, 3, 4)])
def test_c_identity_reduces_to_laplace(shape):
    p = _prob(shape, False, seed=10)
    I = [np.eye(n) for n in shape]
    X1 = oracle.solve_recursive(p["A"], p["B"], None, nmin=2)
    X2 = oracle.solve_recursive(p["A"], p["B"], I, nmin=2)
    assert np.linalg.norm(X1 - X2) / np.linalg.norm(X1) <= 1e-14


@pytest.mark.parametrize("gen", [False, True])
@pytest.mark.parametrize("shape,nmins", [((20, 17, 15), (2, 5, 8, 20)), ((9, 8, 7, 6), (2, 3, 9)),
                                         ((6, 5, 4, 5, 4), (2, 3, 6))])
def test_routes_agree_and_residual(shape, nmins, gen):
    p = _prob(shape, gen, seed=11)
    A, C, B = p["A"], p["C"], p["B"]
    Xa = oracle.solve_backsub(A, B, C)
    normA = sum(np.linalg.norm(A[mu], 2) * np.prod([np.linalg.norm(C[e], 2) for e in range(len(shape)) if e != mu])
                if C is not None else np.linalg.norm(A[mu], 2) for mu in range(len(shape)))
    for nm in nmins:
        Xb = oracle.solve_recursive(A, B, C, nmin=nm)
        assert np.linalg.norm(Xa - Xb) / np.linalg.norm(Xa) <= 1e-13
        R = B - oracle.apply(A, Xb, C)
        assert np.linalg.norm(R) / (normA * np.linalg.norm(Xb)) <= 1e-13


def test_merge_identity():
    # Sec. 2.2 (Laplace): modes 1,2 merge into A'_1 = I (x) A_1 + A_2 (x) I.
    # Generalized d-term form (derived): A' = C_2 (x) A_1 + A_2 (x) C_1, C' = C_2 (x) C_1.
    for gen in (False, True):
        p = _prob((3, 4, 5), gen, seed=12)
        A, C = p["A"], p["C"]
        n1, n2 = 3, 4
        if not gen:
            Ap = np.kron(np.eye(n2), A[0]) + np.kron(A[1], np.eye(n1))
            M2 = operator([Ap, A[2]])
        else:
            Ap = np.kron(C[1], A[0]) + np.kron(A[1], C[0])
            Cp = np.kron(C[1], C[0])
            M2 = operator([Ap, A[2]], [Cp, C[2]])
        M3 = operator(A, C)
        assert np.max(np.abs(M3 - M2)) <= 1e-14 * np.max(np.abs(M3))


@pytest.mark.parametrize("gen", [False, True])
def test_gradient_finite_differences(gen):
    shape = (5, 4, 6)
    p = _prob(shape, gen, seed=13, force=[[1], [2], [3]])
    A, C, B, Xs = p["A"], p["C"], p["B"], p["Xstar"]

    def loss(A_, B_, C_):
        X = oracle.solve_backsub(A_, B_, C_)
        return 0.5 * np.sum((X - Xs) ** 2)

    X = oracle.solve_backsub(A, B, C)
    Lam = oracle.solve_backsub(A, X - Xs, C, transpose=True)
    dA, dC = oracle.grad(A, X, Lam, C)
    rng = np.random.default_rng(14)
    h = 1e-6
    for _ in range(20):
        which = rng.integers(0, 3 if gen else 2)
        mu = int(rng.integers(0, 3))
        n = shape[mu]
        if which == 0:        # direction in B
            E = rng.standard_normal(shape)
            g = np.sum(Lam * E)
            fp = loss(A, B + h * E, C)
            fm = loss(A, B - h * E, C)
        elif which == 1:      # masked direction in A_mu
            E = np.triu(rng.standard_normal((n, n)))
            for s in p["blocks"][mu]:
                E[s + 1, s] = rng.standard_normal()
            g = np.sum(dA[mu] * E)
            Ap = [a.copy() for a in A]; Am = [a.copy() for a in A]
            Ap[mu] = Ap[mu] + h * E; Am[mu] = Am[mu] - h * E
            fp = loss(Ap, B, C); fm = loss(Am, B, C)
        else:                 # direction in C_mu
            E = np.triu(rng.standard_normal((n, n)))
            g = np.sum(dC[mu] * E)
            Cp = [c.copy() for c in C]; Cm = [c.copy() for c in C]
            Cp[mu] = Cp[mu] + h * E; Cm[mu] = Cm[mu] - h * E
            fp = loss(A, B, Cp); fm = loss(A, B, Cm)
        fd = (fp - fm) / (2 * h)
        assert abs(fd - g) <= 1e-6 * max(1.0, abs(g))


def test_gradient_mask():
    p = _prob((6, 5, 4), False, seed=15, force=[[1], [], [2]])
    X = oracle.solve_backsub(p["A"], p["B"])
    Lam = oracle.solve_backsub(p["A"], X, transpose=True)
    dA, _ = oracle.grad(p["A"], X, Lam)
    for mu, g in enumerate(dA):
        n = g.shape[0]
        for i in range(n):
            for j in range(n):
                allowed = i <= j or (i == j + 1 and j in p["blocks"][mu])
                if not allowed:
                    assert g[i, j] == 0.0


def test_structure_rejected():
    A = np.triu(np.ones((5, 5)))
    A[1, 0] = 1.0
    A[2, 1] = 1.0                 # two adjacent subdiagonal entries: not quasi-triangular
    with pytest.raises(oracle.OracleError):
        oracle.solve_backsub([A], np.ones(5))


@pytest.mark.parametrize("gen", [False, True])
def test_trailing_box_is_decoupled(gen):
    """With upper quasi-triangular coefficients and a cut k that splits no 2x2
    block, the trailing box X[k:, k:, k:] solves the trailing sub-problem by
    itself (the fact the full-size GPU tests use to check outputs element by
    element): the C oracle on the whole problem against the dense solve of the
    trailing one."""
    shape = (14, 12, 11)
    p = _prob(shape, gen, seed=17, force=[[3], [5], [2]])
    X = oracle.solve_recursive(p["A"], p["B"], p["C"], nmin=4)
    ks = []
    for a in p["A"]:
        k = a.shape[0] - 6
        while a[k, k - 1] != 0.0:
            k -= 1
        ks.append(k)
    sub = tuple(slice(k, None) for k in ks)
    As = [a[k:, k:] for a, k in zip(p["A"], ks)]
    Cs = None if p["C"] is None else [c[k:, k:] for c, k in zip(p["C"], ks)]
    M = operator(As, Cs)
    Xs = unvec(np.linalg.solve(M, vec(p["B"][sub])), tuple(a.shape[0] for a in As))
    assert np.linalg.norm(X[sub] - Xs) / np.linalg.norm(Xs) <= 1e-13
