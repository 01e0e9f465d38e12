"""Full-size workloads, in the launch configuration the benchmark times.

At these sizes the oracle's whole-tensor solve takes minutes, so the check is
a property that holds at any size, evaluated independently of the CUDA path
on sampled entries: the componentwise residual
    r(u) = |B(u) - A(X)(u)| / (|B(u)| + (|A| |X|)(u))
where A(X)(u) is contracted directly from the definition (Eq. (2.2), and the
d-term form) with numpy in FP64 for each sampled multi-index u (corners
included: u = 0 carries the whole dependency cone).  An FP64 solve is
backward stable to a small multiple of n * eps, so r(u) <= 1e-11; the refined
solve stops at a normwise residual of 1e-12, so r(u) <= 1e-10.  At 256^3 the
trailing 24^3 box (which solves the trailing sub-problem by itself, the
coefficients being upper quasi-triangular) is also compared element by element
with the oracle's solve of that sub-problem.  The 64^3 workload is compared
element by element with the oracle in full.
"""
import numpy as np
import pytest
import torch

import oracle
import synthetic
from tests.gpu_helpers import rel_err, to_dev, to_host

@pytest.fixture(scope="module")
def lib():
    import paper_1905_09539_gb300 as ts
    ts.load()
    return ts


def _samples(shape, count, seed):
    rng = np.random.default_rng(seed)
    us = [tuple(0 for _ in shape), tuple(n - 1 for n in shape), tuple(n // 2 for n in shape)]
    for _ in range(count - len(us)):
        us.append(tuple(int(rng.integers(0, n)) for n in shape))
    return us


def _apply_at(u, X, A, C, absolute=False):
    """A(X)(u) (or (|A| |X|)(u)) from the definition: each term contracts X
    with the u-rows of its factors (A_mu in mode mu, C_eta or I elsewhere)."""
    d = X.ndim
    Xa = np.abs(X) if absolute else X
    total = 0.0
    for mu in range(d):
        rows = []
        for eta in range(d):
            if eta == mu:
                M = A[eta]
            elif C is None:
                rows.append(None)
                continue
            else:
                M = C[eta]
            r = M[u[eta], :].copy()
            # entries below the first subdiagonal (A) / the diagonal (C) are structural zeros
            lo = max(u[eta] - 1, 0) if eta == mu else u[eta]
            r[:lo] = 0.0
            rows.append(np.abs(r) if absolute else r)
        # restrict X to the term's dependency cone (rows vanish below their
        # first structural nonzero; identity factors select u_eta), then
        # contract mode by mode, last first
        idx, vecs = [], []
        for eta in range(d):
            if rows[eta] is None:
                idx.append(slice(u[eta], u[eta] + 1))
                vecs.append(np.ones(1))
            else:
                lo = max(u[eta] - 1, 0) if eta == mu else u[eta]
                idx.append(slice(lo, None))
                vecs.append(rows[eta][lo:])
        T = np.ascontiguousarray(Xa[tuple(idx)])
        for eta in range(d - 1, -1, -1):
            T = np.tensordot(T, vecs[eta], axes=([eta], [0]))
        total += float(T)
    return total


def _check_residual(X, p, tol, count=16, seed=0):
    A, C, B = p["A"], p["C"], p["B"]
    worst = 0.0
    for u in _samples(B.shape, count, seed):
        ax = _apply_at(u, X, A, C)
        den = abs(B[u]) + _apply_at(u, X, A, C, absolute=True)
        worst = max(worst, abs(B[u] - ax) / den)
    assert worst <= tol, worst
    return worst


def _trailing_cut(A, size):
    """First index k >= n - size of the trailing box that splits no 2x2 block (A(k, k-1) = 0)."""
    n = A.shape[0]
    k = n - size
    while k > 1 and A[k, k - 1] != 0.0:
        k -= 1
    return k


def _check_trailing_box(X, p, size, tol):
    """With upper quasi-triangular coefficients, the trailing box X[k:, k:, ...]
    (k not inside a 2x2 block) solves the trailing sub-problem on its own: the
    oracle solves that small problem and the GPU's entries are compared with
    it element by element."""
    ks = [_trailing_cut(a, size) for a in p["A"]]
    sub = tuple(slice(k, None) for k in ks)
    As = [np.asfortranarray(a[k:, k:]) for a, k in zip(p["A"], ks)]
    Cs = None if p["C"] is None else [np.asfortranarray(c[k:, k:]) for c, k in zip(p["C"], ks)]
    Xo = oracle.solve_recursive(As, np.asfortranarray(p["B"][sub]), Cs, nmin=4)
    err = rel_err(np.asfortranarray(X[sub]), Xo)
    assert err <= tol, err
    assert float(np.max(np.abs(X[sub] - Xo)) / np.max(np.abs(Xo))) <= tol


def _solve(lib, p, prec):
    A = [to_dev(a) for a in p["A"]]
    B = to_dev(p["B"])
    if p["C"] is not None:
        X, st = lib.gtsylv_solve(A, [to_dev(c) for c in p["C"]], B, precision=prec)
    else:
        X, st = lib.tsylv_solve(A, B, precision=prec)
    assert st == 0
    torch.cuda.synchronize()
    return to_host(X)


@pytest.mark.gpu
@pytest.mark.slow
def test_config_64cubed_vs_oracle(lib):
    p = synthetic.problem(0, (64, 64, 64))
    Xo = oracle.solve_recursive(p["A"], p["B"], nmin=8)
    for prec in (lib.TSYLV_FP64, lib.TSYLV_FP32_REFINED):
        X = _solve(lib, p, prec)
        assert rel_err(X, Xo) <= 1e-11


@pytest.mark.gpu
@pytest.mark.slow
@pytest.mark.parametrize("gen", [False, True])
@pytest.mark.parametrize("precision", ["fp64", "fp32r"])
def test_config_256cubed(lib, gen, precision):
    p = synthetic.problem(0, (256, 256, 256), generalized=gen)
    prec = lib.TSYLV_FP64 if precision == "fp64" else lib.TSYLV_FP32_REFINED
    X = _solve(lib, p, prec)
    _check_residual(X, p, 1e-11 if precision == "fp64" else 1e-10)
    _check_trailing_box(X, p, 24, 1e-11 if precision == "fp64" else 1e-10)


@pytest.mark.gpu
@pytest.mark.slow
@pytest.mark.parametrize("shape", [(64, 64, 64, 64), (128, 96, 64, 32)])
@pytest.mark.parametrize("precision", ["fp64", "fp32r"])
def test_config_d4_generalized(lib, shape, precision):
    p = synthetic.problem(0, shape, generalized=True)
    prec = lib.TSYLV_FP64 if precision == "fp64" else lib.TSYLV_FP32_REFINED
    X = _solve(lib, p, prec)
    _check_residual(X, p, 1e-11 if precision == "fp64" else 1e-10)


def test_residual_check_catches_a_wrong_solution():
    """The sampled check itself: a solution perturbed at one sampled entry fails."""
    p = synthetic.problem(3, (12, 10, 9), generalized=True)
    X = oracle.solve_recursive(p["A"], p["B"], p["C"], nmin=4)
    _check_residual(X, p, 1e-12)
    Xbad = X.copy()
    Xbad[6, 5, 4] += 1e-6
    with pytest.raises(AssertionError):
        _check_residual(Xbad, p, 1e-11)
