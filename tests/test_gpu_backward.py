"""Adjoint of the solve on the GPU (tsylv_backward and the autograd Function).

For L(X) with gradient dX at the solution X of A(X) = B:
  Lambda = A^{-T}(dX), dB = Lambda,
  dA_mu = -mask_A(Lambda_(mu) [X x_{eta != mu} C_eta]_(mu)^T),
  dC_mu = -mask_C(sum_{nu != mu} Lambda_(mu) [X x_nu A_nu x_{eta != mu, nu} C_eta]_(mu)^T).
Checked against the oracle's FP64 gradient (1e-10 relative per matrix; dB
1e-11 as any FP64 solve) and, through torch.autograd, against central finite
differences with h = 1e-6 on L = 0.5 ||X - X*||^2 along 20 random directions
drawn inside the masks (1e-6 relative).
"""
import numpy as np
import pytest
import torch

import oracle
import synthetic
from tests.gpu_helpers import rel_err, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import paper_1905_09539_gb300 as ts
    ts.load()
    return ts


def _mat_err(G, Go):
    den = np.linalg.norm(Go)
    return float(np.linalg.norm(G - Go) / den) if den > 0 else float(np.linalg.norm(G))


CASES = [
    (False, (40,)), (False, (33, 17)), (False, (5, 4, 6)), (False, (33, 30, 31)), (False, (9, 7, 5, 6)),
    (True, (33, 17)), (True, (5, 4, 6)), (True, (17, 13, 11)), (True, (6, 5, 4, 5)),
]


def _force(shape):
    return [[n // 2 - 1] if n >= 4 else [] for n in shape]


@pytest.mark.parametrize("gen,shape", CASES)
@pytest.mark.parametrize("precision", ["fp64", "fp32r", "df64"])
def test_backward_vs_oracle(lib, gen, shape, precision):
    p = synthetic.problem(21, shape, generalized=gen, force_blocks=_force(shape))
    A, C, B, Xs = p["A"], p["C"], p["B"], p["Xstar"]
    X = oracle.solve_backsub(A, B, C)
    dX = X - Xs
    Lam = oracle.solve_backsub(A, dX, C, transpose=True)
    dAo, dCo = oracle.grad(A, X, Lam, C)
    prec = {"fp64": lib.TSYLV_FP64, "fp32r": lib.TSYLV_FP32_REFINED, "tf32r": lib.TSYLV_TF32_REFINED,
            "df64": lib.TSYLV_DF64}[precision]
    dB, dA, dC = lib.tsylv_backward([to_dev(a) for a in A], to_dev(X), to_dev(dX),
                                    [to_dev(c) for c in C] if gen else None, precision=prec)
    torch.cuda.synchronize()
    assert rel_err(to_host(dB), Lam) <= 1e-11
    for mu in range(len(shape)):
        assert _mat_err(to_host(dA[mu]), dAo[mu]) <= 1e-10, mu
        if gen:
            assert _mat_err(to_host(dC[mu]), dCo[mu]) <= 1e-10, mu
    # masks: exact zeros outside the quasi-triangular pattern / the upper triangle
    for mu, g in enumerate(dA):
        g = to_host(g)
        n = g.shape[0]
        for j in range(n):
            for i in range(j + 2, n):
                assert g[i, j] == 0.0
            if j + 1 < n and j not in p["blocks"][mu]:
                assert g[j + 1, j] == 0.0
        if gen:
            assert np.all(np.tril(to_host(dC[mu]), -1) == 0.0)


def test_backward_without_dB(lib):
    """dB = NULL: Lambda lives in the workspace; dA must not change."""
    p = synthetic.problem(22, (24, 17, 13), force_blocks=_force((24, 17, 13)))
    A = [to_dev(a) for a in p["A"]]
    X = to_dev(oracle.solve_backsub(p["A"], p["B"]))
    dX = to_dev(p["Xstar"])
    _, dA1, _ = lib.tsylv_backward(A, X, dX, want_dB=True)
    dB2, dA2, _ = lib.tsylv_backward(A, X, dX, want_dB=False)
    assert dB2 is None
    for a, b in zip(dA1, dA2):
        assert _mat_err(to_host(b), to_host(a)) <= 1e-13


@pytest.mark.parametrize("gen", [False, True])
def test_backward_into_out_buffers(lib, gen):
    """out=(dB, dA, dC): the gradients land in the caller's tensors and equal
    freshly allocated ones (dB bit for bit; dA, dC to rounding: their
    contractions sum partial products with atomics, in no fixed order); a
    wrong layout is refused."""
    shape = (24, 17, 13)
    p = synthetic.problem(23, shape, generalized=gen, force_blocks=_force(shape))
    A = [to_dev(a) for a in p["A"]]
    C = [to_dev(c) for c in p["C"]] if gen else None
    X = to_dev(oracle.solve_recursive(p["A"], p["B"], p["C"], nmin=4))
    dX = to_dev(p["Xstar"])
    dB1, dA1, dC1 = lib.tsylv_backward(A, X, dX, C)
    oB = lib.empty_fortran(shape, X.device)
    oA = [lib.empty_fortran((m, m), X.device) for m in shape]
    oC = [lib.empty_fortran((m, m), X.device) for m in shape] if gen else None
    dB2, dA2, dC2 = lib.tsylv_backward(A, X, dX, C, out=(oB, oA, oC))
    assert dB2 is oB and all(a is b for a, b in zip(dA2, oA))
    assert torch.equal(dB1, dB2)
    for a, b in zip(dA1, dA2):
        assert _mat_err(to_host(b), to_host(a)) <= 1e-13
    if gen:
        assert all(a is b for a, b in zip(dC2, oC))
        for a, b in zip(dC1, dC2):
            assert _mat_err(to_host(b), to_host(a)) <= 1e-13
    with pytest.raises(ValueError):
        lib.tsylv_backward(A, X, dX, C, out=(torch.empty(shape, dtype=torch.float64, device=X.device), oA, oC))


def _fd_check(lib, shape, gen, seed, recompute=False, h=1e-6, ndir=20):
    p = synthetic.problem(seed, shape, generalized=gen, force_blocks=_force(shape))
    d = len(shape)
    A = [to_dev(a).requires_grad_(True) for a in p["A"]]
    C = [to_dev(c).requires_grad_(True) for c in p["C"]] if gen else None
    B = to_dev(p["B"]).requires_grad_(True)
    Xs = to_dev(p["Xstar"])
    X = lib.solve(A, B, C, recompute=recompute)
    loss = 0.5 * torch.sum((X - Xs) ** 2)
    loss.backward()
    gB = to_host(B.grad)
    gA = [to_host(a.grad) for a in A]
    gC = [to_host(c.grad) for c in C] if gen else None

    def X_of(Ah, Bh, Ch):
        with torch.no_grad():
            return lib.solve([to_dev(a) for a in Ah], to_dev(Bh), [to_dev(c) for c in Ch] if Ch is not None else None)

    def central(pl, mi):
        # (L(X+) - L(X-)) / 2h with L = 0.5 ||X - X*||^2, the difference of the
        # two losses written as 0.5 sum (X+ - X-)(X+ + X- - 2 X*): the same
        # central difference, without cancelling two large sums
        Xp, Xm = X_of(*pl), X_of(*mi)
        return 0.5 * float(torch.sum((Xp - Xm) * (Xp + Xm - 2 * Xs))) / (2 * h)

    rng = np.random.default_rng(seed + 1000)
    Ah, Bh, Ch = p["A"], p["B"], p["C"]
    worst = 0.0
    for _ in range(ndir):
        which = int(rng.integers(0, 3 if gen else 2))
        mu = int(rng.integers(0, d))
        n = shape[mu]
        if which == 0:
            E = np.asfortranarray(rng.standard_normal(shape))
            g = float(np.sum(gB * E))
            fd = central((Ah, Bh + h * E, Ch), (Ah, Bh - h * E, Ch))
        elif which == 1:
            E = np.triu(rng.standard_normal((n, n)))
            for s in p["blocks"][mu]:
                E[s + 1, s] = rng.standard_normal()
            g = float(np.sum(gA[mu] * E))
            Ap = [a.copy() for a in Ah]
            Am = [a.copy() for a in Ah]
            Ap[mu] += h * E
            Am[mu] -= h * E
            fd = central((Ap, Bh, Ch), (Am, Bh, Ch))
        else:
            E = np.triu(rng.standard_normal((n, n)))
            g = float(np.sum(gC[mu] * E))
            Cp = [c.copy() for c in Ch]
            Cm = [c.copy() for c in Ch]
            Cp[mu] += h * E
            Cm[mu] -= h * E
            fd = central((Ah, Bh, Cp), (Ah, Bh, Cm))
        err = abs(fd - g) / max(1.0, abs(g))
        worst = max(worst, err)
    assert worst <= 1e-6, worst


@pytest.mark.parametrize("gen,shape", [(False, (5, 4, 6)), (True, (5, 4, 6)), (False, (20, 16, 12)),
                                       (True, (9, 7, 5, 6))])
def test_autograd_finite_differences(lib, gen, shape):
    _fd_check(lib, shape, gen, seed=31)


def test_autograd_recompute(lib):
    """recompute=True keeps B instead of X and re-solves in backward: same gradients."""
    shape = (12, 10, 9)
    p = synthetic.problem(33, shape, generalized=True, force_blocks=_force(shape))
    grads = []
    for rc in (False, True):
        A = [to_dev(a).requires_grad_(True) for a in p["A"]]
        C = [to_dev(c).requires_grad_(True) for c in p["C"]]
        B = to_dev(p["B"]).requires_grad_(True)
        X = lib.solve(A, B, C, recompute=rc)
        (0.5 * torch.sum((X - to_dev(p["Xstar"])) ** 2)).backward()
        grads.append([to_host(B.grad)] + [to_host(a.grad) for a in A] + [to_host(c.grad) for c in C])
    for g0, g1 in zip(*grads):
        assert _mat_err(g1, g0) <= 1e-13


_CONFIG_CACHE = {}


def _config_oracle(p):
    """Oracle X, Lambda (O-B, forward and reversed recursion) and dA of the
    differentiation workload, computed once per session."""
    if "v" not in _CONFIG_CACHE:
        A, B, Xs = p["A"], p["B"], p["Xstar"]
        X = oracle.solve_recursive(A, B, nmin=8)
        Lam = oracle.solve_recursive(A, X - Xs, nmin=8, transpose=True)
        dAo, _ = oracle.grad(A, X, Lam)
        _CONFIG_CACHE["v"] = (X, Lam, dAo)
    return _CONFIG_CACHE["v"]


@pytest.mark.slow
@pytest.mark.parametrize("precision", ["fp64", "fp32r", "tf32r", "df64"])
def test_differentiation_config(lib, precision):
    """d = 3, n = (200, 160, 120), Laplace form, L = 0.5 ||X - X*||^2: the
    gradient against the oracle's FP64 gradient, and (FP64) central finite
    differences with h = 1e-6 on 20 masked random directions."""
    shape = (200, 160, 120)
    p = synthetic.problem(0, shape)
    A, B, Xs = p["A"], p["B"], p["Xstar"]
    X, Lam, dAo = _config_oracle(p)
    prec = {"fp64": lib.TSYLV_FP64, "fp32r": lib.TSYLV_FP32_REFINED, "tf32r": lib.TSYLV_TF32_REFINED,
            "df64": lib.TSYLV_DF64}[precision]
    Ad = [to_dev(a).requires_grad_(True) for a in A]
    Bd = to_dev(B).requires_grad_(True)
    Xd = lib.solve(Ad, Bd, precision=prec)
    assert rel_err(to_host(Xd), X) <= 1e-11
    (0.5 * torch.sum((Xd - to_dev(Xs)) ** 2)).backward()
    assert rel_err(to_host(Bd.grad), Lam) <= 1e-11
    for mu in range(3):
        assert _mat_err(to_host(Ad[mu].grad), dAo[mu]) <= 1e-10
    if precision == "fp64":
        _fd_check(lib, shape, False, seed=0)
