"""The double-float solve (precision TSYLV_DF64): every value a pair of floats
on the FP32 pipes, the same partition, schedule and back-substitution as the
FP64 solve.  Compared with the CPU oracle element by element (1e-11 relative,
the FP64 parity tolerance: a double-float operation errs by at most 2^-44
relative, far below it) for d = 1..4, both forms, ragged sizes, 2x2 blocks
across split points and coupled groups, the transposed equation and the deep
queue; at 256^3 the trailing box against the oracle and the FP64 residual of
the whole solution.
"""
import numpy as np
import pytest
import torch

import oracle
import synthetic
from tests.gpu_helpers import max_rel, norm_op, rel_err, to_dev, to_host

pytestmark = pytest.mark.gpu
TOL = 1e-11

CASES = [
    (1, (37,)), (1, (100,)),
    (2, (33, 17)), (2, (5, 70)),
    (3, (9, 8, 7)), (3, (24, 17, 13)), (3, (1, 20, 9)),
    (4, (9, 7, 5, 6)), (4, (13, 11, 10, 9)),
]


def _force(shape, te):
    return [[n // 2 - 1] if n > te and n >= 4 else [] for n in shape]


@pytest.fixture(scope="module")
def lib():
    import paper_1905_09539_gb300 as ts
    ts.load()
    return ts


def _solve(lib, p, transposed=False, **kw):
    A = [to_dev(a) for a in p["A"]]
    B = to_dev(p["B"])
    kw.setdefault("precision", lib.TSYLV_DF64)
    if p["C"] is not None:
        fn = lib.gtsylv_solve_transposed if transposed else lib.gtsylv_solve
        X, st = fn(A, [to_dev(c) for c in p["C"]], B, **kw)
    else:
        fn = lib.tsylv_solve_transposed if transposed else lib.tsylv_solve
        X, st = fn(A, B, **kw)
    assert st == 0
    return X


@pytest.mark.parametrize("gen", [False, True])
@pytest.mark.parametrize("d,shape", CASES)
@pytest.mark.parametrize("seed", [0, 1])
def test_df64_parity(lib, d, shape, gen, seed):
    if gen and d == 1:
        pytest.skip("one mode: the d-term form is the Laplace form")
    te = {1: 32, 2: 16, 3: 8, 4: 4}[d]
    p = synthetic.problem(seed, shape, generalized=gen, force_blocks=_force(shape, te) if seed else None)
    Xo = oracle.solve_recursive(p["A"], p["B"], p["C"], nmin=4)
    Xg = to_host(_solve(lib, p))
    assert rel_err(Xg, Xo) <= TOL
    assert max_rel(Xg, Xo) <= TOL


@pytest.mark.parametrize("gen", [False, True])
def test_df64_coupled_groups(lib, gen):
    """2x2 blocks in every mode at the same positions: coupled groups of 2, 4
    and 8 members in one block (warp elimination and precomputed inverses)."""
    shape = (12, 10, 9)
    p = synthetic.problem(7, shape, generalized=gen, force_blocks=[[0, 3, 6], [1, 4, 7], [2, 5]])
    Xo = oracle.solve_recursive(p["A"], p["B"], p["C"], nmin=4)
    assert rel_err(to_host(_solve(lib, p)), Xo) <= TOL


@pytest.mark.parametrize("gen", [False, True])
@pytest.mark.parametrize("shape", [(19, 23), (17, 12, 9), (7, 9, 5, 6)])
def test_df64_transposed(lib, shape, gen):
    te = {2: 16, 3: 8, 4: 4}[len(shape)]
    p = synthetic.problem(5, shape, generalized=gen, force_blocks=_force(shape, te))
    Lo = oracle.solve_backsub(p["A"], p["B"], p["C"], transpose=True)
    Lg = to_host(_solve(lib, p, transposed=True))
    assert rel_err(Lg, Lo) <= TOL


@pytest.mark.parametrize("gen", [False, True])
def test_df64_deep_queue(lib, gen):
    shape = (64, 64, 64)
    p = synthetic.problem(6, shape, generalized=gen)
    Xo = oracle.solve_recursive(p["A"], p["B"], p["C"], nmin=8)
    Xg = to_host(_solve(lib, p))
    assert rel_err(Xg, Xo) <= TOL
    assert max_rel(Xg, Xo) <= TOL


@pytest.mark.parametrize("gen", [False, True])
def test_df64_full_size(lib, gen):
    """256^3: the trailing 24^3 box against the oracle's solve of the trailing
    sub-problem, and the FP64 residual of the whole solution."""
    shape = (256, 256, 256)
    p = synthetic.problem(0, shape, generalized=gen)
    A = [to_dev(a) for a in p["A"]]
    C = [to_dev(c) for c in p["C"]] if gen else None
    B = to_dev(p["B"])
    X = _solve(lib, p)
    _, rho, _ = lib.tsylv_residual(A, B, X, C, residual=lib.TSYLV_RESID_FP64)
    assert rho <= 1e-13, rho
    Xh = to_host(X)
    ks = []
    for a in p["A"]:
        k = a.shape[0] - 24
        while a[k, k - 1] != 0.0:
            k -= 1
        ks.append(k)
    sub = tuple(slice(k, None) for k in ks)
    As = [np.asfortranarray(a[k:, k:]) for a, k in zip(p["A"], ks)]
    Cs = None if not gen else [np.asfortranarray(c[k:, k:]) for c, k in zip(p["C"], ks)]
    Xo = oracle.solve_recursive(As, np.asfortranarray(p["B"][sub]), Cs, nmin=4)
    assert rel_err(np.asfortranarray(Xh[sub]), Xo) <= TOL


def test_df64_singular(lib):
    p = synthetic.problem(8, (12, 10), block_prob=0.0)
    p["A"][0][3, 3] = 1.0
    p["A"][1][7, 7] = -1.0
    A = [to_dev(a) for a in p["A"]]
    _, st = lib.tsylv_solve(A, to_dev(p["B"]), precision=lib.TSYLV_DF64, check=False)
    assert st == 1


@pytest.mark.parametrize("kw", [{"nmin": -1}, {"leaf": (6, 5, 8)}, {"nmin": 4}])
def test_df64_tile_shapes(lib, kw):
    """Other leaf bounds (fixed, per mode, or autotuned) in double-float arithmetic."""
    shape = (29, 22, 18)
    p = synthetic.problem(9, shape, generalized=True, force_blocks=_force(shape, 8))
    Xo = oracle.solve_recursive(p["A"], p["B"], p["C"], nmin=4)
    assert rel_err(to_host(_solve(lib, p, **kw)), Xo) <= TOL


def test_df64_plan_and_in_place(lib):
    """A double-float solve plan (two right-hand sides queued) and an in-place call."""
    shape = (30, 21, 17)
    p = synthetic.problem(10, shape, generalized=True)
    A = [to_dev(a) for a in p["A"]]
    C = [to_dev(c) for c in p["C"]]
    plan = lib.SolvePlan(A, C, precision=lib.TSYLV_DF64)
    B2 = np.asfortranarray(2.0 * p["B"])
    outs = [plan.solve(to_dev(p["B"])), plan.solve(to_dev(B2))]
    torch.cuda.synchronize()
    Xo = oracle.solve_recursive(p["A"], p["B"], p["C"], nmin=4)
    for scale, (X, status) in zip((1.0, 2.0), outs):
        assert int(status.item()) == 0
        assert rel_err(to_host(X), scale * Xo) <= TOL
    plan.close()
    B = to_dev(p["B"])
    X, st = lib.gtsylv_solve(A, C, B, X=B, precision=lib.TSYLV_DF64)
    assert st == 0
    assert rel_err(to_host(X), Xo) <= TOL
