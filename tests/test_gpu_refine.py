"""Residual and mixed-precision refinement on the GPU, against the oracle.

Tolerances: the residual entries agree with the oracle's B - A(X) to
1e-12 of max|A(X)| (FP64: rounding of two different summation orders;
DF64: plus the 2^-48 representation error of its float pairs).  A refined
solve must reach ||B - A(X)|| / (||A|| ||X||) <= 1e-12; its forward error
against the FP64 oracle is then bounded by cond(A) * 1e-12 (cond <= ~20 for
these coefficient distributions), tested at 1e-10.
"""
import numpy as np
import pytest
import torch

import oracle
import synthetic
from tests.gpu_helpers import norm_op, rel_err, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ts():
    import paper_1905_09539_gb300 as m
    m.load()
    return m


SHAPES = [(2, (23, 19)), (3, (17, 12, 9)), (3, (33, 30, 31)), (4, (9, 7, 5, 6))]


@pytest.mark.parametrize("resid", [0, 1])
@pytest.mark.parametrize("gen", [False, True])
@pytest.mark.parametrize("d,shape", SHAPES)
def test_residual_matches_oracle(ts, d, shape, gen, resid):
    p = synthetic.problem(31, shape, generalized=gen, force_blocks=[[n // 2 - 1] if n > 4 else [] for n in shape])
    rng = np.random.default_rng(5)
    X = np.asfortranarray(rng.standard_normal(shape))
    AX = oracle.apply(p["A"], X, p["C"])
    Ro = p["B"] - AX
    A = [to_dev(a) for a in p["A"]]
    C = [to_dev(c) for c in p["C"]] if gen else None
    R, rel, st = ts.tsylv_residual(A, to_dev(p["B"]), to_dev(X), C, residual=resid)
    assert st == 0
    Rg = to_host(R)
    assert np.max(np.abs(Rg - Ro)) <= 1e-12 * np.max(np.abs(AX))
    relo = np.linalg.norm(Ro) / (norm_op(p["A"], p["C"]) * np.linalg.norm(X))
    assert abs(rel - relo) <= 1e-2 * relo  # power-iteration estimates of the 2-norms


@pytest.mark.parametrize("resid", [0, 1])
@pytest.mark.parametrize("gen", [False, True])
@pytest.mark.parametrize("d,shape", SHAPES + [(3, (64, 64, 64))])
def test_fp32_refined_solve(ts, d, shape, gen, resid):
    p = synthetic.problem(32, shape, generalized=gen, force_blocks=[[n // 2 - 1] if n > 4 else [] for n in shape])
    Xo = oracle.solve_recursive(p["A"], p["B"], p["C"], nmin=8)
    A = [to_dev(a) for a in p["A"]]
    info = ts.Info()
    if gen:
        X, st = ts.gtsylv_solve(A, [to_dev(c) for c in p["C"]], to_dev(p["B"]), precision=ts.TSYLV_FP32_REFINED,
                                residual=resid, info=info)
    else:
        X, st = ts.tsylv_solve(A, to_dev(p["B"]), precision=ts.TSYLV_FP32_REFINED, residual=resid, info=info)
    assert st == 0
    assert 0 < info.resid <= 1e-12
    assert 1 <= info.iterations <= 4
    Xg = to_host(X)
    assert rel_err(Xg, Xo) <= 1e-10
    # the residual the solver reports is the one the oracle sees
    R = p["B"] - oracle.apply(p["A"], Xg, p["C"])
    rho = np.linalg.norm(R) / (norm_op(p["A"], p["C"]) * np.linalg.norm(Xg))
    assert rho <= 2e-12


@pytest.mark.parametrize("gen", [False, True])
def test_refined_transposed(ts, gen):
    shape = (19, 17, 13)
    p = synthetic.problem(33, shape, generalized=gen, force_blocks=[[8], [7], [5]])
    Lo = oracle.solve_backsub(p["A"], p["B"], p["C"], transpose=True)
    A = [to_dev(a) for a in p["A"]]
    info = ts.Info()
    if gen:
        L, st = ts.gtsylv_solve_transposed(A, [to_dev(c) for c in p["C"]], to_dev(p["B"]),
                                           precision=ts.TSYLV_FP32_REFINED, info=info)
    else:
        L, st = ts.tsylv_solve_transposed(A, to_dev(p["B"]), precision=ts.TSYLV_FP32_REFINED, info=info)
    assert st == 0 and info.resid <= 1e-12
    assert rel_err(to_host(L), Lo) <= 1e-10


def test_refined_zero_rhs(ts):
    p = synthetic.problem(34, (12, 11, 10))
    B = np.zeros((12, 11, 10), order="F")
    X, st = ts.tsylv_solve([to_dev(a) for a in p["A"]], to_dev(B), precision=ts.TSYLV_FP32_REFINED)
    assert st == 0
    assert np.all(to_host(X) == 0)


def test_refined_iteration_cap(ts):
    # one step cannot reach 1e-12 from FP32 solves: ENOCONV, last iterate returned
    p = synthetic.problem(35, (24, 20, 16))
    info = ts.Info()
    X, st = ts.tsylv_solve([to_dev(a) for a in p["A"]], to_dev(p["B"]), precision=ts.TSYLV_FP32_REFINED,
                           max_refine=1, check=False, info=info)
    assert st == ts._lib.TSYLV_ENOCONV
    assert info.iterations == 1 and 1e-12 < info.resid < 1e-4


@pytest.mark.parametrize("update", [0, 1])
@pytest.mark.parametrize("gen", [False, True])
@pytest.mark.parametrize("shape", [(24, 20, 16), (9, 7, 5, 6)])
def test_reported_residual_is_the_true_one(ts, shape, gen, update):
    """The residual the refinement reports (updated from the FP32 corrections
    by default, re-evaluated at every step with resid_update = 1) is the true
    residual of the returned X: equal to the oracle's up to the power-iteration
    estimate of ||A|| (2e-2 relative) and the rounding of the residual itself
    (1e-14: DF64 evaluation, 2^-48 per operation, or the FP32 update)."""
    p = synthetic.problem(36, shape, generalized=gen, force_blocks=[[n // 2 - 1] for n in shape])
    A = [to_dev(a) for a in p["A"]]
    info = ts.Info()
    if gen:
        X, st = ts.gtsylv_solve(A, [to_dev(c) for c in p["C"]], to_dev(p["B"]), precision=ts.TSYLV_FP32_REFINED,
                                resid_update=update, info=info)
    else:
        X, st = ts.tsylv_solve(A, to_dev(p["B"]), precision=ts.TSYLV_FP32_REFINED, resid_update=update, info=info)
    assert st == 0 and info.iterations >= 2
    Xg = to_host(X)
    R = p["B"] - oracle.apply(p["A"], Xg, p["C"])
    rho = np.linalg.norm(R) / (norm_op(p["A"], p["C"]) * np.linalg.norm(Xg))
    assert abs(info.resid - rho) <= 2e-2 * rho + 1e-14


@pytest.mark.parametrize("d,shape", [(2, (33, 17)), (3, (24, 20, 16)), (3, (40, 33, 17)), (4, (9, 7, 5, 6))])
@pytest.mark.parametrize("max_refine", [10, 2])
def test_pipelined_first_two_steps(ts, d, shape, max_refine):
    """fuse_step = 2 (the first two steps of the Laplace form in one pipelined
    launch) gives the result of separate steps bit for bit, with the same
    iteration count and reported residual."""
    p = synthetic.problem(41, shape, force_blocks=[[n // 2 - 1] if n >= 4 else [] for n in shape])
    A = [to_dev(a) for a in p["A"]]
    B = to_dev(p["B"])
    out = []
    for fuse in (3, 2):
        info = ts.Info()
        X, st = ts.tsylv_solve(A, B, precision=ts.TSYLV_FP32_REFINED, fuse_step=fuse, max_refine=max_refine,
                               info=info, check=False)
        out.append((X, st, info.iterations, info.resid))
    (X0, st0, it0, r0), (X2, st2, it2, r2) = out
    assert st0 == st2 and it0 == it2 and r0 == r2
    assert torch.equal(X0, X2)
    if max_refine >= 3:
        assert st2 == 0 and r2 <= 1e-12


def test_pipelined_steps_full_second_residual(ts):
    """With resid_update = 1 the second residual is re-evaluated in full after
    the pipelined launch, as separate steps do: still the same result."""
    shape = (24, 20, 16)
    p = synthetic.problem(43, shape)
    A = [to_dev(a) for a in p["A"]]
    B = to_dev(p["B"])
    X0, _ = ts.tsylv_solve(A, B, precision=ts.TSYLV_FP32_REFINED, fuse_step=3, resid_update=1)
    X2, _ = ts.tsylv_solve(A, B, precision=ts.TSYLV_FP32_REFINED, fuse_step=2, resid_update=1)
    assert torch.equal(X0, X2)


@pytest.mark.parametrize("fuse", [0, 2, 3])
@pytest.mark.parametrize("d,shape", [(1, (100,)), (2, (33, 17)), (3, (24, 20, 16)), (4, (9, 7, 5, 6))])
def test_fused_and_separate_steps(ts, d, shape, fuse):
    """The first refinement steps of the Laplace form chosen automatically
    (0), the first two pipelined in one launch (2) or as separate launches
    (3): same accuracy against the oracle."""
    p = synthetic.problem(37, shape, force_blocks=[[n // 2 - 1] if n >= 4 else [] for n in shape])
    Xo = oracle.solve_recursive(p["A"], p["B"], nmin=4)
    info = ts.Info()
    X, st = ts.tsylv_solve([to_dev(a) for a in p["A"]], to_dev(p["B"]), precision=ts.TSYLV_FP32_REFINED,
                           fuse_step=fuse, info=info)
    assert st == 0 and info.resid <= 1e-12 and 1 <= info.iterations <= 4
    assert rel_err(to_host(X), Xo) <= 1e-10
