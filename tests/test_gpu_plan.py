"""Solve plans (tsylv_plan_create / _execute / _destroy): repeated FP64
solves queued without host synchronisation.

An execution runs the same kernels on the same partition as tsylv_solve, so
its solution must equal tsylv_solve's bit for bit; both are compared with the
CPU oracle as well (1e-11 relative, the FP64 parity tolerance).  Also checked:
several executions queued back to back before one synchronisation, new
coefficient values with the plan's 2x2 structure, a changed structure
(status -3 on the device), a singular diagonal (status 1), the transposed
equation, the wavefront schedule and the DMMA block updates.
"""
import numpy as np
import pytest
import torch

import oracle
import synthetic
from tests.gpu_helpers import max_rel, rel_err, to_dev, to_host

pytestmark = pytest.mark.gpu
TOL = 1e-11


@pytest.fixture(scope="module")
def lib():
    import paper_1905_09539_gb300 as ts
    ts.load()
    return ts


def _direct(lib, A, C, B, transposed=False, **kw):
    if C is None:
        fn = lib.tsylv_solve_transposed if transposed else lib.tsylv_solve
        X, st = fn(A, B, **kw)
    else:
        fn = lib.gtsylv_solve_transposed if transposed else lib.gtsylv_solve
        X, st = fn(A, C, B, **kw)
    assert st == 0
    return X


@pytest.mark.parametrize("gen", [False, True])
@pytest.mark.parametrize("shape", [(37,), (33, 17), (24, 17, 13), (64, 64, 64), (9, 7, 5, 6)])
def test_plan_matches_solve_and_oracle(lib, shape, gen):
    if gen and len(shape) == 1:
        pytest.skip("one mode: the d-term form is the Laplace form")
    p = synthetic.problem(41, shape, generalized=gen, force_blocks=[[n // 2 - 1] if n > 8 else [] for n in shape])
    A = [to_dev(a) for a in p["A"]]
    C = [to_dev(c) for c in p["C"]] if gen else None
    B = to_dev(p["B"])
    plan = lib.SolvePlan(A, C)
    X, status = plan.solve(B)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    Xd = _direct(lib, A, C, B)
    assert torch.equal(X, Xd)
    Xo = oracle.solve_recursive(p["A"], p["B"], p["C"], nmin=4)
    assert rel_err(to_host(X), Xo) <= TOL
    assert max_rel(to_host(X), Xo) <= TOL
    plan.close()


def test_plan_back_to_back(lib):
    """Four right-hand sides queued before a single synchronisation."""
    shape = (40, 36, 28)
    p = synthetic.problem(42, shape, generalized=True)
    A = [to_dev(a) for a in p["A"]]
    C = [to_dev(c) for c in p["C"]]
    plan = lib.SolvePlan(A, C)
    rng = np.random.default_rng(3)
    Bs = [np.asfortranarray(rng.standard_normal(shape)) for _ in range(4)]
    outs = [plan.solve(to_dev(b)) for b in Bs]
    torch.cuda.synchronize()
    for b, (X, status) in zip(Bs, outs):
        assert int(status.item()) == 0
        Xo = oracle.solve_recursive(p["A"], b, p["C"], nmin=4)
        assert rel_err(to_host(X), Xo) <= TOL


def test_plan_new_values_same_structure(lib):
    """Coefficient values changed in place between executions (structure kept)."""
    shape = (30, 26, 20)
    p = synthetic.problem(43, shape)
    A = [to_dev(a) for a in p["A"]]
    B = to_dev(p["B"])
    plan = lib.SolvePlan(A)
    X1, s1 = plan.solve(B)
    torch.cuda.synchronize()
    for a in A:
        a.mul_(1.5)  # same nonzero pattern
    X2, s2 = plan.solve(B)
    torch.cuda.synchronize()
    assert int(s1.item()) == 0 and int(s2.item()) == 0
    Xo = oracle.solve_recursive([1.5 * a for a in p["A"]], p["B"], None, nmin=4)
    assert rel_err(to_host(X2), Xo) <= TOL
    assert rel_err(to_host(X1) / 1.5, Xo) <= TOL


def test_plan_structure_change_reported(lib):
    """A new nonzero on a subdiagonal that the plan holds as zero: status -3."""
    shape = (20, 18, 16)
    p = synthetic.problem(44, shape, block_prob=0.0)
    A = [to_dev(a) for a in p["A"]]
    B = to_dev(p["B"])
    plan = lib.SolvePlan(A)
    _, s0 = plan.solve(B)
    torch.cuda.synchronize()
    assert int(s0.item()) == 0
    A[1][5, 4] = 0.25
    _, s1 = plan.solve(B)
    torch.cuda.synchronize()
    assert int(s1.item()) == -3
    A[1][5, 4] = 0.0
    X2, s2 = plan.solve(B)
    torch.cuda.synchronize()
    assert int(s2.item()) == 0
    Xo = oracle.solve_recursive(p["A"], p["B"], None, nmin=4)
    assert rel_err(to_host(X2), Xo) <= TOL


def test_plan_singular_status(lib):
    shape = (12, 10)
    p = synthetic.problem(45, shape, block_prob=0.0)
    A = [to_dev(a) for a in p["A"]]
    A[0][3, 3] = 1.0
    A[1][7, 7] = -1.0  # the diagonal entry a1_33 + a2_77 of unknown (3, 7) is zero
    plan = lib.SolvePlan(A)
    _, status = plan.solve(to_dev(p["B"]))
    torch.cuda.synchronize()
    assert int(status.item()) == 1


@pytest.mark.parametrize("gen", [False, True])
def test_plan_transposed(lib, gen):
    shape = (21, 17, 12)
    p = synthetic.problem(46, shape, generalized=gen, force_blocks=[[9], [7], [5]])
    A = [to_dev(a) for a in p["A"]]
    C = [to_dev(c) for c in p["C"]] if gen else None
    G = to_dev(p["B"])
    plan = lib.SolvePlan(A, C, transposed=True)
    L, status = plan.solve(G)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    assert torch.equal(L, _direct(lib, A, C, G, transposed=True))
    Lo = oracle.solve_backsub(p["A"], p["B"], p["C"], transpose=True)
    assert rel_err(to_host(L), Lo) <= TOL


@pytest.mark.parametrize("kw", [{"schedule": 1}, {"fp64_update": 2}, {"nmin": 6}, {"precision": 4}])
def test_plan_options(lib, kw):
    shape = (33, 29, 25)
    p = synthetic.problem(47, shape, generalized=True)
    A = [to_dev(a) for a in p["A"]]
    C = [to_dev(c) for c in p["C"]]
    B = to_dev(p["B"])
    plan = lib.SolvePlan(A, C, **kw)
    X, status = plan.solve(B)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    assert torch.equal(X, _direct(lib, A, C, B, **kw))
    Xo = oracle.solve_recursive(p["A"], p["B"], p["C"], nmin=4)
    assert rel_err(to_host(X), Xo) <= TOL
