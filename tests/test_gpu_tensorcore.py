"""TF32- and BF16-refined solves: the block updates of the low-precision
solve run on the tensor cores (mma.sync, TF32 or BF16 operands, FP32
accumulation), the residual and the correction of X stay FP64-accurate.

Parity with the CPU oracle, element by element: the refinement stops at a
relative residual rho <= 1e-12; the workloads' operators have condition
numbers of about 5-20, so the forward error is below 1e-10 (the tolerance
written here).  The d = 4 d-term workloads (64, 64, 64, 64) and
(128, 96, 64, 32) are compared in full, for every precision, against one
oracle solve each (computed in two worker processes started with 'spawn').
"""
import multiprocessing

import numpy as np
import pytest
import torch

import oracle
import synthetic
from tests.gpu_helpers import max_rel, oracle_recursive_job, rel_err, to_dev, to_host

pytestmark = pytest.mark.gpu
TOL = 1e-10
PRECS = ["tf32r", "bf16r"]


@pytest.fixture(scope="module")
def lib():
    import paper_1905_09539_gb300 as ts
    ts.load()
    return ts


def _prec(ts, name):
    return {"fp64": ts.TSYLV_FP64, "fp32r": ts.TSYLV_FP32_REFINED, "tf32r": ts.TSYLV_TF32_REFINED,
            "bf16r": ts.TSYLV_BF16_REFINED}[name]


def _te(d):
    return {1: 32, 2: 16, 3: 8, 4: 4}[d]


def _force(shape, te):
    return [[n // 2 - 1] if n > te and n >= 4 else [] for n in shape]


def _solve(ts, p, prec, **kw):
    A = [to_dev(a) for a in p["A"]]
    B = to_dev(p["B"])
    info = ts.Info()
    if p["C"] is not None:
        X, st = ts.gtsylv_solve(A, [to_dev(c) for c in p["C"]], B, precision=prec, info=info, check=False, **kw)
    else:
        X, st = ts.tsylv_solve(A, B, precision=prec, info=info, check=False, **kw)
    return X, st, info


CASES = [(1, (100,)), (2, (33, 17)), (2, (40, 40)), (3, (24, 20, 16)), (3, (40, 33, 17)), (4, (9, 7, 5, 6)),
         (4, (13, 11, 10, 9))]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("gen", [False, True])
@pytest.mark.parametrize("d,shape", CASES)
def test_tensorcore_refined_parity(lib, d, shape, gen, prec):
    """Several blocks per mode, ragged tails, 2x2 blocks across split points."""
    if gen and d == 1:
        pytest.skip("d = 1: both forms coincide")
    p = synthetic.problem(11, shape, generalized=gen, force_blocks=_force(shape, _te(d)))
    Xo = oracle.solve_recursive(p["A"], p["B"], p["C"], nmin=4)
    X, st, info = _solve(lib, p, _prec(lib, prec), max_refine=40)
    assert st == 0, lib.status_string(st)
    assert info.resid <= 1e-12 and info.iterations >= 2
    Xg = to_host(X)
    assert rel_err(Xg, Xo) <= TOL and max_rel(Xg, Xo) <= TOL


@pytest.mark.parametrize("prec", PRECS)
def test_tensorcore_deep_queue_dterm(lib, prec):
    """d-term form with more blocks (12 x 10 x 9 = 1080) than the persistent
    kernel has resident CTAs, 2x2 blocks across block boundaries."""
    shape = (96, 80, 72)
    p = synthetic.problem(3, shape, generalized=True, force_blocks=[[7, 31, 55], [15, 39], [23, 47]])
    Xo = oracle.solve_recursive(p["A"], p["B"], p["C"], nmin=4)
    X, st, info = _solve(lib, p, _prec(lib, prec), max_refine=40)
    assert st == 0 and info.resid <= 1e-12
    Xg = to_host(X)
    assert rel_err(Xg, Xo) <= TOL and max_rel(Xg, Xo) <= TOL


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("d,shape", [(2, (33, 17)), (3, (24, 20, 16)), (4, (9, 7, 5, 6))])
def test_tensorcore_pipelined_steps_bitwise(lib, d, shape, prec):
    """The pipelined first two steps (fuse_step = 2) give the result of
    separate steps (fuse_step = 3) bit for bit with tensor-core updates too."""
    p = synthetic.problem(41, shape, force_blocks=_force(shape, 2))
    out = []
    for fuse in (3, 2):
        X, st, info = _solve(lib, p, _prec(lib, prec), fuse_step=fuse, max_refine=40)
        out.append((X, st, info.iterations, info.resid))
    (X0, st0, it0, r0), (X2, st2, it2, r2) = out
    assert st0 == st2 == 0 and it0 == it2 and r0 == r2
    assert torch.equal(X0, X2)


def test_tensorcore_schedule_one_unsupported(lib):
    p = synthetic.problem(1, (9, 8, 7))
    _, st, _ = _solve(lib, p, lib.TSYLV_TF32_REFINED, schedule=1)
    from paper_1905_09539_gb300 import _lib
    assert st == _lib.TSYLV_EUNSUPPORTED


CONFIG3 = [(64, 64, 64, 64), (128, 96, 64, 32)]
_ORACLE3 = {}


def _oracle3():
    if not _ORACLE3:
        ctx = multiprocessing.get_context("spawn")
        with ctx.Pool(len(CONFIG3)) as pool:
            res = pool.map(oracle_recursive_job, [(0, s, True, 2) for s in CONFIG3])
        _ORACLE3.update(zip(CONFIG3, res))
    return _ORACLE3


@pytest.mark.slow
@pytest.mark.parametrize("prec", ["fp64", "fp32r", "tf32r", "bf16r"])
@pytest.mark.parametrize("shape", CONFIG3)
def test_dterm_d4_workloads_against_oracle(lib, shape, prec):
    """d = 4 d-term workloads, every precision, element by element against
    the oracle: FP64 to 1e-11, the refined solves to rho <= 1e-12 and 1e-10."""
    Xo = _oracle3()[shape]
    p = synthetic.problem(0, shape, generalized=True)
    X, st, info = _solve(lib, p, _prec(lib, prec), max_refine=40)
    assert st == 0, lib.status_string(st)
    tol = 1e-11 if prec == "fp64" else TOL
    if prec != "fp64":
        assert info.resid <= 1e-12
    Xg = to_host(X)
    assert rel_err(Xg, Xo) <= tol and max_rel(Xg, Xo) <= tol
