"""The FP64 solve with its block updates on the FP64 tensor cores (DMMA,
opts.fp64_update = 2), d = 2 and 3, against the CPU oracle element by element,
and against the FMA variant (opts.fp64_update = 1).

Both variants skip the zero padding of short blocks (a boundary moved back at
a 2x2 Schur block, a ragged last block): 2x2 blocks are forced across split
points so that the skipped padding is exercised.  Tolerance as for the FP64
solve: 1e-11 relative (Frobenius and max-entry).
"""
import numpy as np
import pytest

import oracle
import synthetic
from tests.gpu_helpers import max_rel, rel_err, to_dev, to_host

pytestmark = pytest.mark.gpu
TOL = 1e-11

CASES = [(2, (16, 16)), (2, (33, 17)), (2, (5, 70)), (2, (47, 61)),
         (3, (8, 8, 8)), (3, (9, 8, 7)), (3, (24, 17, 13)), (3, (33, 30, 31)), (3, (1, 20, 9)), (3, (41, 3, 26))]


def _force(shape, te):
    """2x2 blocks across the first tile boundaries of every mode."""
    return [[k * te - 1 for k in range(1, 4) if k * te < n - 1] for n in shape]


@pytest.fixture(scope="module")
def lib():
    import paper_1905_09539_gb300 as ts
    ts.load()
    return ts


def _solve(lib, p, transposed=False, **kw):
    A = [to_dev(a) for a in p["A"]]
    B = to_dev(p["B"])
    if p["C"] is not None:
        C = [to_dev(c) for c in p["C"]]
        fn = lib.gtsylv_solve_transposed if transposed else lib.gtsylv_solve
        X, st = fn(A, C, B, **kw)
    else:
        fn = lib.tsylv_solve_transposed if transposed else lib.tsylv_solve
        X, st = fn(A, B, **kw)
    assert st == 0
    return to_host(X)


@pytest.mark.parametrize("gen", [False, True])
@pytest.mark.parametrize("d,shape", CASES)
@pytest.mark.parametrize("seed", [0, 1])
def test_dmma_parity(lib, d, shape, gen, seed):
    te = {2: 16, 3: 8}[d]
    p = synthetic.problem(seed, shape, generalized=gen, force_blocks=_force(shape, te) if seed else None)
    Xo = oracle.solve_recursive(p["A"], p["B"], p["C"], nmin=4)
    for upd in (2, 1):
        Xg = _solve(lib, p, fp64_update=upd)
        assert rel_err(Xg, Xo) <= TOL, upd
        assert max_rel(Xg, Xo) <= TOL, upd


@pytest.mark.parametrize("gen", [False, True])
@pytest.mark.parametrize("shape", [(19, 23), (17, 12, 9), (24, 24, 24)])
def test_dmma_transposed_parity(lib, shape, gen):
    te = {2: 16, 3: 8}[len(shape)]
    p = synthetic.problem(5, shape, generalized=gen, force_blocks=_force(shape, te))
    Lo = oracle.solve_backsub(p["A"], p["B"], p["C"], transpose=True)
    Lg = _solve(lib, p, transposed=True, fp64_update=2)
    assert rel_err(Lg, Lo) <= TOL
    assert max_rel(Lg, Lo) <= TOL


@pytest.mark.parametrize("gen", [False, True])
def test_dmma_deep_queue(lib, gen):
    """64^3: 9^3 blocks with the 2x2 structure of the recipe, more blocks than
    the resident CTAs, so blocks wait on blocks held by other running CTAs."""
    shape = (64, 64, 64)
    p = synthetic.problem(6, shape, generalized=gen, force_blocks=_force(shape, 8))
    Xo = oracle.solve_recursive(p["A"], p["B"], p["C"], nmin=8)
    Xg = _solve(lib, p, fp64_update=2)
    assert rel_err(Xg, Xo) <= TOL
    assert max_rel(Xg, Xo) <= TOL


@pytest.mark.parametrize("nmin", [4, 6])
def test_dmma_tile_shapes(lib, nmin):
    """Smaller leaf bounds leave most k steps and output tiles partly padded."""
    shape = (29, 22, 18)
    p = synthetic.problem(7, shape, generalized=True, force_blocks=_force(shape, nmin))
    Xo = oracle.solve_recursive(p["A"], p["B"], p["C"], nmin=4)
    Xg = _solve(lib, p, fp64_update=2, nmin=nmin)
    assert rel_err(Xg, Xo) <= TOL


def test_dmma_unsupported(lib):
    from paper_1905_09539_gb300 import _lib
    p4 = synthetic.problem(8, (5, 4, 6, 3))
    A = [to_dev(a) for a in p4["A"]]
    _, st = lib.tsylv_solve(A, to_dev(p4["B"]), fp64_update=2, check=False)
    assert st == _lib.TSYLV_EUNSUPPORTED
    p3 = synthetic.problem(8, (9, 8, 7))
    A = [to_dev(a) for a in p3["A"]]
    _, st = lib.tsylv_solve(A, to_dev(p3["B"]), fp64_update=2, schedule=1, check=False)
    assert st == _lib.TSYLV_EUNSUPPORTED
    X, st = lib.tsylv_solve(A, to_dev(p3["B"]), fp64_update=2, precision=_lib.TSYLV_FP32_REFINED)
    assert st == 0  # ignored by the refined precisions
