"""Tile shapes (the recursion cutoff of every mode) of single solves.

The block partition of each mode is bounded by a leaf size (opts.nmin for
every mode, opts.leaf mode by mode); opts.nmin = -1 lets the autotuner pick
among its candidate shapes on the first call.  Whatever the shape, the
solution is the same up to rounding: element by element against the oracle
(FP64 1e-11, refined 1e-10).
"""
import numpy as np
import pytest
import torch

import oracle
import synthetic
from tests.gpu_helpers import max_rel, rel_err, to_dev, to_host

pytestmark = pytest.mark.gpu

# the autotuner's candidates: every mode TE, TE - 1, 3/4 TE, TE/2; TE/2 in the last mode only
CANDIDATES = {2: [(16, 16), (15, 15), (12, 12), (8, 8), (16, 8)],
              3: [(8, 8, 8), (7, 7, 7), (6, 6, 6), (4, 4, 4), (8, 8, 4)],
              4: [(4, 4, 4, 4), (3, 3, 3, 3), (2, 2, 2, 2), (4, 4, 4, 2)]}


@pytest.fixture(scope="module")
def lib():
    import paper_1905_09539_gb300 as ts
    ts.load()
    return ts


def _solve(ts, p, **kw):
    A = [to_dev(a) for a in p["A"]]
    B = to_dev(p["B"])
    info = ts.Info()
    if p["C"] is not None:
        X, st = ts.gtsylv_solve(A, [to_dev(c) for c in p["C"]], B, info=info, check=False, **kw)
    else:
        X, st = ts.tsylv_solve(A, B, info=info, check=False, **kw)
    return X, st, info


SHAPES = [(3, (37, 30, 23), leaf) for leaf in CANDIDATES[3] + [(2, 3, 7), (5, 5, 5), (4, 8, 8)]] + \
         [(4, (13, 11, 10, 9), leaf) for leaf in CANDIDATES[4] + [(3, 2, 4, 3)]]


@pytest.mark.parametrize("gen", [False, True])
@pytest.mark.parametrize("d,shape,leaf", SHAPES)
def test_fixed_tile_shape_parity(lib, d, shape, leaf, gen):
    p = synthetic.problem(13, shape, generalized=gen, force_blocks=[[n // 2 - 1, n // 3] for n in shape])
    Xo = oracle.solve_recursive(p["A"], p["B"], p["C"], nmin=4)
    X, st, info = _solve(lib, p, leaf=leaf)
    assert st == 0
    assert tuple(info.leaf[:d]) == leaf
    Xg = to_host(X)
    assert rel_err(Xg, Xo) <= 1e-11 and max_rel(Xg, Xo) <= 1e-11


@pytest.mark.parametrize("prec", ["fp32r", "tf32r"])
@pytest.mark.parametrize("leaf", [(4, 4, 4), (8, 8, 4), (6, 6, 6)])
def test_fixed_tile_shape_refined(lib, leaf, prec):
    p = synthetic.problem(14, (33, 28, 19), generalized=True, force_blocks=[[15], [13], [8]])
    Xo = oracle.solve_recursive(p["A"], p["B"], p["C"], nmin=4)
    precision = lib.TSYLV_FP32_REFINED if prec == "fp32r" else lib.TSYLV_TF32_REFINED
    X, st, info = _solve(lib, p, leaf=leaf, precision=precision, max_refine=40)
    assert st == 0 and info.resid <= 1e-12
    assert rel_err(to_host(X), Xo) <= 1e-10


@pytest.mark.parametrize("gen", [False, True])
@pytest.mark.parametrize("d,shape", [(3, (40, 36, 30)), (4, (12, 10, 9, 8)), (2, (70, 50))])
def test_autotuned_tile_shape(lib, d, shape, gen):
    """nmin = -1: the first call tunes (one timed solve per candidate), the
    second reuses the choice; both results agree with the oracle and with
    each other bit for bit."""
    p = synthetic.problem(15, shape, generalized=gen)
    Xo = oracle.solve_recursive(p["A"], p["B"], p["C"], nmin=4)
    X1, st1, i1 = _solve(lib, p, nmin=-1)
    X2, st2, i2 = _solve(lib, p, nmin=-1)
    assert st1 == 0 and st2 == 0
    assert tuple(i1.leaf[:d]) in CANDIDATES[d] and tuple(i2.leaf[:d]) == tuple(i1.leaf[:d])
    assert torch.equal(X1, X2)
    assert rel_err(to_host(X1), Xo) <= 1e-11


def test_autotune_in_place_takes_default(lib):
    """An in-place call (X == B) is not tuned: it takes the default shape and
    solves correctly."""
    shape = (29, 27, 25)
    p = synthetic.problem(16, shape)
    Xo = oracle.solve_recursive(p["A"], p["B"], None, nmin=4)
    A = [to_dev(a) for a in p["A"]]
    B = to_dev(p["B"])
    info = lib.Info()
    X, st = lib.tsylv_solve(A, B, X=B, nmin=-1, info=info)
    assert st == 0 and X.data_ptr() == B.data_ptr()
    assert tuple(info.leaf[:3]) == (8, 8, 8)
    assert rel_err(to_host(X), Xo) <= 1e-11
