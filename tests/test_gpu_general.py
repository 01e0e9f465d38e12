"""General (dense) coefficients on the GPU: the change-of-basis transform
(tsylv_transform) against mode products on the host, and the whole route of
Alg. 1 (host Schur / QZ reduction, GPU transforms, triangular GPU solve)
against the dense oracle.  Tolerances: transforms 1e-13 relative (dense FP64
products of orthogonal-size factors); solves 1e-10 (the FP64 solve's 1e-11
plus the two orthogonal transforms and the reduction's own backward error).
"""
import numpy as np
import pytest
import torch

import oracle
from tests.gpu_helpers import rel_err, to_dev, to_host
from tests.kron_helpers import mode_product

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ts():
    import paper_1905_09539_gb300 as ts
    ts.load()
    return ts


def _general(rng, n, shift=2.5):
    return np.asfortranarray(rng.standard_normal((n, n)) / np.sqrt(n) + shift * np.eye(n))


@pytest.mark.parametrize("shape", [(37,), (19, 23), (9, 7, 5), (5, 4, 6, 3), (1, 6, 4)])
@pytest.mark.parametrize("pattern", ["all", "trans", "skip"])
def test_transform_matches_mode_products(ts, shape, pattern):
    from paper_1905_09539_gb300.general import transform
    rng = np.random.default_rng(3)
    d = len(shape)
    X = np.asfortranarray(rng.standard_normal(shape))
    M = [np.asfortranarray(rng.standard_normal((n, n))) for n in shape]
    use = [True] * d if pattern != "skip" else [mu % 2 == 0 for mu in range(d)]
    tr = [pattern == "trans" and mu % 2 == 1 for mu in range(d)]
    Y = X
    for mu in range(d):
        if use[mu]:
            Y = mode_product(Y, M[mu].T if tr[mu] else M[mu], mu)
    Mg = [to_dev(m) if use[mu] else None for mu, m in enumerate(M)]
    Yg = transform(to_dev(X), Mg, trans=tr)
    assert rel_err(to_host(Yg), Y) <= 1e-13
    Xg = to_dev(X)
    Yi = transform(Xg, Mg, trans=tr, Y=Xg)  # in place
    assert Yi.data_ptr() == Xg.data_ptr()
    assert rel_err(to_host(Yi), Y) <= 1e-13


@pytest.mark.parametrize("gen", [False, True])
@pytest.mark.parametrize("shape", [(23, 17), (9, 8, 7), (6, 5, 4, 5)])
@pytest.mark.parametrize("precision", ["fp64", "fp32r"])
def test_solve_general_vs_dense_oracle(ts, gen, shape, precision):
    from paper_1905_09539_gb300.general import solve_general
    rng = np.random.default_rng(19)
    A = [_general(rng, n) for n in shape]
    C = [_general(rng, n, 2.0) for n in shape] if gen else None
    B = np.asfortranarray(rng.standard_normal(shape))
    Xo = oracle.solve_dense(A, B, C)
    prec = ts.TSYLV_FP64 if precision == "fp64" else ts.TSYLV_FP32_REFINED
    X, st = solve_general([to_dev(a) for a in A], to_dev(B), None if C is None else [to_dev(c) for c in C],
                          precision=prec)
    assert st == 0
    assert rel_err(to_host(X), Xo) <= 1e-10


def test_solve_general_reuses_reduction_and_buffer(ts):
    """A device-resident reduction and an output buffer: repeated solves give
    the same result in the same buffer."""
    from paper_1905_09539_gb300 import empty_fortran
    from paper_1905_09539_gb300.general import reduce_coefficients, solve_general
    rng = np.random.default_rng(23)
    shape = (12, 10, 9)
    A = [_general(rng, n) for n in shape]
    B = np.asfortranarray(rng.standard_normal(shape))
    Ad = [to_dev(a) for a in A]
    Bd = to_dev(B)
    red = reduce_coefficients(A, device=Bd.device)
    X = empty_fortran(shape, Bd.device)
    X1, st = solve_general(Ad, Bd, X=X, reduced=red)
    first = X1.clone()
    X2, st2 = solve_general(Ad, Bd, X=X, reduced=red)
    assert st == 0 and st2 == 0 and X1.data_ptr() == X.data_ptr() and X2.data_ptr() == X.data_ptr()
    assert torch.equal(first, X2)
    assert rel_err(to_host(X2), oracle.solve_dense(A, B)) <= 1e-10
