"""Coupled groups of the base case (products of 2x2 Schur blocks across the
modes, the perfect-shuffled diagonal blocks of Sec. 2.3), solved several
to a warp: 32 / S groups of S members per warp, ordered by class within an
anti-diagonal.  Modes made mostly of 2x2 blocks, with 1x1 blocks in between,
put groups of every class (2, 4, 8 and, for d = 4, 16 members) in the same
anti-diagonal and more groups of one class than one warp takes; compared with
the oracle element by element (1e-11 relative) in every form and precision
that has coupled groups, bit for bit across runs, and a singular group among
regular ones is reported.
"""
import numpy as np
import pytest
import torch

import oracle
import synthetic
from oracle import two_term
from tests.gpu_helpers import max_rel, rel_err, to_dev, to_host

pytestmark = pytest.mark.gpu
TOL = 1e-11


@pytest.fixture(scope="module")
def lib():
    import paper_1905_09539_gb300 as ts
    ts.load()
    return ts


def _pairs(n, skip_every):
    """2x2 starts covering a mode of size n, a 1x1 block after every
    `skip_every` pairs (so the group classes mix)."""
    out, i, k = [], 0, 0
    while i + 1 < n:
        if skip_every and k == skip_every:
            i += 1
            k = 0
            continue
        out.append(i)
        i += 2
        k += 1
    return out


SHAPES = [
    (2, (40, 36), [3, 0]),
    (3, (24, 20, 17), [3, 2, 0]),
    (3, (16, 16, 16), [0, 0, 0]),  # 4 x 4 x 4 groups of 8 per block: 12 on the middle anti-diagonals
    (4, (12, 10, 9, 8), [2, 0, 1, 0]),
]


def _precision(lib, name):
    return {"fp64": lib.TSYLV_FP64, "fp32r": lib.TSYLV_FP32_REFINED, "df64": lib.TSYLV_DF64}[name]


@pytest.mark.parametrize("prec", ["fp64", "fp32r", "df64"])
@pytest.mark.parametrize("gen", [False, True])
@pytest.mark.parametrize("d,shape,skip", SHAPES)
def test_packed_groups_parity(lib, d, shape, skip, gen, prec):
    force = [_pairs(n, s) for n, s in zip(shape, skip)]
    p = synthetic.problem(61, shape, generalized=gen, force_blocks=force)
    Xo = oracle.solve_recursive(p["A"], p["B"], p["C"], nmin=4)
    A = [to_dev(a) for a in p["A"]]
    B = to_dev(p["B"])
    kw = dict(precision=_precision(lib, prec), max_refine=40)
    out = []
    for _ in range(2):
        if gen:
            X, st = lib.gtsylv_solve(A, [to_dev(c) for c in p["C"]], B, **kw)
        else:
            X, st = lib.tsylv_solve(A, B, **kw)
        assert st == 0, lib.status_string(st)
        out.append(X)
    Xg = to_host(out[0])
    tol = 1e-10 if prec == "fp32r" else TOL
    assert rel_err(Xg, Xo) <= tol and max_rel(Xg, Xo) <= tol
    assert torch.equal(out[0], out[1])


@pytest.mark.parametrize("prec", ["fp64", "df64"])
@pytest.mark.parametrize("d,shape,skip", [s for s in SHAPES if s[0] >= 3])
def test_packed_groups_two_term(lib, d, shape, skip, prec):
    """The two-term form Eq. (3.1): its group systems A_1 x I + C x A_2 x ..."""
    force = [_pairs(n, s) for n, s in zip(shape, skip)]
    p = synthetic.problem(62, shape, generalized=True, force_blocks=force)
    A, C, B = p["A"], p["C"][0], p["B"]
    Xo = two_term.solve_recursive(A, C, B, nmin=4)
    X, st = lib.gsylvten_solve([to_dev(a) for a in A], to_dev(C), to_dev(B), precision=_precision(lib, prec))
    assert st == 0, lib.status_string(st)
    Xg = to_host(X)
    assert rel_err(Xg, Xo) <= TOL and max_rel(Xg, Xo) <= TOL


def _rot(a, b):
    """2x2 block with eigenvalues a +- ib."""
    return np.array([[a, b], [-b, a]])


@pytest.mark.parametrize("prec", ["fp64", "df64"])
def test_singular_group_among_packed(lib, prec):
    """One 8-member group whose Kronecker sum is singular (eigenvalue sum
    (1 + 2i) + (1 + 2i) + (-2 - 4i) = 0) among regular groups solved in the
    same warps: the solve reports TSYLV_ESINGULAR.  The blocks' entries are
    small powers of two, so the elimination is exact and its last pivot is an
    exact zero (an exactly singular matrix with other entries can leave a
    pivot of rounding size above the 16 eps threshold)."""
    shape = (16, 16, 16)
    force = [_pairs(16, 0)] * 3
    p = synthetic.problem(63, shape, force_blocks=force)
    A = [a.copy() for a in p["A"]]
    i = 4  # pair (4, 5) of every mode: an 8-member group in the first block
    A[0][i:i + 2, i:i + 2] = _rot(1.0, 2.0)
    A[1][i:i + 2, i:i + 2] = _rot(1.0, 2.0)
    A[2][i:i + 2, i:i + 2] = _rot(-2.0, 4.0)
    # the operator restricted to the group is singular (checked on the host)
    blk, I2 = [a[i:i + 2, i:i + 2] for a in A], np.eye(2)
    K = np.kron(np.kron(blk[0], I2), I2) + np.kron(np.kron(I2, blk[1]), I2) + np.kron(np.kron(I2, I2), blk[2])
    assert np.linalg.svd(K, compute_uv=False)[-1] < 1e-12
    _, st = lib.tsylv_solve([to_dev(a) for a in A], to_dev(p["B"]), precision=_precision(lib, prec), check=False)
    assert st == lib._lib.TSYLV_ESINGULAR
