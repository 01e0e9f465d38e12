"""The paper's own generalized form, Sec. 3, Eq. (3.1):
    X x_1 A_1 + X x_1 C x_2 A_2 ... x_d A_d = B,
solved on the GPU by gsylvten_solve, element by element against the oracle
of that form (oracle/two_term.py: the recursion of Alg. 5, pinned on the CPU
against the assembled matrix Eq. (1.5) and the closed form).  2x2 blocks sit
across the split points in every mode, so coupled groups of up to 2^d members
appear.  Tolerance 1e-11 (FP64, as the other forms).
"""
import numpy as np
import pytest

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


def _problem(seed, shape, force=None):
    p = synthetic.problem(seed, shape, generalized=True, force_blocks=force)
    return p["A"], p["C"][0], p["B"]


def _te(d):
    return {2: 16, 3: 8, 4: 4}[d]


def _force(shape, te):
    return [[n // 2 - 1, te - 1] if n > te + 2 and n // 2 - 1 not in (te - 2, te, te - 1) else
            ([te - 1] if n > te else []) for n in shape]


def _solve(ts, A, C, B, **kw):
    info = ts.Info()
    X, st = ts.gsylvten_solve([to_dev(a) for a in A], to_dev(C), to_dev(B), info=info, check=False, **kw)
    return X, st, info


CASES = [(2, (33, 17)), (2, (40, 40)), (3, (9, 8, 7)), (3, (24, 20, 16)), (3, (37, 30, 23)), (4, (9, 7, 5, 6)),
         (4, (13, 11, 10, 9))]


@pytest.mark.parametrize("seed", [0, 1])
@pytest.mark.parametrize("d,shape", CASES)
def test_two_term_parity(lib, d, shape, seed):
    force = _force(shape, _te(d)) if seed == 1 else None
    A, C, B = _problem(40 + seed, shape, force)
    Xo = two_term.solve_recursive(A, C, B, nmin=4)
    X, st, info = _solve(lib, A, C, B)
    assert st == 0, lib.status_string(st)
    Xg = to_host(X)
    assert rel_err(Xg, Xo) <= TOL and max_rel(Xg, Xo) <= TOL
    # the equation itself, evaluated by mode products on the host
    R = B - two_term.apply(A, C, Xg)
    assert np.linalg.norm(R) <= 1e-13 * np.linalg.norm(B) * 10


def test_two_term_coupled_groups_every_mode(lib):
    """2x2 blocks at the same index of every mode: coupled groups of 2, 4
    and 8 members inside one block, and 2x2 blocks across block boundaries."""
    shape = (20, 19, 18)
    A, C, B = _problem(44, shape, [[0, 7, 12], [0, 7, 12], [0, 7, 12]])
    Xo = two_term.solve_recursive(A, C, B, nmin=4)
    X, st, _ = _solve(lib, A, C, B)
    assert st == 0
    assert rel_err(to_host(X), Xo) <= TOL


def test_two_term_deep_queue(lib):
    """More blocks (12 x 10 x 9) than resident CTAs of the persistent launch."""
    shape = (96, 80, 72)
    A, C, B = _problem(45, shape, [[7, 31, 55], [15, 39], [23, 47]])
    Xo = two_term.solve_recursive(A, C, B, nmin=8)
    X, st, _ = _solve(lib, A, C, B)
    assert st == 0
    Xg = to_host(X)
    assert rel_err(Xg, Xo) <= TOL and max_rel(Xg, Xo) <= TOL


def test_shifted_kronecker_case(lib):
    """A_1 = -lambda I: (A_d x ... x A_2 x C - lambda I) vec(X) = vec(B), Eq. (1.6)."""
    shape = (14, 11, 9)
    A, C, B = _problem(46, shape)
    lam = 0.75
    A = [np.asfortranarray(-lam * np.eye(shape[0]))] + list(A[1:])
    Xo = two_term.solve_recursive(A, C, B, nmin=4)
    X, st, _ = _solve(lib, A, C, B)
    assert st == 0
    assert rel_err(to_host(X), Xo) <= TOL


@pytest.mark.parametrize("leaf", [(8, 8, 8), (7, 7, 7), (6, 6, 6), (4, 4, 4), (8, 8, 4), (3, 5, 2)])
def test_two_term_tile_shapes(lib, leaf):
    shape = (29, 23, 19)
    A, C, B = _problem(47, shape, _force(shape, 8))
    Xo = two_term.solve_recursive(A, C, B, nmin=4)
    X, st, info = _solve(lib, A, C, B, leaf=leaf)
    assert st == 0 and tuple(info.leaf[:3]) == leaf
    assert rel_err(to_host(X), Xo) <= TOL


def test_two_term_repeat_and_in_place(lib):
    """Graph replay gives the same result bit for bit; X may equal B."""
    import torch
    shape = (21, 18, 15)
    A, C, B = _problem(48, shape)
    Ad = [to_dev(a) for a in A]
    Cd = to_dev(C)
    X1, _ = lib.gsylvten_solve(Ad, Cd, to_dev(B))
    X2, _ = lib.gsylvten_solve(Ad, Cd, to_dev(B))
    assert torch.equal(X1, X2)
    Bd = to_dev(B)
    X3, st = lib.gsylvten_solve(Ad, Cd, Bd, X=Bd)
    assert st == 0 and X3.data_ptr() == Bd.data_ptr() and torch.equal(X3, X1)


@pytest.mark.parametrize("d,shape", [(2, (33, 17)), (3, (24, 20, 16)), (3, (37, 30, 23)), (4, (13, 11, 10, 9))])
def test_two_term_df64(lib, d, shape):
    """The two-term form in double-float arithmetic (precision TSYLV_DF64),
    2x2 blocks across the split points, against the oracle at the FP64
    tolerance."""
    A, C, B = _problem(47, shape, _force(shape, _te(d)))
    Xo = two_term.solve_recursive(A, C, B, nmin=4)
    X, st, _ = _solve(lib, A, C, B, precision=lib.TSYLV_DF64)
    assert st == 0, lib.status_string(st)
    Xg = to_host(X)
    assert rel_err(Xg, Xo) <= TOL and max_rel(Xg, Xo) <= TOL


def test_two_term_df64_deep_queue(lib):
    shape = (96, 80, 72)
    A, C, B = _problem(45, shape, [[7, 31, 55], [15, 39], [23, 47]])
    Xo = two_term.solve_recursive(A, C, B, nmin=8)
    X, st, _ = _solve(lib, A, C, B, precision=lib.TSYLV_DF64)
    assert st == 0
    assert rel_err(to_host(X), Xo) <= TOL
