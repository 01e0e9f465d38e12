"""Parity of the CUDA path with the CPU oracle (element by element).

Sizes span several blocks per mode and ragged tails; 2x2 Schur blocks are
placed across split points of the recursion.  Tolerance: 1e-11 relative
(Frobenius and max-entry) for the FP64 solve, as the FP64 path must agree
with the oracle to that relative error.
"""
import numpy as np
import pytest
import torch

import oracle
import synthetic
from tests.gpu_helpers import max_rel, rel_err, to_dev, to_host

pytestmark = pytest.mark.gpu
TOL = 1e-11

CASES = [
    (1, (1,)), (1, (37,)), (1, (100,)),
    (2, (16, 16)), (2, (33, 17)), (2, (5, 70)),
    (3, (8, 8, 8)), (3, (9, 8, 7)), (3, (24, 17, 13)), (3, (33, 30, 31)), (3, (1, 20, 9)),
    (4, (4, 4, 4, 4)), (4, (9, 7, 5, 6)), (4, (13, 11, 10, 9)),
]


def _split_force(shape, te):
    """2x2 blocks that straddle the first split point of each mode."""
    out = []
    for n in shape:
        if n > te and n >= 4:
            out.append([n // 2 - 1])
        else:
            out.append([])
    return out


def _te(d):
    return {1: 32, 2: 16, 3: 8, 4: 4}[d]


@pytest.fixture(scope="module")
def lib():
    import paper_1905_09539_gb300 as ts
    ts.load()
    return ts


@pytest.mark.parametrize("gen", [False, True])
@pytest.mark.parametrize("d,shape", CASES)
@pytest.mark.parametrize("seed", [0, 1])
def test_solve_parity(lib, d, shape, gen, seed):
    force = _split_force(shape, _te(d)) if seed == 1 else None
    p = synthetic.problem(seed, shape, generalized=gen, force_blocks=force)
    Xo = oracle.solve_recursive(p["A"], p["B"], p["C"], nmin=4)
    A = [to_dev(a) for a in p["A"]]
    B = to_dev(p["B"])
    if gen:
        C = [to_dev(c) for c in p["C"]]
        X, st = lib.gtsylv_solve(A, C, B)
    else:
        X, st = lib.tsylv_solve(A, B)
    assert st == 0
    Xg = to_host(X)
    assert rel_err(Xg, Xo) <= TOL
    assert max_rel(Xg, Xo) <= TOL


@pytest.mark.parametrize("gen", [False, True])
@pytest.mark.parametrize("d,shape", [(2, (19, 23)), (3, (17, 12, 9)), (3, (24, 24, 24)), (4, (7, 9, 5, 6))])
def test_transposed_parity(lib, d, shape, gen):
    p = synthetic.problem(5, shape, generalized=gen, force_blocks=_split_force(shape, _te(d)))
    Lo = oracle.solve_backsub(p["A"], p["B"], p["C"], transpose=True)
    A = [to_dev(a) for a in p["A"]]
    G = to_dev(p["B"])
    if gen:
        L, st = lib.gtsylv_solve_transposed(A, [to_dev(c) for c in p["C"]], G)
    else:
        L, st = lib.tsylv_solve_transposed(A, G)
    assert st == 0
    Lg = to_host(L)
    assert rel_err(Lg, Lo) <= TOL
    assert max_rel(Lg, Lo) <= TOL


def test_all_positions_in_2x2_blocks(lib):
    shape = (16, 10, 12)
    force = [list(range(0, n - 1, 2)) for n in shape]
    for gen in (False, True):
        p = synthetic.problem(7, shape, generalized=gen, force_blocks=force)
        Xo = oracle.solve_backsub(p["A"], p["B"], p["C"])
        A = [to_dev(a) for a in p["A"]]
        if gen:
            X, st = lib.gtsylv_solve(A, [to_dev(c) for c in p["C"]], to_dev(p["B"]))
        else:
            X, st = lib.tsylv_solve(A, to_dev(p["B"]))
        assert st == 0
        assert rel_err(to_host(X), Xo) <= TOL


def test_diagonal_closed_form(lib):
    rng = np.random.default_rng(3)
    shape = (20, 13, 9)
    a = [rng.uniform(1, 2, n) for n in shape]
    A = [np.asfortranarray(np.diag(v)) for v in a]
    B = np.asfortranarray(rng.standard_normal(shape))
    Xc = B / sum(np.meshgrid(*a, indexing="ij"))
    X, st = lib.tsylv_solve([to_dev(m) for m in A], to_dev(B))
    assert st == 0
    assert np.max(np.abs(to_host(X) - Xc) / np.abs(Xc)) <= 1e-14


def test_in_place(lib):
    p = synthetic.problem(2, (20, 18, 9))
    Xo = oracle.solve_recursive(p["A"], p["B"], nmin=4)
    B = to_dev(p["B"])
    X, st = lib.tsylv_solve([to_dev(a) for a in p["A"]], B, X=B)
    assert st == 0 and X.data_ptr() == B.data_ptr()
    assert rel_err(to_host(B), Xo) <= TOL


def test_repeat_calls_replay_graph(lib):
    p = synthetic.problem(4, (17, 16, 15), generalized=True)
    Xo = oracle.solve_recursive(p["A"], p["B"], p["C"], nmin=4)
    A = [to_dev(a) for a in p["A"]]
    C = [to_dev(c) for c in p["C"]]
    B = to_dev(p["B"])
    X = lib.empty_fortran(B.shape, B.device) if hasattr(lib, "empty_fortran") else None
    from paper_1905_09539_gb300 import empty_fortran
    X = empty_fortran(tuple(B.shape), B.device)
    for _ in range(3):
        X.zero_()
        lib.gtsylv_solve(A, C, B, X=X)
        assert rel_err(to_host(X), Xo) <= TOL
    X2, _ = lib.gtsylv_solve(A, C, B, use_graph=0)
    assert rel_err(to_host(X2), Xo) <= TOL


@pytest.mark.parametrize("split", [1, 2, 8])
def test_cluster_split_sizes_agree(lib, split):
    """Wavefront schedule: short wavefronts split over clusters of 1, 2, 8 CTAs."""
    p = synthetic.problem(6, (40, 33, 24), generalized=True)
    Xo = oracle.solve_recursive(p["A"], p["B"], p["C"], nmin=8)
    X, st = lib.gtsylv_solve([to_dev(a) for a in p["A"]], [to_dev(c) for c in p["C"]], to_dev(p["B"]), split=split,
                             schedule=1)
    assert st == 0
    assert rel_err(to_host(X), Xo) <= TOL


@pytest.mark.parametrize("gen", [False, True])
@pytest.mark.parametrize("d,shape", [(1, (100,)), (2, (33, 17)), (3, (24, 17, 13)), (3, (33, 30, 31)),
                                     (4, (13, 11, 10, 9))])
@pytest.mark.parametrize("precision", ["fp64", "fp32r"])
def test_schedules_agree_with_oracle(lib, d, shape, gen, precision):
    """The persistent dataflow schedule (default) and the wavefront schedule
    (automatic cluster split, and no split) all match the oracle; without a
    cluster split the wavefront schedule sums every block update in the same
    order as the persistent one, so those two agree to the last bit."""
    p = synthetic.problem(2, shape, generalized=gen, force_blocks=_split_force(shape, _te(d)))
    Xo = oracle.solve_recursive(p["A"], p["B"], p["C"], nmin=4)
    prec = lib.TSYLV_FP64 if precision == "fp64" else lib.TSYLV_FP32_REFINED
    A = [to_dev(a) for a in p["A"]]
    B = to_dev(p["B"])
    out = []
    for sched, split in ((0, 0), (1, 1), (1, 0)):
        if gen:
            X, st = lib.gtsylv_solve(A, [to_dev(c) for c in p["C"]], B, schedule=sched, split=split, precision=prec)
        else:
            X, st = lib.tsylv_solve(A, B, schedule=sched, split=split, precision=prec)
        assert st == 0
        assert rel_err(to_host(X), Xo) <= TOL
        out.append(X)
    if precision == "fp64":
        assert torch.equal(out[0], out[1])


@pytest.mark.parametrize("gen", [False, True])
@pytest.mark.parametrize("precision", ["fp64", "fp32r"])
def test_inverse_budget_overflow(lib, gen, precision):
    """Two modes made of 2x2 blocks throughout: every 8^3 block has 128
    four-member coupled groups, 2048 inverse entries, twice the budget of
    precomputed inverses; the rest are solved by in-step elimination.  The
    result matches the oracle and is the same, bit for bit, in every run."""
    shape = (16, 16, 12)
    pairs = list(range(0, 16, 2))
    p = synthetic.problem(47, shape, generalized=gen, force_blocks=[pairs, pairs, []], block_prob=0.0)
    Xo = oracle.solve_recursive(p["A"], p["B"], p["C"], nmin=4)
    prec = lib.TSYLV_FP64 if precision == "fp64" else lib.TSYLV_FP32_REFINED
    A = [to_dev(a) for a in p["A"]]
    C = [to_dev(c) for c in p["C"]] if gen else None
    B = to_dev(p["B"])
    out = []
    for _ in range(2):
        X, st = lib.gtsylv_solve(A, C, B, precision=prec) if gen else lib.tsylv_solve(A, B, precision=prec)
        assert st == 0
        out.append(X)
    assert rel_err(to_host(out[0]), Xo) <= (TOL if precision == "fp64" else 1e-10)
    assert torch.equal(out[0], out[1])


def test_bounded_wait_times_out_and_context_survives(lib):
    """Failure detection without a GPU fault: a persistent solve whose first
    block is withheld waits for a flag nothing sets; the bounded wait runs out
    (50 ms), the launch ends with TSYLV_ETIMEOUT read back on the host, and the
    next solve in the same context is correct."""
    import time
    t0 = time.perf_counter()
    st = lib.selftest_wait_timeout(0.05)
    dt = time.perf_counter() - t0
    assert st == lib._lib.TSYLV_ETIMEOUT
    assert dt < 30.0
    p = synthetic.problem(3, (20, 17, 9))
    Xo = oracle.solve_recursive(p["A"], p["B"], nmin=4)
    X, st = lib.tsylv_solve([to_dev(a) for a in p["A"]], to_dev(p["B"]))
    assert st == 0 and rel_err(to_host(X), Xo) <= TOL


def test_singular_reported(lib):
    # a1_i + a2_j + a3_k = 0 at one position: exactly singular
    shape = (9, 8, 7)
    p = synthetic.problem(8, shape)
    A = [a.copy() for a in p["A"]]
    A[0][3, 3] = -(A[1][2, 2] + A[2][4, 4])
    A[0][2, 3] = 0.0 if A[0][3, 2] == 0 else A[0][2, 3]
    _, st = lib.tsylv_solve([to_dev(a) for a in A], to_dev(p["B"]), check=False)
    assert st == lib._lib.TSYLV_ESINGULAR


def test_nonfinite_reported(lib):
    p = synthetic.problem(9, (10, 9, 8))
    B = p["B"].copy()
    B[5, 4, 3] = np.nan
    _, st = lib.tsylv_solve([to_dev(a) for a in p["A"]], to_dev(B), check=False)
    assert st == lib._lib.TSYLV_ENONFINITE


def test_bad_structure_rejected(lib):
    p = synthetic.problem(10, (10, 9, 8))
    A = [a.copy() for a in p["A"]]
    A[1][3, 2] = 0.5
    A[1][4, 3] = 0.5      # two consecutive subdiagonal entries
    _, st = lib.tsylv_solve([to_dev(a) for a in A], to_dev(p["B"]), check=False)
    assert st == -3


@pytest.mark.parametrize("prec", ["fp64", "fp32r"])
@pytest.mark.parametrize("shape,force", [
    # d = 3: 12 x 10 x 9 = 1080 blocks, more than the resident CTAs of the
    # persistent d-term kernel, so blocks wait on blocks of running CTAs
    ((96, 80, 72), [[7, 31, 55], [15, 39], [23, 47]]),
    # d = 4: 6 x 6 x 5 x 5 = 900 blocks, more than the d = 4 kernel's resident CTAs
    ((24, 24, 20, 20), [[3, 11], [7], [3, 15], [11]]),
])
def test_dterm_deep_queue_parity(lib, shape, force, prec):
    """d-term form in the deep-queue regime of the persistent schedule, 2x2
    blocks across block boundaries: element by element against O-B."""
    p = synthetic.problem(9, shape, generalized=True, force_blocks=force)
    Xo = oracle.solve_recursive(p["A"], p["B"], p["C"], nmin=4)
    A = [to_dev(a) for a in p["A"]]
    C = [to_dev(c) for c in p["C"]]
    prec_id = lib.TSYLV_FP64 if prec == "fp64" else lib.TSYLV_FP32_REFINED
    X, st = lib.gtsylv_solve(A, C, to_dev(p["B"]), precision=prec_id)
    assert st == 0
    Xg = to_host(X)
    tol = TOL if prec == "fp64" else 1e-10
    assert rel_err(Xg, Xo) <= tol
    assert max_rel(Xg, Xo) <= tol


@pytest.mark.parametrize("gen", [False, True])
def test_wait_limit_option(lib, gen):
    """opts.wait_ms only bounds the device-side waits: a solve with a longer
    limit (its own captured schedule) gives the default solve's result bit
    for bit."""
    p = synthetic.problem(2, (24, 20, 16), generalized=gen)
    A = [to_dev(a) for a in p["A"]]
    B = to_dev(p["B"])
    C = [to_dev(c) for c in p["C"]] if gen else None
    out = []
    for w in (2000, 30000):
        if gen:
            X, st = lib.gtsylv_solve(A, C, B, wait_ms=w)
        else:
            X, st = lib.tsylv_solve(A, B, wait_ms=w)
        assert st == 0
        out.append(X)
    assert torch.equal(out[0], out[1])


def _force_d5(shape):
    """A 2x2 block at the first index of every mode (a 32-member coupled group
    in the corner block) and one across the first tile boundary."""
    out = []
    for n in shape:
        f = [0]
        if n > 5:
            f.append(3)  # (3, 4) straddles the boundary at 4 of the 4-wide tiles
        out.append(f)
    return out


@pytest.mark.parametrize("prec", ["fp64", "fp32r", "tf32r"])
@pytest.mark.parametrize("shape", [(4, 4, 4, 4, 4), (9, 7, 6, 5, 6), (13, 9, 8, 7, 6)])
def test_d5_laplace_parity(lib, shape, prec):
    """d = 5, the Laplace form (the order of the paper's merged-mode sweeps):
    element by element against O-B, every precision."""
    p = synthetic.problem(31, shape, force_blocks=_force_d5(shape))
    Xo = oracle.solve_recursive(p["A"], p["B"], None, nmin=4)
    prec_id = {"fp64": lib.TSYLV_FP64, "fp32r": lib.TSYLV_FP32_REFINED, "tf32r": lib.TSYLV_TF32_REFINED}[prec]
    info = lib.Info()
    X, st = lib.tsylv_solve([to_dev(a) for a in p["A"]], to_dev(p["B"]), precision=prec_id, max_refine=40,
                            info=info)
    assert st == 0
    tol = TOL if prec == "fp64" else 1e-10
    Xg = to_host(X)
    assert rel_err(Xg, Xo) <= tol and max_rel(Xg, Xo) <= tol


def test_d5_transposed_and_schedules(lib):
    """d = 5: the transposed solve against O-A on A^T, and both block
    schedules (persistent and wavefront) bit for bit."""
    shape = (9, 8, 6, 5, 6)
    p = synthetic.problem(32, shape, force_blocks=_force_d5(shape))
    A = [to_dev(a) for a in p["A"]]
    B = to_dev(p["B"])
    Lo = oracle.solve_backsub(p["A"], p["B"], None, transpose=True)
    L, st = lib.tsylv_solve_transposed(A, B)
    assert st == 0 and rel_err(to_host(L), Lo) <= TOL
    X0, _ = lib.tsylv_solve(A, B, schedule=0)
    X1, _ = lib.tsylv_solve(A, B, schedule=1, split=1)
    assert torch.equal(X0, X1)


def test_d5_generalized_unsupported(lib):
    from paper_1905_09539_gb300 import _lib
    p = synthetic.problem(33, (4, 4, 4, 4, 4), generalized=True)
    _, st = lib.gtsylv_solve([to_dev(a) for a in p["A"]], [to_dev(c) for c in p["C"]], to_dev(p["B"]), check=False)
    assert st == _lib.TSYLV_EUNSUPPORTED
