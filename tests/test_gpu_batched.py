"""Batched persistent solve (tsylv_solve_batched) on the GPU.

Every equation of a batch must equal its own single solve (1e-12 relative,
the batch runs the same block partition, updates and base case) and the
oracle (1e-11).  Batches follow the batching workload: independent d = 3
equations with every n_mu drawn uniformly from {8, ..., 48}.
"""
import numpy as np
import pytest
import torch

import oracle
import synthetic
from tests.gpu_helpers import rel_err, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import paper_1905_09539_gb300 as ts
    ts.load()
    return ts


def _problems(ps, gen):
    out = []
    for p in ps:
        A = [to_dev(a) for a in p["A"]]
        B = to_dev(p["B"])
        out.append((A, B, [to_dev(c) for c in p["C"]]) if gen else (A, B))
    return out


def _single(lib, pr, gen):
    if gen:
        return lib.gtsylv_solve(pr[0], pr[2], pr[1])[0]
    return lib.tsylv_solve(pr[0], pr[1])[0]


@pytest.mark.parametrize("gen", [False, True])
def test_batch_small_vs_single_and_oracle(lib, gen):
    ps = synthetic.batch(5, count=24, lo=8, hi=20)
    ps = [synthetic.problem([5, 100 + i], p["shape"], generalized=gen,
                            force_blocks=[[n // 2 - 1] for n in p["shape"]] if i % 3 == 0 else None)
          for i, p in enumerate(ps)]
    prs = _problems(ps, gen)
    info = lib.Info()
    Xs, st = lib.tsylv_solve_batched(prs, generalized=gen, info=info)
    assert all(s == 0 for s in st)
    assert info.launches >= 4
    for p, pr, X in zip(ps, prs, Xs):
        Xo = oracle.solve_recursive(p["A"], p["B"], p["C"], nmin=4)
        Xs1 = to_host(_single(lib, pr, gen))
        Xb = to_host(X)
        assert rel_err(Xb, Xs1) <= 1e-12
        assert rel_err(Xb, Xo) <= 1e-11


def test_batch_mixed_orders(lib):
    shapes = [(37,), (5, 70), (16, 16), (9, 8, 7), (24, 17, 13), (4, 4, 4, 4), (9, 7, 5, 6), (1,), (1, 20, 9)]
    ps = [synthetic.problem([6, i], s, force_blocks=[[n // 2 - 1] if n >= 4 else [] for n in s])
          for i, s in enumerate(shapes)]
    prs = _problems(ps, False)
    Xs, st = lib.tsylv_solve_batched(prs)
    assert all(s == 0 for s in st)
    for p, X in zip(ps, Xs):
        Xo = oracle.solve_backsub(p["A"], p["B"])
        assert rel_err(to_host(X), Xo) <= 1e-11


def test_batch_count_one_and_fixed_grid(lib):
    p = synthetic.problem(7, (33, 30, 31), force_blocks=[[15], [14], [15]])
    prs = _problems([p], False)
    Xo = oracle.solve_backsub(p["A"], p["B"])
    for split in (0, 1, 2):
        Xs, st = lib.tsylv_solve_batched(prs, split=split)
        assert st == [0]
        assert rel_err(to_host(Xs[0]), Xo) <= 1e-11


def test_batch_graph_replay_and_eager(lib):
    ps = synthetic.batch(8, count=16, lo=8, hi=30)
    prs = _problems(ps, False)
    X1, _ = lib.tsylv_solve_batched(prs)
    X2, _ = lib.tsylv_solve_batched(prs)
    X3, _ = lib.tsylv_solve_batched(prs, use_graph=0)
    for a, b, c in zip(X1, X2, X3):
        assert torch.equal(a, b)
        assert torch.equal(a, c)


def test_batch_bad_structure(lib):
    ps = synthetic.batch(9, count=4, lo=8, hi=12)
    prs = _problems(ps, False)
    A = prs[2][0][1].clone()
    A[2, 1] = 0.5
    A[3, 2] = 0.5  # two adjacent sub-diagonal entries
    prs[2] = ([prs[2][0][0], A, prs[2][0][2]], prs[2][1])
    with pytest.raises(lib.TsylvError) as ei:
        lib.tsylv_solve_batched(prs)
    assert ei.value.status == -6


def test_batch_singular_status(lib):
    ps = synthetic.batch(10, count=6, lo=8, hi=12)
    # equation 4: a1_i + a2_j + a3_k = 0 at one position (no 2x2 blocks)
    q = synthetic.problem([10, 4], (9, 8, 7), block_prob=0.0)
    A = [a.copy() for a in q["A"]]
    A[0][3, 3] = -(A[1][2, 2] + A[2][4, 4])
    ps[4] = {"A": A, "B": q["B"], "C": None}
    prs = _problems(ps, False)
    Xs, st = lib.tsylv_solve_batched(prs, check=False)
    assert st[4] == lib._lib.TSYLV_ESINGULAR
    assert all(s == 0 for i, s in enumerate(st) if i != 4)


@pytest.mark.parametrize("gen", [False, True])
def test_batch_workload_512(lib, gen):
    """512 equations, n_mu ~ U{8..48}: each equals its single solve; a sample
    of 12 equations against the oracle."""
    ps = synthetic.batch(0, count=512, generalized=gen)
    prs = _problems(ps, gen)
    Xs, st = lib.tsylv_solve_batched(prs, generalized=gen)
    assert all(s == 0 for s in st)
    worst = 0.0
    for pr, X in zip(prs, Xs):
        worst = max(worst, rel_err(to_host(X), to_host(_single(lib, pr, gen))))
    assert worst <= 1e-12, worst
    rng = np.random.default_rng(11)
    for i in rng.choice(512, size=12, replace=False):
        p = ps[int(i)]
        Xo = oracle.solve_recursive(p["A"], p["B"], p["C"], nmin=4)
        assert rel_err(to_host(Xs[int(i)]), Xo) <= 1e-11


@pytest.mark.parametrize("gen", [False, True])
def test_batch_refined_small(lib, gen):
    """FP32-refined batch: every equation reaches rel. residual <= 1e-12 and
    matches the oracle to 1e-10 (the refinement's accuracy, not FP64 parity)."""
    ps = synthetic.batch(12, count=20, lo=8, hi=24)
    ps = [synthetic.problem([12, 200 + i], p["shape"], generalized=gen,
                            force_blocks=[[n // 2 - 1] for n in p["shape"]] if i % 4 == 0 else None)
          for i, p in enumerate(ps)]
    prs = _problems(ps, gen)
    info = lib.Info()
    Xs, st = lib.tsylv_solve_batched(prs, generalized=gen, precision=lib.TSYLV_FP32_REFINED, info=info)
    assert all(s == 0 for s in st)
    assert 2 <= info.iterations <= 4 and info.resid <= 1e-12
    for p, X in zip(ps, Xs):
        Xo = oracle.solve_recursive(p["A"], p["B"], p["C"], nmin=4)
        assert rel_err(to_host(X), Xo) <= 1e-10


@pytest.mark.parametrize("gen", [False, True])
def test_batch_refined_workload_512(lib, gen):
    ps = synthetic.batch(0, count=512, generalized=gen)
    prs = _problems(ps, gen)
    X64, st64 = lib.tsylv_solve_batched(prs, generalized=gen)
    info = lib.Info()
    X32, st32 = lib.tsylv_solve_batched(prs, generalized=gen, precision=lib.TSYLV_FP32_REFINED, info=info)
    assert all(s == 0 for s in st64) and all(s == 0 for s in st32)
    assert info.resid <= 1e-12
    worst = max(rel_err(to_host(a), to_host(b)) for a, b in zip(X32, X64))
    assert worst <= 1e-10, worst


def test_batch_refined_mixed_orders_unsupported(lib):
    shapes = [(9, 8, 7), (5, 6)]
    ps = [synthetic.problem([13, i], s) for i, s in enumerate(shapes)]
    with pytest.raises((lib.TsylvError, ValueError)):
        lib.tsylv_solve_batched(_problems(ps, False), precision=lib.TSYLV_FP32_REFINED)


def test_batch_in_place_first_call_tuned(lib):
    """X_pool == B_pool on the first call of a new batch: the autotuner's
    timing runs must leave B untouched (each equation against the oracle)."""
    ps = synthetic.batch(17, count=20, lo=8, hi=24)
    prs = _problems(ps, False)
    pools = lib.BatchPools(prs)
    info = lib.Info()
    st = pools.solve(info=info, inplace=True)
    assert all(s == 0 for s in st)
    for p, X in zip(ps, pools.solutions()):
        Xo = oracle.solve_recursive(p["A"], p["B"], None, nmin=4)
        assert rel_err(to_host(X), Xo) <= 1e-11


SHAPE_CANDIDATES = {3: [(8, 8, 8), (7, 7, 7), (6, 6, 6), (4, 4, 4), (8, 8, 4)],
                    2: [(16, 16), (15, 15), (12, 12), (8, 8), (16, 8)]}


@pytest.mark.parametrize("gen", [False, True])
def test_batch_tuned_tile_shape(lib, gen):
    """The batch autotuner picks a tile shape among its candidates; every
    equation agrees with the oracle."""
    ps = synthetic.batch(19, count=40, lo=8, hi=40)
    ps = [synthetic.problem([19, 200 + i], p["shape"], generalized=gen) for i, p in enumerate(ps)]
    info = lib.Info()
    Xs, st = lib.tsylv_solve_batched(_problems(ps, gen), generalized=gen, info=info)
    assert all(s == 0 for s in st)
    assert tuple(info.leaf[:3]) in SHAPE_CANDIDATES[3]
    for p, X in zip(ps, Xs):
        assert rel_err(to_host(X), oracle.solve_recursive(p["A"], p["B"], p["C"], nmin=4)) <= 1e-11


@pytest.mark.parametrize("leaf", [(8, 8, 8), (7, 7, 7), (6, 6, 6), (4, 4, 4), (8, 8, 4), (2, 3, 5)])
@pytest.mark.parametrize("prec", ["fp64", "fp32r"])
def test_batch_fixed_tile_shape(lib, leaf, prec):
    """Every tile shape the tuner can pick (and an odd one), fixed through
    opts.leaf, FP64 and FP32-refined: each equation against the oracle."""
    ps = synthetic.batch(23, count=12, lo=8, hi=30)
    ps = [synthetic.problem([23, 300 + i], p["shape"], force_blocks=[[n // 2 - 1] for n in p["shape"]])
          for i, p in enumerate(ps)]
    info = lib.Info()
    precision = lib.TSYLV_FP64 if prec == "fp64" else lib.TSYLV_FP32_REFINED
    Xs, st = lib.tsylv_solve_batched(_problems(ps, False), info=info, leaf=leaf, precision=precision)
    assert all(s == 0 for s in st)
    tol = 1e-11 if prec == "fp64" else 1e-10
    for p, X in zip(ps, Xs):
        assert rel_err(to_host(X), oracle.solve_recursive(p["A"], p["B"], None, nmin=4)) <= tol


def test_batch_with_d5_equations(lib):
    """A batch mixing orders 3, 4 and 5 (the Laplace form; one persistent
    launch per order): each equation against the oracle."""
    shapes = [(12, 9, 10), (6, 5, 7, 6), (5, 4, 6, 5, 4), (9, 7, 5, 6, 4), (20, 13, 9)]
    ps = [synthetic.problem([37, i], s, force_blocks=[[0] for _ in s]) for i, s in enumerate(shapes)]
    Xs, st = lib.tsylv_solve_batched(_problems(ps, False))
    assert all(s == 0 for s in st)
    for p, X in zip(ps, Xs):
        assert rel_err(to_host(X), oracle.solve_recursive(p["A"], p["B"], None, nmin=4)) <= 1e-11


@pytest.mark.parametrize("gen", [False, True])
def test_batch_df64(lib, gen):
    """The double-float batch: every equation against the oracle (1e-11, the
    FP64 parity tolerance) and against its own double-float single solve;
    mixed orders d = 1..4, 2x2 blocks across split points."""
    shapes = [(37,), (5, 70), (16, 16), (9, 8, 7), (24, 17, 13), (9, 7, 5, 6), (1, 20, 9), (30, 22, 18)]
    if gen:
        shapes = [s for s in shapes if len(s) >= 2]
    ps = [synthetic.problem([14, i], s, generalized=gen, force_blocks=[[n // 2 - 1] if n >= 4 else [] for n in s])
          for i, s in enumerate(shapes)]
    prs = _problems(ps, gen)
    Xs, st = lib.tsylv_solve_batched(prs, generalized=gen, precision=lib.TSYLV_DF64)
    assert all(s == 0 for s in st)
    for p, pr, X in zip(ps, prs, Xs):
        Xo = oracle.solve_recursive(p["A"], p["B"], p["C"], nmin=4)
        assert rel_err(to_host(X), Xo) <= 1e-11
        if gen:
            Xs1 = lib.gtsylv_solve(pr[0], pr[2], pr[1], precision=lib.TSYLV_DF64)[0]
        else:
            Xs1 = lib.tsylv_solve(pr[0], pr[1], precision=lib.TSYLV_DF64)[0]
        assert rel_err(to_host(X), to_host(Xs1)) <= 1e-12


def test_batch_df64_workload_512(lib):
    ps = synthetic.batch(0, count=512)
    prs = _problems(ps, False)
    X64, st64 = lib.tsylv_solve_batched(prs)
    Xdf, stdf = lib.tsylv_solve_batched(prs, precision=lib.TSYLV_DF64)
    assert all(s == 0 for s in st64) and all(s == 0 for s in stdf)
    worst = max(rel_err(to_host(a), to_host(b)) for a, b in zip(Xdf, X64))
    assert worst <= 1e-12, worst
