"""Parity of the complex-triangular solves (ztsylv_solve / zgtsylv_solve)
with the complex CPU oracle, element by element.

Sizes span several blocks per mode and ragged tails, for d = 1..4 and both
the Laplace and the d-term forms.  At the full 256^3 size the oracle checks
sampled outputs -- the trailing box X[k:, k:, k:] of an upper triangular
problem solves the trailing sub-problem by itself -- and the residual of the
whole solution.  Tolerance: 1e-11 relative (Frobenius and max-entry), as for
the real FP64 solve.
"""
import numpy as np
import pytest
import scipy.linalg as sla
import torch

import oracle
import synthetic
from oracle import complex_tri as ct
from tests.gpu_helpers import max_rel, rel_err

pytestmark = pytest.mark.gpu
TOL = 1e-11

CASES = [
    (1, (1,)), (1, (37,)), (1, (100,)),
    (2, (16, 16)), (2, (33, 17)), (2, (5, 70)),
    (3, (8, 8, 8)), (3, (9, 8, 7)), (3, (24, 17, 13)), (3, (1, 20, 9)),
    (4, (4, 4, 4, 4)), (4, (9, 7, 5, 6)), (4, (13, 11, 10, 9)),
]


def to_dev_z(a):
    a = np.asfortranarray(a, dtype=np.complex128)
    t = torch.from_numpy(a)
    out = torch.empty_strided(t.shape, t.stride(), dtype=torch.complex128, device="cuda")
    out.copy_(t)
    return out


def to_host_z(t):
    return np.asfortranarray(t.detach().cpu().numpy())


@pytest.fixture(scope="module")
def lib():
    import paper_1905_09539_gb300 as ts
    ts.load()
    return ts


def _solve(lib, p, **kw):
    A = [to_dev_z(a) for a in p["A"]]
    C = None if p["C"] is None else [to_dev_z(c) for c in p["C"]]
    X, st = lib.ztsylv_solve(A, to_dev_z(p["B"]), C, **kw)
    assert st == 0
    return to_host_z(X)


@pytest.mark.parametrize("gen", [False, True])
@pytest.mark.parametrize("d,shape", CASES)
def test_complex_parity(lib, d, shape, gen):
    if gen and d == 1:
        pytest.skip("the d-term form of one mode is the Laplace form times a constant")
    p = synthetic.complex_problem(31, shape, generalized=gen)
    Xo = ct.solve_recursive(p["A"], p["B"], p["C"], nmin=4)
    Xg = _solve(lib, p)
    assert rel_err(Xg, Xo) <= TOL
    assert max_rel(Xg, Xo) <= TOL


@pytest.mark.parametrize("gen", [False, True])
def test_lower_triangle_never_read(lib, gen):
    """Entries below the diagonal of A_mu and C_mu are not part of the input."""
    shape = (21, 18, 11)
    p = synthetic.complex_problem(32, shape, generalized=gen)
    Xo = ct.solve_recursive(p["A"], p["B"], p["C"], nmin=4)
    rng = np.random.default_rng(5)
    junk = lambda M: M + np.tril(1e3 * (rng.standard_normal(M.shape) + 1j), -1)
    q = dict(p, A=[junk(a) for a in p["A"]], C=None if p["C"] is None else [junk(c) for c in p["C"]])
    Xg = _solve(lib, q)
    assert rel_err(Xg, Xo) <= TOL


@pytest.mark.parametrize("nmin", [2, 4, 8])
def test_complex_tile_shapes(lib, nmin):
    """Explicit recursion cutoffs choose other block shapes; the result does not change."""
    shape = (26, 19, 15)
    p = synthetic.complex_problem(33, shape, generalized=True)
    Xo = ct.solve_recursive(p["A"], p["B"], p["C"], nmin=4)
    Xg = _solve(lib, p, nmin=nmin)
    assert rel_err(Xg, Xo) <= TOL


@pytest.mark.parametrize("gen", [False, True])
def test_complex_schur_pipeline(lib, gen):
    """The route the paper's experiments take (Sec. 2.4): a real quasi-
    triangular problem, each coefficient reduced to complex Schur form (QZ for
    the d-term form), the right-hand side transformed, the complex triangular
    problem solved on the GPU, the solution transformed back -- against the
    real C oracle on the original problem."""
    shape = (40, 33, 28)
    p = synthetic.problem(34, shape, generalized=gen)
    T, S, Qh, Z = [], [], [], []
    for mu, a in enumerate(p["A"]):
        if gen:
            AA, BB, Q, ZZ = sla.qz(a, p["C"][mu], output="complex")
            T.append(np.triu(AA))
            S.append(np.triu(BB))
            Qh.append(Q.conj().T)
            Z.append(ZZ)
        else:
            t, u = sla.schur(a, output="complex")
            T.append(np.triu(t))
            Qh.append(u.conj().T)
            Z.append(u)
    Bt = p["B"].astype(complex)
    for mu in range(3):
        Bt = ct._mode(Bt, Qh[mu], mu)
    Xt = _solve(lib, {"A": T, "C": S if gen else None, "B": Bt})
    X = Xt
    for mu in range(3):
        X = ct._mode(X, Z[mu], mu)
    Xo = oracle.solve_recursive(p["A"], p["B"], p["C"], nmin=4)
    assert np.max(np.abs(X.imag)) <= 1e-11 * np.max(np.abs(Xo))
    assert rel_err(X.real, Xo) <= 1e-11


@pytest.mark.parametrize("gen", [False, True])
def test_complex_full_size_sampled(lib, gen):
    """256^3, the size the bench times: deep dataflow queue, every block of
    the partition in flight.  The trailing 20^3 box is checked element by
    element against the oracle's solve of the trailing sub-problem, the whole
    solution by its residual."""
    shape = (256, 256, 256)
    p = synthetic.complex_problem(35, shape, generalized=gen)
    Xg = _solve(lib, p)
    k = 236
    sub = (slice(k, None),) * 3
    As = [a[k:, k:] for a in p["A"]]
    Cs = None if p["C"] is None else [c[k:, k:] for c in p["C"]]
    Xs = ct.solve_recursive(As, p["B"][sub], Cs, nmin=5)
    assert rel_err(Xg[sub], Xs) <= TOL
    assert max_rel(Xg[sub], Xs) <= TOL
    R = p["B"] - ct.apply(p["A"], Xg, p["C"])
    nA = sum(np.linalg.norm(a, 2) for a in p["A"]) if not gen else \
        sum(np.linalg.norm(p["A"][mu], 2) * np.prod([np.linalg.norm(p["C"][e], 2) for e in range(3) if e != mu])
            for mu in range(3))
    assert np.linalg.norm(R) / (nA * np.linalg.norm(Xg)) <= 1e-14


def test_complex_info_and_timing(lib):
    from paper_1905_09539_gb300 import _lib
    p = synthetic.complex_problem(36, (48, 40, 36))
    inf = _lib.Info()
    A = [to_dev_z(a) for a in p["A"]]
    X, st = lib.ztsylv_solve(A, to_dev_z(p["B"]), info=inf, timing=1)
    assert st == 0
    assert inf.tiles > 0 and inf.flops > 0
    assert inf.t_total_ms > 0 and 0 < inf.t_waves_ms <= inf.t_total_ms
    Xo = ct.solve_recursive(p["A"], p["B"], None, nmin=4)
    assert rel_err(to_host_z(X), Xo) <= TOL
