"""The seeded input recipe (synthetic.py) matches its stated distributions:
A_mu strictly upper N(0,1)/sqrt(n), diagonal U[1,2], 2x2 blocks [[a, b], [-b, a]]
with a ~ U[1,2], b ~ U[0.1,1] covering about 10% of the diagonal positions;
C_mu strictly upper N(0,1)/sqrt(n), diagonal U[1,2]; B, X* ~ N(0,1); batch
mode sizes one integer draw per mode from U{8..48}; everything reproducible
from the seed."""
import numpy as np

import synthetic


def test_quasi_triangular_structure_and_distributions():
    fracs, offs, diags, bs = [], [], [], []
    for seed in range(6):
        p = synthetic.problem(seed, (256, 256, 256), generalized=True)
        for A, starts in zip(p["A"], p["blocks"]):
            n = A.shape[0]
            assert np.all(np.tril(A, -2) == 0)
            sub = np.diag(A, -1)
            nz = set(np.nonzero(sub)[0].tolist())
            assert nz == set(starts)
            assert all(i + 1 not in nz for i in nz)  # no two adjacent subdiagonal entries
            for i in starts:
                a, b, c, e = A[i, i], A[i, i + 1], A[i + 1, i], A[i + 1, i + 1]
                assert a == e and c == -b and 1 <= a <= 2 and 0.1 <= b <= 1
                bs.append(b)
            fracs.append(2 * len(starts) / n)
            mask = np.triu(np.ones((n, n), dtype=bool), 1)
            for i in starts:
                mask[i, i + 1] = False
            offs.append(A[mask] * np.sqrt(n))
            single = [i for i in range(n) if i not in nz and i - 1 not in nz]
            diags.append(A[single, single])
        for Cm in p["C"]:
            n = Cm.shape[0]
            assert np.all(np.tril(Cm, -1) == 0)
            assert np.all((np.diag(Cm) >= 1) & (np.diag(Cm) <= 2))
    frac = np.mean(fracs)
    assert 0.07 <= frac <= 0.13, frac          # ~10% of the positions in 2x2 blocks
    off = np.concatenate(offs)
    assert abs(off.mean()) < 0.01 and abs(off.std() - 1) < 0.01
    dg = np.concatenate(diags)
    assert dg.min() >= 1 and dg.max() <= 2 and abs(dg.mean() - 1.5) < 0.02
    assert abs(np.mean(bs) - 0.55) < 0.05


def test_right_hand_sides_and_reproducibility():
    p = synthetic.problem(0, (64, 64, 64))
    q = synthetic.problem(0, (64, 64, 64))
    r = synthetic.problem(1, (64, 64, 64))
    assert np.array_equal(p["B"], q["B"]) and all(np.array_equal(a, b) for a, b in zip(p["A"], q["A"]))
    assert not np.array_equal(p["B"], r["B"])
    for X in (p["B"], p["Xstar"]):
        assert abs(X.mean()) < 0.01 and abs(X.std() - 1) < 0.01
        assert X.flags.f_contiguous


def test_batch_shapes():
    shapes = synthetic.batch_shapes(0)
    assert len(shapes) == 512 and all(len(s) == 3 for s in shapes)
    v = np.array(shapes).ravel()
    assert v.min() >= 8 and v.max() <= 48
    assert set(range(8, 49)) <= set(v.tolist())  # every size drawn
    assert abs(v.mean() - 28) < 1.0
    assert synthetic.batch_shapes(0) == shapes and synthetic.batch_shapes(1) != shapes
