"""Structural pins from the printed merge examples (Sec. 2.3 and Sec. 3.3).

The merged coefficients and their perfect-shuffle permutations printed in the
paper fix (i) the Kronecker order of the merge, (ii) the reading n1 = 4,
n2 = 3 of the example, and (iii) that after the shuffle every diagonal block
is a coupled group of size prod(s_mu) <= 4 -- the groups that the
back-substitution of the oracle (and the base case of the solver) solves as
small dense systems.
"""
import os

import numpy as np

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    rows = [l.split() for l in open(os.path.join(GOLD, name)) if l.strip() and not l.startswith("#")]
    return np.array(rows, dtype=int)


def _patterns():
    A1 = np.array([[1, 1, 1, 1], [0, 1, 1, 1], [0, 1, 1, 1], [0, 0, 0, 1]])
    A2 = np.array([[1, 1, 1], [0, 1, 1], [0, 1, 1]])
    rng = np.random.default_rng(0)
    # generic values on the pattern, so no accidental cancellation
    return A1 * rng.uniform(1, 2, A1.shape), A2 * rng.uniform(1, 2, A2.shape)


def _shuffle_last8():
    # rows 4..11 ordered as (i1, i2) with i1 = 0..3 fast, i2 = 1..2 slow;
    # the perfect shuffle makes i2 the fast index
    perm = list(range(4))
    for i1 in range(4):
        for i2 in (1, 2):
            perm.append(i1 + 4 * i2)
    return np.array(perm)


def test_laplace_merge_pattern():
    A1, A2 = _patterns()
    Ap = np.kron(np.eye(3), A1) + np.kron(A2, np.eye(4))
    assert np.array_equal((Ap != 0).astype(int), _load("merge_laplace.txt"))
    P = _shuffle_last8()
    assert np.array_equal((Ap[np.ix_(P, P)] != 0).astype(int), _load("merge_laplace_shuffled.txt"))


def test_generalized_merge_pattern():
    A1, A2 = _patterns()
    Ap = np.kron(A2, A1)
    assert np.array_equal((Ap != 0).astype(int), _load("merge_generalized.txt"))
    P = _shuffle_last8()
    assert np.array_equal((Ap[np.ix_(P, P)] != 0).astype(int), _load("merge_generalized_shuffled.txt"))


def _diag_blocks(pattern):
    """Finest partition into consecutive diagonal blocks making the matrix block upper triangular."""
    n = pattern.shape[0]
    cuts, start = [], 0
    for e in range(1, n + 1):
        if e == n or not pattern[e:, start:e].any():
            # check nothing below in columns [start, e)
            if not pattern[e:, :e].any():
                cuts.append(e - start)
                start = e
    return cuts


def test_shuffled_groups_are_products_of_block_sizes():
    # A_1 blocks (1, 2, 1), A_2 blocks (1, 2): the coupled groups of the merged
    # mode are the Cartesian products; in A_2's 2x2 block they have sizes
    # 1*2, 2*2, 1*2 = 2, 4, 2 -- the diagonal blocks printed after the shuffle.
    pat = _load("merge_laplace_shuffled.txt")
    blocks = _diag_blocks(pat)
    assert blocks == [1, 2, 1, 2, 4, 2]
    assert max(blocks) <= 4
    pat_g = _load("merge_generalized_shuffled.txt")
    assert _diag_blocks(pat_g) == [1, 2, 1, 2, 4, 2]
