"""Seeded synthetic inputs for the triangular tensor Sylvester solver.

This module only draws random numbers; it holds none of the method's
arithmetic.  Both the oracle tests and the CUDA-path tests/benchmarks take
their inputs from here, so the two sides see identical data.

Distributions (the experiments use randomly generated coefficients, Sec. 2.4;
the per-entry recipe below is fixed here):
  A_mu : strictly upper entries N(0,1)/sqrt(n), diagonal U[1,2]; walking
         i = 0..n-2, a 2x2 block [[a, b], [-b, a]] (eigenvalues a +- b i,
         a ~ U[1,2], b ~ U[0.1,1]) starts at i with probability 1/19 and the walk
         then skips to i+2.  The expected share of diagonal positions inside
         2x2 blocks is 2q/(1+q) = 10% for q = 1/19.
  C_mu : strictly upper entries N(0,1)/sqrt(n), diagonal U[1,2].
  B    : N(0,1).     X* (target for a loss): N(0,1).
Streams: numpy PCG64 children of SeedSequence(seed), spawned in the fixed order
A_1..A_d, C_1..C_d, B, X*.  All arrays are Fortran ordered (mode 1 fastest).
"""
import numpy as np

BLOCK_PROB = 1.0 / 19.0


def quasi_triangular(rng, n, block_prob=BLOCK_PROB, force_blocks=()):
    """Upper quasi-triangular n x n matrix; returns (A, list of 2x2 start indices)."""
    A = np.triu(rng.standard_normal((n, n)) / np.sqrt(n), 1)
    A[np.arange(n), np.arange(n)] = rng.uniform(1.0, 2.0, n)
    starts = []
    forced = set(force_blocks)
    i = 0
    while i < n - 1:
        u = rng.uniform()
        if i in forced or (not forced and u < block_prob):
            a = rng.uniform(1.0, 2.0)
            b = rng.uniform(0.1, 1.0)
            A[i, i] = a
            A[i + 1, i + 1] = a
            A[i, i + 1] = b
            A[i + 1, i] = -b
            starts.append(i)
            i += 2
        else:
            i += 1
    return np.asfortranarray(A), starts


def upper_triangular(rng, n):
    C = np.triu(rng.standard_normal((n, n)) / np.sqrt(n), 1)
    C[np.arange(n), np.arange(n)] = rng.uniform(1.0, 2.0, n)
    return np.asfortranarray(C)


def problem(seed, shape, generalized=False, force_blocks=None, block_prob=BLOCK_PROB):
    """Seeded problem of the given mode sizes.

    force_blocks: optional list (one entry per mode) of 2x2 start positions to
    place instead of the random walk (used by tests to put a 2x2 block across
    every split point).
    """
    d = len(shape)
    kids = np.random.SeedSequence(seed).spawn(2 * d + 2)
    A, blocks = [], []
    for mu in range(d):
        fb = () if force_blocks is None else force_blocks[mu]
        a, s = quasi_triangular(np.random.Generator(np.random.PCG64(kids[mu])), shape[mu],
                                block_prob=block_prob, force_blocks=fb)
        A.append(a)
        blocks.append(s)
    C = None
    if generalized:
        C = [upper_triangular(np.random.Generator(np.random.PCG64(kids[d + mu])), shape[mu])
             for mu in range(d)]
    rb = np.random.Generator(np.random.PCG64(kids[2 * d]))
    B = np.asfortranarray(rb.standard_normal(tuple(shape)))
    rx = np.random.Generator(np.random.PCG64(kids[2 * d + 1]))
    Xstar = np.asfortranarray(rx.standard_normal(tuple(shape)))
    return {"A": A, "C": C, "B": B, "Xstar": Xstar, "blocks": blocks, "shape": tuple(shape)}


def batch_shapes(seed, count=512, lo=8, hi=48, d=3):
    """Mode sizes of a batch of independent equations: one integer draw per mode, U{lo..hi}."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, 0xBA7C])))
    return [tuple(int(v) for v in rng.integers(lo, hi + 1, size=d)) for _ in range(count)]


def batch(seed, count=512, lo=8, hi=48, d=3, generalized=False):
    shapes = batch_shapes(seed, count, lo, hi, d)
    return [problem([seed, 1 + e], s, generalized=generalized) for e, s in enumerate(shapes)]


# ---- the complex-triangular variant (the coefficients of Sec. 2.4 after a
# complex Schur reduction): complex upper triangular A_mu whose diagonal holds
# the eigenvalues of the real recipe above -- real part U[1,2]; the pairs a +- b i
# of 2x2 blocks (walk as above, b ~ U[0.1,1]) as two conjugate diagonal entries --
# strictly upper entries (N(0,1) + i N(0,1)) / sqrt(2 n); C_mu complex upper
# triangular with diagonal U[1,2] + i U[-0.5,0.5] and the same strictly upper
# entries; B, X*: (N(0,1) + i N(0,1)) / sqrt(2).  Streams as problem().

def complex_triangular(rng, n, block_prob=BLOCK_PROB):
    """Complex upper triangular n x n matrix with the eigenvalue recipe above."""
    A = np.triu(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)), 1) / np.sqrt(2.0 * n)
    diag = rng.uniform(1.0, 2.0, n).astype(np.complex128)
    i = 0
    while i < n - 1:
        if rng.uniform() < block_prob:
            a = rng.uniform(1.0, 2.0)
            b = rng.uniform(0.1, 1.0)
            diag[i], diag[i + 1] = a + 1j * b, a - 1j * b
            i += 2
        else:
            i += 1
    A[np.arange(n), np.arange(n)] = diag
    return np.asfortranarray(A)


def complex_upper(rng, n):
    C = np.triu(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)), 1) / np.sqrt(2.0 * n)
    C[np.arange(n), np.arange(n)] = rng.uniform(1.0, 2.0, n) + 1j * rng.uniform(-0.5, 0.5, n)
    return np.asfortranarray(C)


def complex_problem(seed, shape, generalized=False):
    """Seeded complex-triangular problem of the given mode sizes."""
    d = len(shape)
    kids = np.random.SeedSequence(seed).spawn(2 * d + 2)
    A = [complex_triangular(np.random.Generator(np.random.PCG64(kids[mu])), shape[mu]) for mu in range(d)]
    C = None
    if generalized:
        C = [complex_upper(np.random.Generator(np.random.PCG64(kids[d + mu])), shape[mu]) for mu in range(d)]
    rb = np.random.Generator(np.random.PCG64(kids[2 * d]))
    B = np.asfortranarray((rb.standard_normal(tuple(shape)) + 1j * rb.standard_normal(tuple(shape))) / np.sqrt(2.0))
    return {"A": A, "C": C, "B": B, "shape": tuple(shape)}
