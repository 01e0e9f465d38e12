"""Helpers shared by the GPU tests: numpy (oracle side) <-> torch CUDA (solver side)."""
import numpy as np
import torch


def to_dev(a):
    """Fortran-ordered numpy array -> CUDA tensor with the same (column-major) memory."""
    a = np.asfortranarray(a, dtype=np.float64)
    t = torch.from_numpy(a)
    assert t.stride() == tuple(int(s // 8) for s in a.strides)
    out = torch.empty_strided(t.shape, t.stride(), dtype=torch.float64, device="cuda")
    out.copy_(t)
    return out


def to_host(t):
    t = t.detach().cpu()
    return np.asfortranarray(t.numpy())


def rel_err(X, Xo):
    return float(np.linalg.norm(X - Xo) / np.linalg.norm(Xo))


def max_rel(X, Xo):
    return float(np.max(np.abs(X - Xo)) / np.max(np.abs(Xo)))


def norm_op(A, C=None):
    d = len(A)
    if C is None:
        return sum(np.linalg.norm(a, 2) for a in A)
    return sum(np.linalg.norm(A[mu], 2) * np.prod([np.linalg.norm(C[e], 2) for e in range(d) if e != mu])
               for mu in range(d))


def oracle_recursive_job(args):
    """O-B solve of a seeded problem in a worker process (started with the
    'spawn' method, so that no CUDA state is inherited): (seed, shape,
    generalized, nmin) -> X.  Used to compute large oracle results in
    parallel with each other."""
    import oracle
    import synthetic
    seed, shape, gen, nmin = args
    p = synthetic.problem(seed, shape, generalized=gen)
    return oracle.solve_recursive(p["A"], p["B"], p["C"], nmin=nmin)
