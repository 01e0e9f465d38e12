"""Batched solve of many independent equations (C ABI tsylv_solve_batched)."""
import ctypes

import torch

from . import _lib


def tsylv_solve_batched(problems, *, generalized=False, opts=None, check=True, stream=None, info=None, **kw):
    """problems: list of (A list, B[, C list]) with CUDA tensors.  Returns (X list, statuses)."""
    from . import TsylvError, _dims, _opts, _stream, empty_fortran, fortran, workspace
    lib = _lib.load()
    o = _opts(opts, kw)
    count = len(problems)
    ds, ns, offA, offX = [], [], [], []
    apool, cpool, bpool = [], [], []
    pa = px = 0
    dev = problems[0][1].device
    for pr in problems:
        A, B = pr[0], pr[1]
        C = pr[2] if generalized else None
        d = B.dim()
        ds.append(d)
        for mu in range(d):
            m = B.shape[mu]
            ns.append(m)
            offA.append(pa)
            apool.append(fortran(A[mu]).permute(1, 0).reshape(-1))
            if generalized:
                cpool.append(fortran(C[mu]).permute(1, 0).reshape(-1))
            pa += m * m
        offX.append(px)
        bpool.append(fortran(B).permute(*range(d - 1, -1, -1)).reshape(-1))
        px += B.numel()
    Ap = torch.cat(apool).contiguous()
    Cp = torch.cat(cpool).contiguous() if generalized else None
    Bp = torch.cat(bpool).contiguous()
    Xp = torch.empty_like(Bp)
    cd = (ctypes.c_int * count)(*ds)
    cn = (ctypes.c_int64 * len(ns))(*ns)
    coA = (ctypes.c_int64 * len(offA))(*offA)
    coX = (ctypes.c_int64 * len(offX))(*offX)
    nbytes = lib.tsylv_batched_workspace_bytes(count, cd, cn, 1 if generalized else 0, ctypes.byref(o))
    work = workspace(nbytes, dev)
    per = (ctypes.c_int * count)()
    inf = info if info is not None else _lib.Info()
    st = lib.tsylv_solve_batched(count, cd, cn, coA, coX, Ap.data_ptr(), Cp.data_ptr() if Cp is not None else None,
                                 Bp.data_ptr(), Xp.data_ptr(), work.data_ptr(), work.numel(), ctypes.byref(o), per,
                                 ctypes.byref(inf), _stream(stream))
    if check and st != 0:
        raise TsylvError(st, "tsylv_solve_batched")
    Xs = []
    for e, pr in enumerate(problems):
        B = pr[1]
        d = B.dim()
        flat = Xp[offX[e]:offX[e] + B.numel()]
        Xs.append(flat.reshape(tuple(B.shape[::-1])).permute(*range(d - 1, -1, -1)))
    return Xs, [per[i] for i in range(count)]
