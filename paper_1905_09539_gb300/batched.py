"""Batched solve of many independent equations (C ABI tsylv_solve_batched)."""
import ctypes

import torch

from . import _lib


class BatchPools:
    """Column-major pools of a batch: A (and C) matrices, B, X, with the host
    offset tables of the C ABI.  Built once; solve() may be called many times."""

    def __init__(self, problems, generalized=False):
        from . import fortran
        self.count = len(problems)
        self.generalized = generalized
        self.shapes = []
        ds, ns, offA, offX = [], [], [], []
        apool, cpool, bpool = [], [], []
        pa = px = 0
        for pr in problems:
            A, B = pr[0], pr[1]
            C = pr[2] if generalized else None
            d = B.dim()
            ds.append(d)
            self.shapes.append(tuple(B.shape))
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
        self.A = torch.cat(apool).contiguous()
        self.C = torch.cat(cpool).contiguous() if generalized else None
        self.B = torch.cat(bpool).contiguous()
        self.X = torch.empty_like(self.B)
        self.offX = offX
        self.unknowns = px
        self.c_d = (ctypes.c_int * self.count)(*ds)
        self.c_n = (ctypes.c_int64 * len(ns))(*ns)
        self.c_offA = (ctypes.c_int64 * len(offA))(*offA)
        self.c_offX = (ctypes.c_int64 * len(offX))(*offX)
        self.per = (ctypes.c_int * self.count)()

    def solve(self, *, opts=None, check=True, stream=None, info=None, inplace=False, **kw):
        """Solve every equation into self.X (inplace: into the B pool, which
        then becomes self.X); returns the list of statuses."""
        from . import TsylvError, _opts, _stream, workspace
        lib = _lib.load()
        o = _opts(opts, kw)
        nbytes = lib.tsylv_batched_workspace_bytes(self.count, self.c_d, self.c_n, 1 if self.generalized else 0,
                                                   ctypes.byref(o))
        if nbytes == 0:
            raise ValueError("tsylv_solve_batched: invalid shapes or unsupported precision")
        work = workspace(nbytes, self.B.device)
        inf = info if info is not None else _lib.Info()
        st = lib.tsylv_solve_batched(self.count, self.c_d, self.c_n, self.c_offA, self.c_offX, self.A.data_ptr(),
                                     self.C.data_ptr() if self.C is not None else None, self.B.data_ptr(),
                                     (self.B if inplace else self.X).data_ptr(), work.data_ptr(), work.numel(),
                                     ctypes.byref(o), self.per, ctypes.byref(inf), _stream(stream))
        if inplace:
            self.X = self.B
        if check and st != 0:
            raise TsylvError(st, "tsylv_solve_batched")
        return [self.per[i] for i in range(self.count)]

    def solutions(self):
        """Views of self.X as the column-major solution tensors."""
        Xs = []
        for off, shape in zip(self.offX, self.shapes):
            d = len(shape)
            n = 1
            for s in shape:
                n *= s
            Xs.append(self.X[off:off + n].reshape(tuple(shape[::-1])).permute(*range(d - 1, -1, -1)))
        return Xs


def tsylv_solve_batched(problems, *, generalized=False, opts=None, check=True, stream=None, info=None, **kw):
    """problems: list of (A list, B[, C list]) with CUDA tensors.  Returns (X list, statuses)."""
    pools = BatchPools(problems, generalized)
    st = pools.solve(opts=opts, check=check, stream=stream, info=info, **kw)
    return pools.solutions(), st
