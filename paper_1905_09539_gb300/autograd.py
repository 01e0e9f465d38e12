"""torch.autograd.Function over the C ABI: forward = tsylv_solve / gtsylv_solve,
backward = tsylv_backward (transposed solve + masked gradient contractions)."""
import torch

from . import _lib


class _TsylvSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, opts_kw, recompute, B, *mats):
        from . import gtsylv_solve, tsylv_solve
        d = B.dim()
        A = list(mats[:d])
        C = list(mats[d:]) if len(mats) > d else None
        if C is None:
            X, _ = tsylv_solve(A, B, **opts_kw)
        else:
            X, _ = gtsylv_solve(A, C, B, **opts_kw)
        ctx.opts_kw = opts_kw
        ctx.recompute = recompute
        ctx.d = d
        ctx.gen = C is not None
        if recompute:
            # memory-saving mode: keep B, recompute X in backward
            ctx.save_for_backward(B, *mats)
        else:
            ctx.save_for_backward(X, *mats)
        return X

    @staticmethod
    def backward(ctx, dX):
        from . import gtsylv_solve, tsylv_backward, tsylv_solve
        saved = ctx.saved_tensors
        d = ctx.d
        mats = saved[1:]
        A = list(mats[:d])
        C = list(mats[d:]) if ctx.gen else None
        if ctx.recompute:
            B = saved[0]
            X = (gtsylv_solve(A, C, B, **ctx.opts_kw) if ctx.gen else tsylv_solve(A, B, **ctx.opts_kw))[0]
        else:
            X = saved[0]
        need_B = ctx.needs_input_grad[2]
        need_A = any(ctx.needs_input_grad[3:3 + d])
        need_C = ctx.gen and any(ctx.needs_input_grad[3 + d:])
        dB, dA, dC = tsylv_backward(A, X, dX.contiguous() if not dX.is_contiguous() else dX, C,
                                    want_dB=True, want_dA=need_A, want_dC=need_C, **ctx.opts_kw)
        grads = [None, None, dB if need_B else None]
        grads += list(dA) if dA is not None else [None] * d
        if ctx.gen:
            grads += list(dC) if dC is not None else [None] * d
        return tuple(grads)


def solve(A, B, C=None, *, precision=_lib.TSYLV_FP64, recompute=False, **opts):
    """Differentiable X = A^{-1}(B) (Laplace form, or the d-term generalized
    form when C is given).  Gradients flow to B, A_mu and C_mu; the gradient of
    A_mu is masked to its quasi-triangular pattern, that of C_mu to the upper
    triangle.  recompute=True stores B instead of X and re-solves in backward."""
    opts_kw = dict(opts)
    opts_kw["precision"] = precision
    mats = list(A) + (list(C) if C is not None else [])
    return _TsylvSolve.apply(opts_kw, recompute, B, *mats)
