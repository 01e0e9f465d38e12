"""ctypes view of the C ABI in include/tsylv.h (libtsylv.so, built in-tree)."""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtsylv.so")

TSYLV_OK = 0
TSYLV_ESINGULAR = 1
TSYLV_ENONFINITE = 2
TSYLV_ENOCONV = 3
TSYLV_ECUDA = 4
TSYLV_ETIMEOUT = 5
TSYLV_EUNSUPPORTED = 6
TSYLV_ESCRATCH = 7

TSYLV_FP64 = 0
TSYLV_FP32_REFINED = 1
TSYLV_TF32_REFINED = 2
TSYLV_BF16_REFINED = 3
TSYLV_DF64 = 4

TSYLV_RESID_DF64 = 0
TSYLV_RESID_FP64 = 1


class Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("max_refine", ctypes.c_int), ("tol", ctypes.c_double),
                ("residual", ctypes.c_int), ("nmin", ctypes.c_int), ("split", ctypes.c_int),
                ("use_graph", ctypes.c_int), ("host_io", ctypes.c_int), ("timing", ctypes.c_int),
                ("schedule", ctypes.c_int), ("partition", ctypes.c_int), ("resid_update", ctypes.c_int),
                ("fuse_step", ctypes.c_int), ("wait_ms", ctypes.c_int), ("leaf", ctypes.c_int * 5),
                ("fp64_update", ctypes.c_int)]


class Info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("waves", ctypes.c_int), ("launches", ctypes.c_int),
                ("tiles", ctypes.c_int), ("resid", ctypes.c_double), ("norm_A", ctypes.c_double),
                ("flops", ctypes.c_double), ("t_total_ms", ctypes.c_double), ("t_waves_ms", ctypes.c_double),
                ("t_resid_ms", ctypes.c_double),
                ("batch_order", ctypes.c_int),
                ("batch_ctas_per_sm", ctypes.c_int),
                ("leaf", ctypes.c_int * 5)]

    def as_dict(self):
        return {k: (list(getattr(self, k)) if k == "leaf" else getattr(self, k)) for k, _ in self._fields_}


EXPORTS = [
    "tsylv_opts_default", "tsylv_status_string", "tsylv_workspace_bytes", "tsylv_solve", "gtsylv_solve",
    "tsylv_solve_transposed", "gtsylv_solve_transposed", "tsylv_residual", "tsylv_backward_workspace_bytes",
    "tsylv_backward", "tsylv_batched_workspace_bytes", "tsylv_solve_batched", "tsylv_last_error",
    "tsylv_solve_noalloc", "tsylv_residual_workspace_bytes", "tsylv_selftest_wait_timeout",
    "tsylv_transform", "tsylv_transform_workspace_bytes", "gsylvten_solve", "gsylvten_workspace_bytes",
    "ztsylv_solve", "zgtsylv_solve", "ztsylv_workspace_bytes", "tsylv_plan_create", "tsylv_plan_execute",
    "tsylv_plan_destroy",
]

_lib = None


def load(path=LIB_PATH):
    """Load libtsylv.so; raises if it has not been built (no fallback path exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libtsylv.so is missing: build it with `python -c 'import __graft_entry__ as g; "
                           "g.build()'` (the solver has no CPU fallback)")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    I = ctypes.c_int
    I64P = ctypes.POINTER(ctypes.c_int64)
    OP = ctypes.POINTER(Opts)
    IP = ctypes.POINTER(Info)
    S = ctypes.c_size_t
    lib.tsylv_opts_default.argtypes = [OP]
    lib.tsylv_opts_default.restype = None
    lib.tsylv_status_string.argtypes = [I]
    lib.tsylv_status_string.restype = ctypes.c_char_p
    lib.tsylv_last_error.argtypes = []
    lib.tsylv_last_error.restype = ctypes.c_char_p
    lib.tsylv_workspace_bytes.argtypes = [I, I64P, I, OP]
    lib.tsylv_workspace_bytes.restype = S
    lib.tsylv_solve.argtypes = [I, I64P, P, P, P, P, S, OP, IP, P]
    lib.gtsylv_solve.argtypes = [I, I64P, P, P, P, P, P, S, OP, IP, P]
    lib.tsylv_solve_transposed.argtypes = [I, I64P, P, P, P, P, S, OP, IP, P]
    lib.gtsylv_solve_transposed.argtypes = [I, I64P, P, P, P, P, P, S, OP, IP, P]
    lib.tsylv_residual.argtypes = [I, I64P, P, P, P, P, P, ctypes.POINTER(ctypes.c_double), P, S, OP, P]
    lib.tsylv_residual_workspace_bytes.argtypes = [I, I64P, I]
    lib.tsylv_residual_workspace_bytes.restype = S
    lib.tsylv_backward_workspace_bytes.argtypes = [I, I64P, I, OP]
    lib.tsylv_backward_workspace_bytes.restype = S
    lib.tsylv_backward.argtypes = [I, I64P, P, P, P, P, P, P, P, P, S, OP, IP, P]
    lib.tsylv_batched_workspace_bytes.argtypes = [I, ctypes.POINTER(I), I64P, I, OP]
    lib.tsylv_batched_workspace_bytes.restype = S
    lib.tsylv_solve_batched.argtypes = [I, ctypes.POINTER(I), I64P, I64P, I64P, P, P, P, P, P, S, OP,
                                        ctypes.POINTER(I), IP, P]
    lib.tsylv_solve_noalloc.argtypes = [I, I64P, P, P, P, OP, IP, P]
    lib.tsylv_solve_noalloc.restype = I
    lib.tsylv_selftest_wait_timeout.argtypes = [ctypes.c_longlong, P]
    lib.tsylv_selftest_wait_timeout.restype = I
    lib.tsylv_transform_workspace_bytes.argtypes = [I, I64P]
    lib.tsylv_transform_workspace_bytes.restype = S
    lib.tsylv_transform.argtypes = [I, I64P, P, ctypes.POINTER(I), P, P, P, S, P]
    lib.tsylv_transform.restype = I
    lib.gsylvten_workspace_bytes.argtypes = [I, I64P, OP]
    lib.gsylvten_workspace_bytes.restype = S
    lib.gsylvten_solve.argtypes = [I, I64P, P, P, P, P, P, S, OP, IP, P]
    lib.gsylvten_solve.restype = I
    lib.ztsylv_workspace_bytes.argtypes = [I, I64P, I, OP]
    lib.ztsylv_workspace_bytes.restype = S
    lib.ztsylv_solve.argtypes = [I, I64P, P, P, P, P, S, OP, IP, P]
    lib.ztsylv_solve.restype = I
    lib.zgtsylv_solve.argtypes = [I, I64P, P, P, P, P, P, S, OP, IP, P]
    lib.zgtsylv_solve.restype = I
    lib.tsylv_plan_create.argtypes = [ctypes.POINTER(P), I, I64P, P, P, I, P, S, OP, P]
    lib.tsylv_plan_create.restype = I
    lib.tsylv_plan_execute.argtypes = [P, P, P, P, S, P, P]
    lib.tsylv_plan_execute.restype = I
    lib.tsylv_plan_destroy.argtypes = [P]
    lib.tsylv_plan_destroy.restype = None
    for f in ("tsylv_solve", "gtsylv_solve", "tsylv_solve_transposed", "gtsylv_solve_transposed",
              "tsylv_residual", "tsylv_backward", "tsylv_solve_batched"):
        getattr(lib, f).restype = I
    _lib = lib
    return lib


def default_opts(**kw):
    o = Opts()
    load().tsylv_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError("unknown option %r" % k)
        if k == "leaf":
            v = (ctypes.c_int * 5)(*(list(v) + [0] * (5 - len(v))))
        setattr(o, k, v)
    return o


def status_string(s):
    return load().tsylv_status_string(int(s)).decode()


def last_error():
    return load().tsylv_last_error().decode()
