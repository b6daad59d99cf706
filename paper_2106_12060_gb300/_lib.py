"""ctypes binding of libgbcca.so (include/gbcca.h).  Argument marshalling only:
every computation runs in the library's CUDA kernels.  Loading fails loudly
when the library has not been built; there is no fallback path."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgbcca.so")

BF16, FP32, FP64 = 0, 1, 2
COUNTSKETCH, SRHT, IDENTITY, EXACT = 0, 1, 2, 3
OK, ERR_INVALID_ARG, ERR_UNSUPPORTED, ERR_OOM, ERR_NOT_SPD, ERR_MAXITER, ERR_TIMEOUT, ERR_CUDA, ERR_STATE = (
    0, -1, -2, -3, -4, -5, -6, -7, -8)
Q_SKETCH_X, Q_SKETCH_Y, Q_R_X, Q_R_Y, Q_WARM_U, Q_WARM_V, Q_HISTORY, Q_CLASS_MEANS, Q_RITZ = range(9)


class Options(C.Structure):
    _fields_ = [
        ("sketch", C.c_int32),
        ("s", C.c_int64),
        ("seed", C.c_uint64),
        ("max_iter", C.c_int32),
        ("gtol", C.c_double),
        ("refine", C.c_int32),
        ("warm_start", C.c_int32),
        ("check_every", C.c_int32),
        ("time_passes", C.c_int32),
        ("graphs", C.c_int32),
        ("rtol", C.c_double),
        ("tensor_cores", C.c_int32),
        ("warm_iters", C.c_int32),
        ("wait_cycles", C.c_int64),
        ("retraction", C.c_int32),
    ]


class ServerOptions(C.Structure):
    _fields_ = [
        ("hbm_budget", C.c_int64),
        ("max_active", C.c_int32),
        ("tick_iters", C.c_int32),
        ("graphs", C.c_int32),
    ]


class Request(C.Structure):
    _fields_ = [
        ("kind", C.c_int32),
        ("dtype", C.c_int32),
        ("n", C.c_int64),
        ("dx", C.c_int32),
        ("dy", C.c_int32),
        ("k", C.c_int32),
        ("n_classes", C.c_int32),
        ("lambda_x", C.c_double),
        ("lambda_y", C.c_double),
        ("X", C.c_void_p),
        ("ldx", C.c_int64),
        ("Y", C.c_void_p),
        ("ldy", C.c_int64),
        ("labels", C.c_void_p),
        ("opt", Options),
    ]


class RequestTimes(C.Structure):
    _fields_ = [
        ("submit_s", C.c_double),
        ("admit_s", C.c_double),
        ("finish_s", C.c_double),
        ("device_bytes", C.c_int64),
    ]


class BatchOptions(C.Structure):
    _fields_ = [
        ("clusters", C.c_int32),
        ("graphs", C.c_int32),
        ("batch_iters", C.c_int32),
    ]


class BatchReport(C.Structure):
    _fields_ = [
        ("iterations", C.c_int32),
        ("clusters", C.c_int32),
        ("batched_plans", C.c_int32),
        ("reserved", C.c_int32),
        ("batched_pass_ms", C.c_double),
        ("batched_pass_bytes", C.c_double),
    ]


class Info(C.Structure):
    _fields_ = [
        ("iters", C.c_int32),
        ("passes", C.c_int32),
        ("status", C.c_int32),
        ("stalled", C.c_int32),
        ("grad_norm", C.c_double),
        ("grad_norm0", C.c_double),
        ("objective", C.c_double),
        ("pass_ms", C.c_double),
        ("pass_count", C.c_int32),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


# name -> (restype, argtypes)
SIGNATURES = {
    "gbcca_default_options": (C.c_int, [C.POINTER(Options)]),
    "cca_plan": (C.c_int, [C.POINTER(C.c_void_p), C.c_int64, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                           C.POINTER(Options)]),
    "cca_precondition": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_double,
                                   C.c_double, C.c_void_p, C.c_void_p, C.c_void_p]),
    "cca_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p,
                            C.POINTER(Info), C.c_void_p]),
    "lda_plan": (C.c_int, [C.POINTER(C.c_void_p), C.c_int64, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                           C.POINTER(Options)]),
    "lda_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_double, C.c_void_p, C.c_double,
                            C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(Info), C.c_void_p]),
    "gbcca_fused_pass": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                   C.c_void_p]),
    "gbcca_query_size": (C.c_int64, [C.c_void_p, C.c_int32]),
    "gbcca_query": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p]),
    "gbcca_sketch_draws": (C.c_int, [C.c_int32, C.c_int64, C.c_int64, C.c_uint64, C.c_void_p, C.c_void_p,
                                     C.c_void_p]),
    "gbcca_sketch_gram_noalloc": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64, C.c_int32, C.c_double, C.c_void_p,
                                            C.c_void_p]),
    "gbcca_sketch_gram_noalloc_max_d": (C.c_int32, []),
    "gbcca_default_batch_options": (C.c_int, [C.POINTER(BatchOptions)]),
    "gbcca_batch_create": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.c_int32,
                                     C.POINTER(BatchOptions)]),
    "gbcca_batch_solve": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                    C.POINTER(C.c_void_p), C.POINTER(Info), C.POINTER(BatchReport), C.c_void_p]),
    "gbcca_batch_fused_pass": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                         C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.c_void_p]),
    "gbcca_batch_destroy": (None, [C.c_void_p]),
    "gbcca_default_server_options": (C.c_int, [C.POINTER(ServerOptions)]),
    "gbcca_server_create": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(ServerOptions)]),
    "gbcca_server_submit": (C.c_int, [C.c_void_p, C.POINTER(Request), C.POINTER(C.c_int64)]),
    "gbcca_server_step": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.c_void_p]),
    "gbcca_server_state": (C.c_int, [C.c_void_p, C.c_int64]),
    "gbcca_server_result": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(Info),
                                      C.POINTER(RequestTimes)]),
    "gbcca_server_destroy": (None, [C.c_void_p]),
    "gbcca_launch_count": (C.c_int64, []),
    "gbcca_plan_destroy": (None, [C.c_void_p]),
    "gbcca_status_string": (C.c_char_p, [C.c_int]),
    "gbcca_last_error": (C.c_char_p, []),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libgbcca.so (raises OSError if it is missing or does not load)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError(f"{path} is missing: build it with paper_2106_12060_gb300.build.build()")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class GbccaError(RuntimeError):
    def __init__(self, code: int, where: str):
        lib = load()
        msg = lib.gbcca_last_error().decode(errors="replace")
        super().__init__(f"{where}: {lib.gbcca_status_string(code).decode()} ({code}): {msg}")
        self.code = code


def check(code: int, where: str, allow=(OK,)):
    if code not in allow:
        raise GbccaError(code, where)
    return code
