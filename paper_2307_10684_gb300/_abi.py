"""ctypes declarations mirroring include/adr.h."""
from __future__ import annotations

import ctypes
import os
from functools import reduce

_PKG = os.path.dirname(os.path.abspath(__file__))
library_path = os.path.join(_PKG, "_build", "libadr_gb300.so")

ADR_OK, ADR_EINVAL, ADR_ENOMEM, ADR_ECUDA, ADR_EUNSUPPORTED, ADR_ETIMEOUT, ADR_ENUMERIC, \
    ADR_EBUSY = range(8)
SCHNAKENBERG, FHN, BRUSSELATOR, NO_REACTION, FHN_RHO, DIB = range(6)
ETD2RKDS, LAWSON2B = range(2)
STATE_AUTO, STATE_PLAIN, STATE_COMPENSATED = range(3)
FP64, FP32, TF32X3, BF16X3 = range(4)

c_int32, c_int64, c_double, c_void_p = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p


class AdrProblem(ctypes.Structure):
    _fields_ = [("d", c_int32), ("model", c_int32), ("precision", c_int32), ("scheme", c_int32),
                ("n", c_int64 * 3), ("lo", c_double * 3), ("hi", c_double * 3),
                ("diff", c_double * 2), ("adv", (c_double * 3) * 2), ("params", c_double * 16),
                ("tau", c_double), ("state", c_int32), ("reserved", c_int32)]


class AdrStats(ctypes.Structure):
    _fields_ = [("launches", c_int64), ("steps", c_int64), ("timing", c_int32),
                ("nkernels", c_int32), ("device_error", c_int32), ("shared_matrices", c_int32),
                ("name", (ctypes.c_char * 32) * 16),
                ("count", c_int64 * 16), ("ms", c_double * 16), ("flops", c_double * 16),
                ("bytes", c_double * 16)]


class AdrTuning(ctypes.Structure):
    _fields_ = [("kernel", c_int32), ("reserved", c_int32 * 7)]


class AdrTerm(ctypes.Structure):
    _fields_ = [("comp", c_int32), ("pow", c_int32 * 4), ("coef", c_double)]


class AdrGeneralProblem(ctypes.Structure):
    _fields_ = [("d", c_int32), ("m", c_int32), ("precision", c_int32), ("nterms", c_int32),
                ("n", c_int64 * 3), ("A", (ctypes.POINTER(c_double) * 3) * 4),
                ("terms", ctypes.POINTER(AdrTerm)), ("tau", c_double)]


class AdrPlan(ctypes.c_void_p):
    pass


# name -> (restype, argtypes); every symbol include/adr.h declares
SIGNATURES = {
    "adr_plan_create": (c_int32, [ctypes.POINTER(AdrProblem), c_void_p, ctypes.POINTER(AdrPlan)]),
    "adr_plan_create_tuned": (c_int32, [ctypes.POINTER(AdrProblem), ctypes.POINTER(AdrTuning),
                                        c_void_p, ctypes.POINTER(AdrPlan)]),
    "adr_autotune": (c_int32, [ctypes.POINTER(AdrProblem), c_void_p, c_int32,
                               ctypes.POINTER(AdrTuning), ctypes.POINTER(ctypes.c_float)]),
    "adr_plan_set_kernel": (c_int32, [AdrPlan, c_int32]),
    "adr_selftest_bounded_wait": (c_int32, [c_void_p, c_int32, c_int64, ctypes.POINTER(c_int32),
                                            ctypes.POINTER(c_int64)]),
    "adr_plan_destroy": (c_int32, [AdrPlan]),
    "adr_plan_set_stream": (c_int32, [AdrPlan, c_void_p]),
    "adr_step": (c_int32, [AdrPlan, c_void_p, c_void_p, c_int64]),
    "adr_plan_reset_state": (c_int32, [AdrPlan]),
    "adr_plan_create_general": (c_int32, [ctypes.POINTER(AdrGeneralProblem), c_void_p,
                                          ctypes.POINTER(AdrPlan)]),
    "adr_step_general": (c_int32, [AdrPlan, ctypes.POINTER(c_void_p), c_int64]),
    "adr_plan_set_indicators": (c_int32, [AdrPlan, c_int32]),
    "adr_plan_indicator_log": (c_int32, [AdrPlan, ctypes.POINTER(c_double), c_int64,
                                         ctypes.POINTER(c_int64)]),
    "adr_run": (c_int32, [AdrPlan, c_void_p, c_void_p, c_double, c_double, c_int64,
                          ctypes.POINTER(c_int64), ctypes.POINTER(c_double)]),
    "adr_plan_time_mode_products": (c_int32, [AdrPlan, c_void_p, c_void_p, c_int32,
                                              ctypes.POINTER(c_double), ctypes.POINTER(c_int32)]),
    "adr_plan_mode_product_macs": (c_int32, [AdrPlan, ctypes.POINTER(c_double),
                                             ctypes.POINTER(c_double)]),
    "adr_solve": (c_int32, [AdrPlan, c_void_p, c_void_p, c_void_p, c_void_p, c_int64]),
    "adr_plan_bytes": (c_int32, [ctypes.POINTER(AdrProblem), ctypes.POINTER(ctypes.c_size_t),
                                 ctypes.POINTER(ctypes.c_size_t)]),
    "adr_plan_matrix": (c_int32, [AdrPlan, c_int32, c_int32, c_int32, ctypes.POINTER(c_double)]),
    "adr_plan_set_timing": (c_int32, [AdrPlan, c_int32]),
    "adr_plan_stats": (c_int32, [AdrPlan, ctypes.POINTER(AdrStats)]),
    "adr_max_abs_diff": (c_int32, [c_void_p, c_void_p, c_int32, c_void_p, c_int64,
                                   ctypes.POINTER(c_double)]),
    "adr_max_abs_diff_noalloc": (c_int32, [c_void_p, c_void_p, c_int32, c_void_p, c_int64,
                                           ctypes.POINTER(c_double)]),
    "adr_batch_create": (c_int32, [ctypes.POINTER(AdrPlan), c_int32, c_void_p,
                                   ctypes.POINTER(c_void_p)]),
    "adr_batch_destroy": (c_int32, [c_void_p]),
    "adr_batch_step": (c_int32, [c_void_p, ctypes.POINTER(c_void_p), ctypes.POINTER(c_void_p),
                                ctypes.POINTER(c_int64)]),
    "adr_batch_set_timing": (c_int32, [c_void_p, c_int32]),
    "adr_batch_stats": (c_int32, [c_void_p, ctypes.POINTER(AdrStats)]),
    "adr_batch_is_grouped": (c_int32, [c_void_p]),
    "adr_indicators": (c_int32, [AdrPlan, c_void_p, c_void_p, c_void_p, c_void_p,
                                 ctypes.POINTER(c_double)]),
    "adr_status_str": (ctypes.c_char_p, [c_int32]),
    "adr_last_error": (ctypes.c_char_p, []),
}

_lib = None


class AdrError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


def lib():
    """The loaded library; raises ImportError if it was not built."""
    global _lib
    if _lib is None:
        if not os.path.exists(library_path):
            raise ImportError(f"libadr_gb300.so not built ({library_path}); run "
                              "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(library_path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(status: int):
    if status != ADR_OK:
        L = lib()
        raise AdrError(status, f"{L.adr_status_str(status).decode()}: "
                               f"{L.adr_last_error().decode()}")


def prod(xs):
    return reduce(lambda a, b: a * b, xs, 1)
