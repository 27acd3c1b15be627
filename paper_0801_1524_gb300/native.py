"""ctypes declarations of the C ABI in include/bfly.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbfly.so")

BFLY_OK = 0
BFLY_ERR_INVALID_ARG = 1
STATUS = {0: "OK", 1: "INVALID_ARG", 2: "OUT_OF_MEMORY", 3: "CUDA", 4: "UNSUPPORTED", 5: "TIMEOUT"}
BFLY_C64, BFLY_C128 = 0, 1
BFLY_PREC_FP64, BFLY_PREC_FP32, BFLY_PREC_TC = 0, 1, 2
BFLY_FLAG_HOST_ONLY = 1
BFLY_FLAG_TEST_STALL = 2
BFLY_FLAG_AUTOTUNE = 4
BFLY_FLAG_ONE_STAGE = 8
BFLY_FLAG_RHS_GROUPS = 16
BFLY_FLAG_DATAFLOW = 32

# Every function the header declares, with (restype, argtypes).
_vp, _i, _i64, _d = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double


class Opts(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int), ("max_nrhs", ctypes.c_int), ("flags", ctypes.c_uint),
                ("smem_kb", ctypes.c_int), ("tune_cache", ctypes.c_char_p),
                ("stages", ctypes.c_int), ("reserved", ctypes.c_int)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("p", ctypes.c_int), ("L", ctypes.c_int),
                ("prec", ctypes.c_int), ("N", ctypes.c_double), ("rho", ctypes.c_double),
                ("nx", ctypes.c_int64),
                ("nk", ctypes.c_int64), ("total_pairs", ctypes.c_int64),
                ("max_pairs", ctypes.c_int64), ("workspace_bytes", ctypes.c_int64),
                ("tiles_read_fwd", ctypes.c_int64), ("tiles_written_fwd", ctypes.c_int64),
                ("jobs_fwd", ctypes.c_int64), ("chunks_fwd", ctypes.c_int64),
                ("flops_fwd", ctypes.c_double), ("lane_use_fwd", ctypes.c_double),
                ("smem_kb", ctypes.c_int),
                ("blocks_per_sm", ctypes.c_int), ("tuned_ms", ctypes.c_double),
                ("plan_seconds", ctypes.c_double), ("steps", ctypes.c_int),
                ("stages_per_launch", ctypes.c_int), ("rhs_groups", ctypes.c_int),
                ("dataflow", ctypes.c_int)]


SIGNATURES = {
    "bfly_plan_create": (_i, [ctypes.POINTER(_vp), _i, _d, _i64, _vp, _i64, _vp, _i,
                              ctypes.POINTER(Opts)]),
    "bfly_plan_destroy": (None, [_vp]),
    "bfly_execute": (_i, [_vp, _vp, _vp, _i, _i, _vp]),
    "bfly_execute_noalloc": (_i, [_vp, _vp, _vp, _i, _i, _vp]),
    "bfly_execute_to_stage": (_i, [_vp, _vp, _i, _vp, _i, _i, _i, _vp]),
    "bfly_execute_from_stage": (_i, [_vp, _vp, _i, _vp, _i, _i, _i, _vp]),
    "bfly_execute_adjoint": (_i, [_vp, _vp, _vp, _i, _i, _vp]),
    "bfly_execute_host": (_i, [_vp, _vp, _vp, _i, _i, _i, _vp]),
    "bfly_direct": (_i, [_vp, _vp, _vp, _i, _i, _i, _vp]),
    "bfly_execute_events": (_i, [_vp, _vp, _vp, _i, _i, _i, _vp, ctypes.POINTER(_vp), _i]),
    "bfly_plan_info": (_i, [_vp, ctypes.POINTER(PlanInfo)]),
    "bfly_batch_create": (_i, [ctypes.POINTER(_vp), _i, ctypes.POINTER(_vp)]),
    "bfly_batch_execute": (_i, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), _i, _i, _vp]),
    "bfly_batch_status": (_i, [_vp, ctypes.POINTER(ctypes.c_int)]),
    "bfly_batch_destroy": (None, [_vp]),
    "bfly_device_status": (_i, [_vp, ctypes.POINTER(ctypes.c_int)]),
    "bfly_stream_status": (_i, [_vp, _vp, ctypes.POINTER(ctypes.c_int)]),
    "bfly_measure_peak": (_i, [_i, ctypes.POINTER(_d), ctypes.POINTER(_d)]),
    "bfly_plan_stage": (_i, [_vp, _i, ctypes.POINTER(_i64), ctypes.POINTER(_i64)]),
    "bfly_plan_step": (_i, [_vp, _i, ctypes.POINTER(_i), ctypes.POINTER(_i)]),
    "bfly_plan_program": (_i, [_vp, _i, _i, _i, _vp, _i64, ctypes.POINTER(_i64)]),
    "bfly_plan_boxes": (_i, [_vp, _i, _i, _vp, _i64, ctypes.POINTER(_i64)]),
    "bfly_last_error": (ctypes.c_char_p, []),
    "bfly_version": (ctypes.c_char_p, []),
}

_lib = None


class BflyError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS.get(status, status)}: {msg}")
        self.status = status


def load(build_if_missing: bool = True):
    """Loads libbfly.so (building it first if it is missing); raises if it cannot."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        if not build_if_missing:
            raise RuntimeError(f"{LIB_PATH} is missing; run paper_0801_1524_gb300.build.build()")
        from . import build as _build
        _build.build()
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(status: int, where: str):
    if status != BFLY_OK:
        raise BflyError(status, where, load().bfly_last_error().decode())
