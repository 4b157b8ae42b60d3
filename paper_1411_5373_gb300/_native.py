"""ctypes declarations of the C ABI in include/fdmt.h.

Loading fails loudly when the compiled library is missing: there is no
Python or CPU fallback for any entry point.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfdmt_gb300.so")

# enum fdmt_status
OK = 0
ERR_INVALID_ARG = -1
ERR_UNSUPPORTED = -2
ERR_CUDA = -3
ERR_NO_MEMORY = -4
ERR_TIMEOUT = -5
ERR_WORKSPACE = -6

# enum fdmt_dtype
U8_I32 = 0
F32_F32 = 1
F32_F16STATE = 2

# enum fdmt_flags
PLAN_HOST_ONLY = 1 << 0
SCHED_PLAIN = 0
SCHED_FUSED = 1 << 4

_c_plan = ctypes.c_void_p
_p = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_u32 = ctypes.c_uint32
_sz = ctypes.c_size_t

# name -> (restype, argtypes); mirrors include/fdmt.h one to one.
SIGNATURES = {
    "fdmt_plan": (ctypes.c_int, [ctypes.c_double, ctypes.c_double, _i32, _i64, _i32, _i32, _u32,
                                 ctypes.POINTER(_c_plan)]),
    "fdmt_plan_curve": (ctypes.c_int, [ctypes.c_double, ctypes.c_double, _i32, _i64, _i32, _i32, _u32, _p, _p,
                                       ctypes.POINTER(_c_plan)]),
    "fdmt_plan_ex": (ctypes.c_int, [ctypes.c_double, ctypes.c_double, _i32, _i64, _i32, _i32, _u32,
                                    _p, ctypes.POINTER(_c_plan)]),
    "fdmt_destroy": (None, [_c_plan]),
    "fdmt_workspace_bytes": (ctypes.c_int, [_c_plan, ctypes.POINTER(_sz)]),
    "fdmt_adjoint_workspace_bytes": (ctypes.c_int, [_c_plan, ctypes.POINTER(_sz)]),
    "fdmt_execute": (ctypes.c_int, [_c_plan, _p, _p, _p, _p, _sz, _p]),
    "fdmt_execute_static": (ctypes.c_int, [_c_plan, _p, _p, _p, _p]),
    "fdmt_execute_host": (ctypes.c_int, [_c_plan, _p, _p, _p, _p, _p, _p, _p, _sz, _p]),
    "fdmt_adjoint": (ctypes.c_int, [_c_plan, _p, _p, _p, _p, _p, _p, _sz, _p]),
    "fdmt_search": (ctypes.c_int, [_p, _i32, _i32, _i64, _i32, _i64, _p, _p, _p, _sz, _p]),
    "fdmt_execute_search": (ctypes.c_int, [_c_plan, _p, _p, _p, _i32, _p, _p, _p, _sz, _p]),
    "fdmt_execute_search_workspace_bytes": (ctypes.c_int, [_c_plan, _i32, ctypes.POINTER(_sz)]),
    "fdmt_search_workspace_bytes": (ctypes.c_int, [_i32, _i64, _i32, ctypes.POINTER(_sz)]),
    "fdmt_stream_create": (ctypes.c_int, [ctypes.c_double, ctypes.c_double, _i32, _i64, _i32, _i32, _u32,
                                          ctypes.POINTER(_c_plan)]),
    "fdmt_stream_push": (ctypes.c_int, [_c_plan, _p, _p, _p]),
    "fdmt_stream_reset": (ctypes.c_int, [_c_plan, _p]),
    "fdmt_stream_info": (ctypes.c_int, [_c_plan, ctypes.POINTER(_i64), ctypes.POINTER(_i64)]),
    "fdmt_stream_destroy": (None, [_c_plan]),
    "fdmt_filterbank": (ctypes.c_int, [_p, _i64, _i32, _i32, _p, _i64, _p]),
    "fdmt_fft_plan": (ctypes.c_int, [ctypes.c_double, ctypes.c_double, _i32, _i64, _i32, _i32, _i32, _i32, _u32,
                                     ctypes.POINTER(_c_plan)]),
    "fdmt_fft_destroy": (None, [_c_plan]),
    "fdmt_fft_workspace_bytes": (ctypes.c_int, [_c_plan, ctypes.POINTER(_sz)]),
    "fdmt_fft_info": (ctypes.c_int, [_c_plan, ctypes.POINTER(_i32), ctypes.POINTER(_i64), ctypes.POINTER(_i64),
                                     ctypes.POINTER(_i32)]),
    "fdmt_fft_execute": (ctypes.c_int, [_c_plan, _p, _p, _p, _sz, _p]),
    "fdmt_fft_profile_enable": (ctypes.c_int, [_c_plan, _i32]),
    "fdmt_fft_profile_read": (ctypes.c_int, [_c_plan, ctypes.POINTER(_i32), ctypes.POINTER(ctypes.c_float), _i32,
                                             ctypes.POINTER(_i64)]),
    "fdmt_plan_shape": (ctypes.c_int, [_c_plan, _p, _p, _p, _p]),
    "fdmt_pipeline_create": (ctypes.c_int, [_c_plan, ctypes.POINTER(_c_plan)]),
    "fdmt_pipeline_push": (ctypes.c_int, [_c_plan, _p, _p]),
    "fdmt_pipeline_wait": (ctypes.c_int, [_c_plan]),
    "fdmt_pipeline_destroy": (None, [_c_plan]),
    "fdmt_error_string": (ctypes.c_char_p, [ctypes.c_int]),
    "fdmt_profile_enable": (ctypes.c_int, [_c_plan, _i32]),
    "fdmt_profile_read": (ctypes.c_int, [_c_plan, _p, _p, _p, _i32, ctypes.POINTER(_i64)]),
    "fdmt_kernel_name": (ctypes.c_char_p, [_i32]),
    "fdmt_plan_batch": (ctypes.c_int, [_i32, _p, _i32, _u32, _p, ctypes.POINTER(_c_plan)]),
    "fdmt_destroy_batch": (None, [_c_plan]),
    "fdmt_batch_workspace_bytes": (ctypes.c_int, [_c_plan, ctypes.POINTER(_sz)]),
    "fdmt_execute_batch": (ctypes.c_int, [_c_plan, _p, _p, _p, _sz, _p]),
    "fdmt_batch_drop_level": (ctypes.c_int, [_c_plan, _i32, _i32]),
    "fdmt_batch_levels": (ctypes.c_int, [_c_plan, _i32, ctypes.POINTER(_i32), _p, _p, _i32]),
    "fdmt_device_status": (ctypes.c_int, [_c_plan, _p]),
    "fdmt_fused_tables": (ctypes.c_int, [_c_plan, _i32, _p, _i64, ctypes.POINTER(_i64)]),
    "fdmt_schedule_info": (ctypes.c_int, [_c_plan, ctypes.POINTER(_i32), _p, _i32, ctypes.POINTER(_i32)]),
    "fdmt_num_levels": (ctypes.c_int, [_c_plan, ctypes.POINTER(_i32)]),
    "fdmt_band_rows": (ctypes.c_int, [_c_plan, _i32, ctypes.POINTER(_i32), _i32]),
    "fdmt_band_dl": (ctypes.c_int, [_c_plan, _i32, _i32, ctypes.POINTER(_i32), _i32]),
    "fdmt_input_map": (ctypes.c_int, [_c_plan, _p, _i32, ctypes.POINTER(_i32)]),
}



class BeamDesc(ctypes.Structure):
    """struct fdmt_beam_desc."""
    _fields_ = [("f_min", ctypes.c_double), ("f_max", ctypes.c_double), ("nf", _i32), ("nd", _i32),
                ("nt", _i64)]


class BatchParams(ctypes.Structure):
    """struct fdmt_batch_params."""
    _fields_ = [("rows_per_item", _i32), ("tile", _i32), ("blocks_per_sm", _i32), ("wait_ms", _i32),
                ("schedule", _i32), ("fused_tile", _i32), ("smem_budget", _i32)]


class CurveParams(ctypes.Structure):
    """struct fdmt_curve_params."""
    _fields_ = [("gamma", ctypes.c_double), ("d_min", _i32), ("descending", _i32)]


class ScheduleParams(ctypes.Structure):
    """struct fdmt_schedule_params."""
    _fields_ = [("tile", _i32), ("smem_budget", _i32), ("n_bounds", _i32), ("bounds", _i32 * 32),
                ("group_tile", _i32 * 32), ("group_budget", _i32 * 32), ("staging", _i32),
                ("state16", _i32), ("search_widths", _i32), ("adjoint_schedule", _i32), ("adjoint_tile", _i32),
                ("adjoint_smem_budget", _i32), ("adjoint_n_bounds", _i32), ("adjoint_bounds", _i32 * 32),
                ("adjoint_group_tile", _i32 * 32), ("adjoint_group_budget", _i32 * 32)]


_lib = None


class FdmtError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = error_string(status) if _lib is not None else str(status)
        super().__init__(f"{where}: {msg} (status {status})")


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load the compiled library (once) and declare every entry point."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(
            f"FDMT CUDA library not built: {path} is missing. "
            "Run `python -m paper_1411_5373_gb300.build` (or __graft_entry__.build()).")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def error_string(status: int) -> str:
    return load().fdmt_error_string(int(status)).decode()


def check(status: int, where: str) -> None:
    if status != OK:
        raise FdmtError(status, where)
