"""ctypes view of the shtgb C ABI (include/sht.h).

Loads ``libshtgb.so`` from this package directory.  There is no fallback:
if the library is missing or cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libshtgb.so")

SHT_OK = 0
STATUS = {0: "SHT_OK", 1: "SHT_ERR_INVALID_ARG", 2: "SHT_ERR_UNSUPPORTED", 3: "SHT_ERR_OOM",
          4: "SHT_ERR_CUDA", 5: "SHT_ERR_TIMEOUT", 6: "SHT_ERR_INTERNAL"}
GRIDS = {"gauss": 0, "equiangular_cc": 1, "equiangular_trapz": 2}
PRECISIONS = {"fp32": 0, "bf16": 1, "split_bf16": 2}
TABLE_SOURCES = {"streamed": 0, "recurrence": 1, "mixed": 2}
KERNEL_COUNT = 10


class sht_plan_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("device", ctypes.c_int), ("max_batch", ctypes.c_int64),
                ("max_channels", ctypes.c_int), ("table_source", ctypes.c_int), ("reserved", ctypes.c_int * 6)]


class sht_batch_item(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_void_p), ("count", ctypes.c_int64), ("input", ctypes.c_void_p),
                ("output", ctypes.c_void_p)]


class sht_batch_opts(ctypes.Structure):
    _fields_ = [("direction", ctypes.c_int), ("tune", ctypes.c_int), ("tune_cache", ctypes.c_char_p),
                ("profile", ctypes.c_int), ("reserved", ctypes.c_int * 8)]


BATCH_DIRECTIONS = {"forward": 0, "inverse": 1}

_i, _i64, _p, _d = ctypes.c_int, ctypes.c_int64, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)
_ip, _i64p = ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int64)

# name -> (argtypes, restype); the declarations of include/sht.h
SIGNATURES = {
    "sht_plan_opts_default": ([ctypes.POINTER(sht_plan_opts)], None),
    "sht_plan": ([ctypes.POINTER(_p), _i, _i, _i, _i, _i, ctypes.POINTER(sht_plan_opts)], _i),
    "sht_plan_destroy": ([_p], _i),
    "sht_plan_info": ([_p, _ip, _ip, _ip, _ip, _ip, _ip, _i64p, _i64p, _i64p], _i),
    "sht_plan_grid": ([_p, _d, _d], _i),
    "sht_plan_check": ([_p], _i),
    "sht_forward": ([_p, _p, _p, _i64, _p], _i),
    "sht_inverse": ([_p, _p, _p, _i64, _p], _i),
    "sht_forward_adjoint": ([_p, _p, _p, _i64, _p], _i),
    "sht_inverse_adjoint": ([_p, _p, _p, _i64, _p], _i),
    "spectral_filter": ([_p, _p, _p, _p, _i64, _i, _i, _p], _i),
    "spectral_filter_adjoint": ([_p, _p, _p, _p, _p, _p, _i64, _i, _i, _p], _i),
    "sht_spectral_block": ([_p, _p, _p, _p, _i64, _i, _i, _p], _i),
    "spectral_filter_inverse": ([_p, _p, _p, _p, _i64, _i, _i, _p], _i),
    "sht_forward_static_scratch": ([_p, _p, _p, _i64, _p], _i),
    "sht_spectral_block_adjoint": ([_p, _p, _p, _p, _i64, _i, _i, _p], _i),
    "sht_spectral_block_weight_grad": ([_p, _p, _p, _p, _i64, _i, _i, _p], _i),
    "sht_spectral_block_backward": ([_p, _p, _p, _p, _p, _p, _i64, _i, _i, _p], _i),
    "sht_analysis_rows": ([_p, _p, _p, _i64, _i, _i, _p], _i),
    "sht_synthesis_rows": ([_p, _p, _p, _i64, _i, _i, _p], _i),
    "sht_legendre_orders": ([_p, _i, _p, _p, _i64, _i, _i, _p], _i),
    "sht_profile_begin": ([_p, _i], _i),
    "sht_profile_collect": ([_p, _i64p, ctypes.POINTER(ctypes.c_double), _i64p], _i),
    "sht_profile_end": ([_p], _i),
    "sht_kernel_name": ([_i], ctypes.c_char_p),
    "sht_status_string": ([_i], ctypes.c_char_p),
    "sht_last_error_message": ([], ctypes.c_char_p),
    "sht_version": ([], ctypes.c_char_p),
    "sht_debug_fail_alloc_after": ([_i], None),
    "sht_debug_stall": ([_p, _i64, _p], _i),
    "sht_batch_opts_default": ([ctypes.POINTER(sht_batch_opts)], None),
    "sht_batch_create": ([ctypes.POINTER(_p), ctypes.POINTER(sht_batch_item), _i, ctypes.POINTER(sht_batch_opts), _p],
                         _i),
    "sht_batch_run": ([_p, _p], _i),
    "sht_batch_describe": ([_p, ctypes.c_char_p, _i], _i),
    "sht_batch_stage_count": ([_p], _i),
    "sht_batch_stage_name": ([_p, _i], ctypes.c_char_p),
    "sht_batch_profile_begin": ([_p, _i], _i),
    "sht_batch_profile_collect": ([_p, _i64p, ctypes.POINTER(ctypes.c_double)], _i),
    "sht_batch_destroy": ([_p], _i),
    "sht_pipe_create": ([ctypes.POINTER(_p), _p, _i64, _i, _i, _i], _i),
    "sht_pipe_block": ([_p, _p, _p, _p, _p], _i),
    "sht_pipe_wait": ([_p], _i),
    "sht_pipe_destroy": ([_p], _i),
    "sht_angular_psd": ([_p, _p, _i64, _i, _i, _p], _i),
    "sht_spectral_crps": ([_p, _p, _p, _p, _p, _i, _i64, _i, _i, _i, _i, _i, _p], _i),
    "sht_zonal_psd": ([_p, _p, _p, _i64, _p], _i),
    "sht_disco_create": ([ctypes.POINTER(_p), _i, _i, _i, _i, _i, _i, _i, ctypes.c_double, _i], _i),
    "sht_disco_info": ([_p, _ip, _i64p], _i),
    "sht_disco_forward": ([_p, _p, _p, _i64, _p], _i),
    "sht_disco_backward": ([_p, _p, _p, _i64, _p], _i),
    "sht_disco_check": ([_p], _i),
    "sht_disco_destroy": ([_p], _i),
    "sht_diffusion_step": ([_p, _p, _i64, _i, _i, _d, _i, ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                            ctypes.c_uint64, _p], _i),
    "sht_spectral_crps_backward": ([_p, _p, _p, _p, _p, _i, _i64, _i, _i, _i, _i, _i, _p], _i),
    "sht_spatial_crps": ([_p, _p, _p, _p, _p, _i, _i64, _i, _p], _i),
}

_lock = threading.Lock()
_lib = None


class ShtError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"shtgb CUDA library not built ({LIB_PATH} missing); run "
                    "`python -c 'import __graft_entry__ as g; g.build()'` first")
            handle = ctypes.CDLL(LIB_PATH)
            for name, (args, res) in SIGNATURES.items():
                fn = getattr(handle, name)
                fn.argtypes = args
                fn.restype = res
            _lib = handle
        return _lib


def check(status: int) -> None:
    if status != SHT_OK:
        msg = lib().sht_last_error_message().decode(errors="replace")
        raise ShtError(status, msg)
