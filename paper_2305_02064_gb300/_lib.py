"""ctypes binding of libmmsar (include/mmsar.h): argument marshalling only.

Every step of the imaging path runs in the library's CUDA kernels; this
module only turns PyTorch tensors into device pointers and a stream handle.
There is no CPU path: if the library cannot be loaded, the calls raise.
"""
from __future__ import annotations

import ctypes
import math
import os
import threading

from . import build as _build

_LIB = None
_LOCK = threading.Lock()

MMSAR_OK = 0
STATUS = {0: "MMSAR_OK", 1: "MMSAR_ERR_INVALID_ARG", 2: "MMSAR_ERR_UNSUPPORTED_SIZE",
          3: "MMSAR_ERR_OUT_OF_MEMORY", 4: "MMSAR_ERR_CUDA", 5: "MMSAR_ERR_DEVICE_TIMEOUT",
          6: "MMSAR_ERR_NONFINITE"}
DTYPES = {"c64": 0, "f16": 1, "bf16": 2}

# Every symbol include/mmsar.h declares (checked by the CPU test suite).
EXPORTS = ["mmsar_options_default", "mmsar_plan_create", "mmsar_plan_workspace_bytes", "mmsar_plan_info",
           "mmsar_stage_count", "mmsar_stage_name", "mmsar_plan_set_stage_events",
           "mmsar_image", "mmsar_poll_error", "mmsar_peak_scratch_bytes", "mmsar_peak", "mmsar_last_error",
           "mmsar_plan_destroy", "mmsar_version", "mmsar_static_workspace_bytes", "mmsar_image_static",
           "mmsar_quantize_echo", "mmsar_image_batch", "mmsar_image_batch_fused", "mmsar_backproject",
           "mmsar_plan_set_tiles", "mmsar_plan_get_tiles", "mmsar_plan_set_wait_test"]


class MmsarError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class Request(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_void_p), ("workspace", ctypes.c_void_p), ("workspace_bytes", ctypes.c_size_t),
                ("echo", ctypes.c_void_p), ("echo_scale", ctypes.c_void_p), ("pos", ctypes.c_void_p),
                ("tx", ctypes.c_void_p), ("rx", ctypes.c_void_p), ("vol", ctypes.c_void_p)]


class Shape(ctypes.Structure):
    _fields_ = [("n_tx", ctypes.c_int), ("n_rx", ctypes.c_int), ("n_pos", ctypes.c_int), ("n_k", ctypes.c_int),
                ("f0_hz", ctypes.c_double), ("df_hz", ctypes.c_double), ("dtype", ctypes.c_int)]


class Grid(ctypes.Structure):
    _fields_ = [("x0", ctypes.c_double), ("y0", ctypes.c_double), ("z0", ctypes.c_double),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
                ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int)]


class Tiles(ctypes.Structure):
    _fields_ = [("grid_freqs_per_lane", ctypes.c_int), ("grid_warps_per_cta", ctypes.c_int),
                ("grid_grouped", ctypes.c_int), ("grid_tensor_cores", ctypes.c_int)]


class Options(ctypes.Structure):
    _fields_ = [("z_ref", ctypes.c_double), ("z_scene", ctypes.c_double), ("compensate", ctypes.c_int),
                ("nufft_tol", ctypes.c_double), ("mx", ctypes.c_int), ("my", ctypes.c_int)]


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libmmsar.so (building it in-tree with nvcc when absent)."""
    global _LIB
    with _LOCK:
        if _LIB is not None:
            return _LIB
        path = _build.LIB
        if not os.path.exists(path):
            if not build_if_missing:
                raise OSError(f"{path} is missing; build it with paper_2305_02064_gb300.build.build()")
            _build.build()
        lib = ctypes.CDLL(path)
        vp, sz = ctypes.c_void_p, ctypes.c_size_t
        lib.mmsar_options_default.argtypes = [ctypes.POINTER(Options)]
        lib.mmsar_options_default.restype = None
        lib.mmsar_plan_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(Shape), ctypes.POINTER(Grid),
                                          ctypes.POINTER(Options)]
        lib.mmsar_plan_create.restype = ctypes.c_int
        lib.mmsar_plan_workspace_bytes.argtypes = [vp, ctypes.POINTER(sz)]
        lib.mmsar_plan_workspace_bytes.restype = ctypes.c_int
        ip = ctypes.POINTER(ctypes.c_int)
        lib.mmsar_plan_info.argtypes = [vp, ip, ip, ip, ip]
        lib.mmsar_plan_info.restype = ctypes.c_int
        lib.mmsar_stage_count.argtypes = []
        lib.mmsar_stage_count.restype = ctypes.c_int
        lib.mmsar_stage_name.argtypes = [ctypes.c_int]
        lib.mmsar_stage_name.restype = ctypes.c_char_p
        lib.mmsar_plan_set_stage_events.argtypes = [vp, ctypes.POINTER(vp), ctypes.c_int]
        lib.mmsar_plan_set_stage_events.restype = ctypes.c_int
        lib.mmsar_image.argtypes = [vp, vp, sz, vp, vp, vp, vp, vp, vp, vp]
        lib.mmsar_image.restype = ctypes.c_int
        lib.mmsar_poll_error.argtypes = [vp, vp]
        lib.mmsar_poll_error.restype = ctypes.c_int
        lib.mmsar_peak_scratch_bytes.argtypes = [ctypes.c_int64]
        lib.mmsar_peak_scratch_bytes.restype = sz
        lib.mmsar_peak.argtypes = [vp, ctypes.c_int64, vp, vp, vp]
        lib.mmsar_peak.restype = ctypes.c_int
        lib.mmsar_last_error.argtypes = []
        lib.mmsar_last_error.restype = ctypes.c_char_p
        lib.mmsar_plan_destroy.argtypes = [vp]
        lib.mmsar_plan_destroy.restype = None
        lib.mmsar_static_workspace_bytes.argtypes = []
        lib.mmsar_static_workspace_bytes.restype = sz
        lib.mmsar_image_static.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp]
        lib.mmsar_image_static.restype = ctypes.c_int
        lib.mmsar_quantize_echo.argtypes = [vp, ctypes.c_int64, ctypes.c_int, vp, vp, vp, vp]
        lib.mmsar_quantize_echo.restype = ctypes.c_int
        lib.mmsar_image_batch.argtypes = [ctypes.POINTER(Request), ctypes.c_int, ctypes.POINTER(vp), ctypes.c_int]
        lib.mmsar_image_batch.restype = ctypes.c_int
        lib.mmsar_image_batch_fused.argtypes = [ctypes.POINTER(Request), ctypes.c_int, vp,
                                                ctypes.POINTER(ctypes.c_int)]
        lib.mmsar_image_batch_fused.restype = ctypes.c_int
        lib.mmsar_backproject.argtypes = [vp, vp, vp, vp, vp, vp, ctypes.c_int64, vp, vp]
        lib.mmsar_backproject.restype = ctypes.c_int
        lib.mmsar_plan_set_tiles.argtypes = [vp, ctypes.POINTER(Tiles)]
        lib.mmsar_plan_set_tiles.restype = ctypes.c_int
        lib.mmsar_plan_set_wait_test.argtypes = [vp, ctypes.c_int]
        lib.mmsar_plan_set_wait_test.restype = ctypes.c_int
        lib.mmsar_plan_get_tiles.argtypes = [vp, ctypes.POINTER(Tiles)]
        lib.mmsar_plan_get_tiles.restype = ctypes.c_int
        lib.mmsar_version.argtypes = []
        lib.mmsar_version.restype = ctypes.c_char_p
        _LIB = lib
        return lib


def check(code: int):
    if code != MMSAR_OK:
        msg = load().mmsar_last_error().decode(errors="replace")
        raise MmsarError(code, msg)


def _nan(v):
    return math.nan if v is None else float(v)
