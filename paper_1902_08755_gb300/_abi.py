"""ctypes mirror of include/ec.h and the loader for libec.so.

There is no fallback: if the CUDA library cannot be loaded, every entry point
raises.  Struct layouts must match include/ec.h field for field.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))

EC_OK, EC_ERR_INVALID_ARG, EC_ERR_CAPACITY, EC_ERR_CUDA = 0, 1, 2, 3
EC_ERR_CORRUPT, EC_ERR_UNSUPPORTED, EC_ERR_TIMEOUT = 4, 5, 6
EC_RGBA8, EC_RGBA32F, EC_RGBA16F = 0, 1, 2
EC_MAX_SOURCES = 512
EC_RLE_CHUNK = 4096
EC_RLE_MAX_ELEMS = 1 << 27
EC_RLE_MAX_JOBS = 512
EC_RLE_NOALLOC_MAX_CHUNKS = 8192

STATUS_NAMES = {0: "EC_OK", 1: "EC_ERR_INVALID_ARG", 2: "EC_ERR_CAPACITY", 3: "EC_ERR_CUDA",
                4: "EC_ERR_CORRUPT", 5: "EC_ERR_UNSUPPORTED", 6: "EC_ERR_TIMEOUT"}


class EcError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {STATUS_NAMES.get(code, code)}")
        self.code = code


class ec_rect(C.Structure):
    _fields_ = [("x", C.c_int32), ("y", C.c_int32), ("w", C.c_int32), ("h", C.c_int32)]

    def tup(self):
        return (self.x, self.y, self.w, self.h)


class ec_image(C.Structure):
    _fields_ = [("pvp", ec_rect), ("roi", ec_rect), ("pitch", C.c_int32), ("format", C.c_int32),
                ("color", C.c_void_p), ("depth", C.c_void_p)]


class ec_target(C.Structure):
    _fields_ = [("pvp", ec_rect), ("pitch", C.c_int32), ("format", C.c_int32),
                ("color", C.c_void_p), ("depth", C.c_void_p)]


class ec_rle_job(C.Structure):
    _fields_ = [("src", C.c_void_p), ("dst", C.c_void_p), ("capacity", C.c_size_t),
                ("d_size", C.c_void_p), ("w", C.c_int32), ("h", C.c_int32),
                ("pitch", C.c_int32), ("mode", C.c_uint32)]


class ec_job(C.Structure):
    _fields_ = [("mode", C.c_int32), ("n", C.c_int32), ("in_", C.c_void_p), ("order", C.c_void_p),
                ("out", ec_target), ("winner", C.c_void_p), ("t_final", C.c_void_p)]


class ec_batch_config(C.Structure):
    _fields_ = [("depth_tile_w", C.c_int32), ("depth_tile_h", C.c_int32),
                ("alpha32_tile_w", C.c_int32), ("alpha32_tile_h", C.c_int32),
                ("alpha16_tile_w", C.c_int32), ("alpha16_tile_h", C.c_int32),
                ("ctas_per_sm", C.c_int32)]


EC_JOB_DEPTH, EC_JOB_ALPHA = 0, 1
EC_SCHED_STREAM, EC_SCHED_DIRECT_SEND, EC_SCHED_BINARY_SWAP, EC_SCHED_TWO_THREE_SWAP = 0, 1, 2, 3
EC_SCHED_RLE, EC_SCHED_FUSED = 1, 2


EC_SCHED_LAUNCH_KINDS = ("rle_compress", "rle_decompress", "fused_depth", "composite")


class ec_sched_launch(C.Structure):
    _fields_ = [("level", C.c_int32), ("kind", C.c_int32), ("bytes", C.c_uint64)]


class ec_yuv_job(C.Structure):
    _fields_ = [("src", C.c_void_p), ("dst", C.c_void_p), ("w", C.c_int32), ("h", C.c_int32),
                ("pitch", C.c_int32), ("packed_pitch", C.c_int32)]


class ec_sched_message(C.Structure):
    _fields_ = [("level", C.c_int32), ("sender", C.c_int32), ("receiver", C.c_int32),
                ("fused", C.c_int32), ("piece", ec_rect)]
assert C.sizeof(ec_job) == 80 and C.sizeof(ec_batch_config) == 28
assert C.sizeof(ec_image) == 56 and C.sizeof(ec_target) == 40 and C.sizeof(ec_rle_job) == 48

_P = C.c_void_p
_I = C.c_int32
_R = ec_rect
_S = C.c_int  # ec_status

# name -> (restype, argtypes), exactly the declarations of include/ec.h
SIGNATURES = {
    "ec_create": (_S, [C.POINTER(C.c_void_p), C.c_int]),
    "ec_destroy": (None, [_P]),
    "ec_status_sync": (_S, [_P, _P]),
    "ec_status_string": (C.c_char_p, [_S]),
    "ec_composite_depth": (_S, [_P, _P, _I, _P, _P, C.POINTER(ec_rect), _P]),
    "ec_composite_alpha": (_S, [_P, _P, _P, _I, _P, _P, C.POINTER(ec_rect), _P]),
    "ec_composite_alpha_backward": (_S, [_P, _P, _P, _I, _R, _P, _P, _I, _P]),
    "ec_composite_alpha_fwd_bwd": (_S, [_P, _P, _P, _I, _P, _P, _P, _P, _I, C.POINTER(ec_rect), _P]),
    "ec_composite_depth_backward": (_S, [_P, _P, _R, _P, _I, _P, _P, _P, _P]),
    "ec_detect_roi": (_S, [_P, _P, _I, _I, _P, _P, _P]),
    "ec_assemble_tiles": (_S, [_P, _P, _I, _P, _P]),
    "ec_assemble_pixels": (_S, [_P, _P, _P, _P, _I, _I, _I, _P, _P]),
    "ec_average": (_S, [_P, _P, _I, _P, _P]),
    "ec_rle_max_size": (C.c_size_t, [_I, _I]),
    "ec_rle_compress": (_S, [_P, _P, _I, _I, _I, C.c_uint32, _P, C.c_size_t, _P, _P]),
    "ec_rle_decompress": (_S, [_P, _P, C.c_size_t, _P, _I, _I, _I, _P]),
    "ec_rle_compress_batch": (_S, [_P, _P, _I, _P]),
    "ec_rle_decompress_batch": (_S, [_P, _P, _I, _P]),
    "ec_batch_plan": (_S, [_P, _P, _I, _P, C.POINTER(C.c_void_p)]),
    "ec_batch_run": (_S, [_P, _P]),
    "ec_batch_get_config": (_S, [_P, _P, _P, _P]),
    "ec_batch_free": (None, [_P]),
    "ec_yuv_encode": (_S, [_P, _P, _I, _I, _I, _P, _I, _P]),
    "ec_yuv_decode": (_S, [_P, _P, _I, _I, _I, _P, _I, _P]),
    "ec_selftest_wait_timeout": (_S, [_P, _P]),
    "ec_yuv_encode_batch": (_S, [_P, _P, _I, _P]),
    "ec_yuv_decode_batch": (_S, [_P, _P, _I, _P]),
    "ec_schedule_plan": (_S, [_P, _I, _I, _P, _I, _P, _P, C.c_uint32, C.POINTER(C.c_void_p)]),
    "ec_schedule_run": (_S, [_P, _P]),
    "ec_schedule_geometry": (_S, [_I, _P, _I, ec_rect, _P, _I, _P, _P, _P]),
    "ec_schedule_info": (_S, [_P, _P, _P, _P, _P]),
    "ec_schedule_messages": (_S, [_P, _P, _I]),
    "ec_schedule_launches": (_S, [_P, _P, _I]),
    "ec_schedule_run_launch": (_S, [_P, _I, _P]),
    "ec_schedule_stream_sizes": (_S, [_P, _P, _I, _P]),
    "ec_schedule_free": (None, [_P]),
    "ec_rle_compress_noalloc": (_S, [_P, _I, _I, _I, C.c_uint32, _P, C.c_size_t, _P, _P, _P]),
}

_lib = None
_lock = threading.Lock()


def lib_path() -> str:
    return os.path.join(HERE, "libec.so")


def load(build_if_missing: bool = True):
    """Load libec.so (building it with nvcc first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_missing:
            from . import build as _build
            try:
                _build.build()
            except (OSError, RuntimeError) as e:
                if not os.path.exists(lib_path()):
                    raise RuntimeError(f"libec.so is missing and could not be built: {e}") from e
        if not os.path.exists(lib_path()):
            raise RuntimeError("libec.so is missing: run paper_1902_08755_gb300.build.build()")
        L = C.CDLL(lib_path())
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
        return _lib


def check(code: int, what: str):
    if code != EC_OK:
        raise EcError(code, what)
