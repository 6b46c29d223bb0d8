"""CPU oracle for sort-last compositing and the RLE pixel codec (test infrastructure).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path
(``paper_1902_08755_gb300``) never imports it and shares no code with it; the two
meet only through the seeded input generators in ``synthetic/``.

The arithmetic lives in ``ec_oracle.c`` (plain single-threaded C, double
precision for alpha); this module is argument marshalling over ctypes.
Thesis references (Eilemann, arXiv 1902.08755): 5.2.1 depth-sorted and spatial
(ordered) sort-last compositing, 5.3 region of interest, 5.5.1 RLE with
per-component streams and the swizzle preconditioner.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ec_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

OK, EINVAL, ECAP, ECORRUPT = 0, 1, 2, 4
F32, F16 = 1, 2


def build(force: bool = False) -> str:
    """Compile ec_oracle.c into liboracle.so with the host C compiler."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "ec_oracle.h"))
    ):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
        )
        os.replace(tmp, _LIB)
    return _LIB


class Rect(C.Structure):
    _fields_ = [("x", C.c_int32), ("y", C.c_int32), ("w", C.c_int32), ("h", C.c_int32)]

    def tup(self):
        return (self.x, self.y, self.w, self.h)


class _DepthSrc(C.Structure):
    _fields_ = [("pvp", Rect), ("roi", Rect), ("pitch", C.c_int32),
                ("color", C.c_void_p), ("depth", C.c_void_p)]


class _Layer(C.Structure):
    _fields_ = [("pvp", Rect), ("roi", Rect), ("pitch", C.c_int32), ("color", C.c_void_p)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        L.orc_composite_depth.restype = C.c_int
        L.orc_composite_depth.argtypes = [C.c_void_p, C.c_int32, C.c_int32, Rect, C.c_int32,
                                          C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(Rect)]
        L.orc_composite_alpha.restype = C.c_int
        L.orc_composite_alpha.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, Rect,
                                          C.c_void_p, C.c_void_p, C.POINTER(Rect)]
        L.orc_composite_alpha_backward.restype = C.c_int
        L.orc_composite_alpha_backward.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p,
                                                   Rect, C.c_void_p, C.c_void_p]
        L.orc_composite_depth_backward.restype = C.c_int
        L.orc_composite_depth_backward.argtypes = [C.c_void_p, Rect, C.c_void_p, C.c_int32,
                                                   C.c_void_p, C.c_void_p, C.c_void_p]
        L.orc_assemble_tiles.restype = C.c_int
        L.orc_assemble_tiles.argtypes = [C.c_void_p, C.c_int32, C.c_int32, Rect, C.c_int32, C.c_void_p]
        L.orc_assemble_pixels.restype = C.c_int
        L.orc_assemble_pixels.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32,
                                          C.c_int32, C.c_int32, C.c_int32, Rect, C.c_int32, C.c_void_p]
        L.orc_average.restype = C.c_int
        L.orc_average.argtypes = [C.c_void_p, C.c_int32, C.c_int32, Rect, C.c_int32, C.c_void_p]
        L.orc_detect_roi.restype = C.c_int
        L.orc_detect_roi.argtypes = [Rect, Rect, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p,
                                     C.c_int32, C.c_void_p, C.POINTER(Rect)]
        L.orc_rle_max_size.restype = C.c_size_t
        L.orc_rle_max_size.argtypes = [C.c_int32, C.c_int32]
        L.orc_swizzle.restype = C.c_uint32
        L.orc_swizzle.argtypes = [C.c_uint32]
        L.orc_unswizzle.restype = C.c_uint32
        L.orc_unswizzle.argtypes = [C.c_uint32]
        L.orc_rle_compress.restype = C.c_int64
        L.orc_rle_compress.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_uint32,
                                       C.c_void_p, C.c_size_t]
        L.orc_yuv_encode.restype = C.c_int
        L.orc_yuv_encode.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_void_p]
        L.orc_yuv_decode.restype = C.c_int
        L.orc_yuv_decode.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_int32]
        L.orc_rle_decompress.restype = C.c_int
        L.orc_rle_decompress.argtypes = [C.c_void_p, C.c_size_t, C.c_void_p, C.c_int32,
                                         C.c_int32, C.c_int32]
        _lib = L
    return _lib


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: oracle error {code}")
        self.code = code


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data


def _rect(r) -> Rect:
    return Rect(*[int(v) for v in r])


@dataclass
class Image:
    """A stored partial image: pvp/roi in destination coordinates, arrays [h][pitch](...)."""
    pvp: tuple
    roi: tuple
    color: np.ndarray
    depth: Optional[np.ndarray] = None

    @property
    def pitch(self) -> int:
        return int(self.color.shape[1])


def _check_c(a: np.ndarray, what: str):
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError(f"{what} must be C-contiguous")


def _check_covers(im: "Image"):
    """The arrays must hold the pvp's rows and columns (the C code trusts them)."""
    w, h = int(im.pvp[2]), int(im.pvp[3])
    for a in (im.color, im.depth):
        if a is not None and h > 0 and w > 0 and (a.ndim < 2 or a.shape[0] < h or a.shape[1] < w):
            raise ValueError("image arrays are smaller than their pvp")


def composite_depth(images: Sequence[Image], out_pvp, out_pitch: Optional[int] = None):
    """Depth-test merge (thesis 5.2.1).  Colour is any 4/8/16-byte pixel type copied
    bit for bit.  Returns (color, depth, winner, out_roi)."""
    out_pvp = tuple(int(v) for v in out_pvp)
    W, H = out_pvp[2], out_pvp[3]
    pitch = W if out_pitch is None else int(out_pitch)
    srcs = (_DepthSrc * max(1, len(images)))()
    cb = None
    dtype, inner = np.uint32, ()
    for i, im in enumerate(images):
        _check_c(im.color, "color")
        _check_c(im.depth, "depth")
        _check_covers(im)
        b = im.color.itemsize * int(np.prod(im.color.shape[2:], dtype=np.int64))
        if cb is None:
            cb, dtype, inner = b, im.color.dtype, im.color.shape[2:]
        elif cb != b:
            raise ValueError("mixed colour formats")
        srcs[i] = _DepthSrc(_rect(im.pvp), _rect(im.roi), im.pitch, _ptr(im.color), _ptr(im.depth))
    if cb is None:
        cb = 4
    color = np.zeros((max(H, 0), max(pitch, 0)) + tuple(inner), dtype=dtype)
    depth = np.zeros((max(H, 0), max(pitch, 0)), dtype=np.float32)
    winner = np.zeros((max(H, 0), max(W, 0)), dtype=np.int16)
    roi = Rect()
    rc = lib().orc_composite_depth(srcs, len(images), cb, _rect(out_pvp), pitch, _ptr(color),
                                   _ptr(depth), _ptr(winner), C.byref(roi))
    if rc:
        raise OracleError(rc, "composite_depth")
    return color, depth, winner, roi.tup()


def _layers(images: Sequence[Image]):
    arr = (_Layer * max(1, len(images)))()
    fmt = None
    for i, im in enumerate(images):
        _check_c(im.color, "color")
        _check_covers(im)
        f = F32 if im.color.dtype == np.float32 else F16 if im.color.dtype == np.float16 else None
        if f is None or im.color.shape[2:] != (4,):
            raise ValueError("alpha layers are [h][pitch][4] float32 or float16")
        if fmt is None:
            fmt = f
        elif fmt != f:
            raise ValueError("mixed layer formats")
        arr[i] = _Layer(_rect(im.pvp), _rect(im.roi), im.pitch, _ptr(im.color))
    return arr, (fmt or F32)


def _order(order, n):
    if order is None:
        return None
    o = np.ascontiguousarray(np.asarray(order, dtype=np.int32))
    if o.shape != (n,):
        raise ValueError("order must have n entries")
    return o


def composite_alpha(layers: Sequence[Image], out_pvp, order=None):
    """Front-to-back premultiplied 'over' in float64.  Returns (out[h][w][4], T[h][w], out_roi)."""
    out_pvp = tuple(int(v) for v in out_pvp)
    arr, fmt = _layers(layers)
    o = _order(order, len(layers))
    out = np.zeros((out_pvp[3], out_pvp[2], 4), dtype=np.float64)
    t = np.zeros((out_pvp[3], out_pvp[2]), dtype=np.float64)
    roi = Rect()
    rc = lib().orc_composite_alpha(arr, len(layers), fmt, _ptr(o), _rect(out_pvp), _ptr(out),
                                   _ptr(t), C.byref(roi))
    if rc:
        raise OracleError(rc, "composite_alpha")
    return out, t, roi.tup()


def composite_alpha_backward(layers: Sequence[Image], out_pvp, g: np.ndarray, order=None,
                             fill: float = 0.0):
    """dL/dlayer for L = sum(g*out).  Returns one float64 [h][pitch][4] array per layer;
    elements the definition does not write keep ``fill``."""
    out_pvp = tuple(int(v) for v in out_pvp)
    arr, fmt = _layers(layers)
    o = _order(order, len(layers))
    g = np.ascontiguousarray(g, dtype=np.float64)
    grads = [np.full(im.color.shape, fill, dtype=np.float64) for im in layers]
    ptrs = (C.c_void_p * max(1, len(layers)))(*[_ptr(a) for a in grads])
    rc = lib().orc_composite_alpha_backward(arr, len(layers), fmt, _ptr(o), _rect(out_pvp),
                                            _ptr(g), ptrs)
    if rc:
        raise OracleError(rc, "composite_alpha_backward")
    return grads


def composite_depth_backward(winner: np.ndarray, out_pvp, g: np.ndarray, pvps, pitches,
                             fill: float = 0.0):
    """Route the upstream colour gradient to the winning source of every pixel."""
    n = len(pvps)
    winner = np.ascontiguousarray(winner, dtype=np.int16)
    g = np.ascontiguousarray(g, dtype=np.float32)
    grads = [np.full((pvps[i][3], pitches[i], 4), fill, dtype=np.float32) for i in range(n)]
    rp = (Rect * max(1, n))(*[_rect(r) for r in pvps])
    pp = (C.c_int32 * max(1, n))(*[int(p) for p in pitches])
    ptrs = (C.c_void_p * max(1, n))(*[_ptr(a) for a in grads])
    rc = lib().orc_composite_depth_backward(_ptr(winner), _rect(out_pvp), _ptr(g), n, rp, pp,
                                            ptrs)
    if rc:
        raise OracleError(rc, "composite_depth_backward")
    return grads


def _pixel_bytes(a: np.ndarray) -> int:
    return a.itemsize * int(np.prod(a.shape[2:], dtype=np.int64))


def assemble_tiles(images: Sequence[Image], out: np.ndarray, out_pvp) -> np.ndarray:
    """Sort-first / tile assembly: copy every image's roi (clipped to out_pvp) into
    a copy of out ([h][pitch](...)), in order; returns the assembled array."""
    out = np.ascontiguousarray(out).copy()
    bpp = _pixel_bytes(out)
    arr = (_Layer * max(1, len(images)))()
    for i, im in enumerate(images):
        _check_c(im.color, "color")
        if _pixel_bytes(im.color) != bpp:
            raise ValueError("pixel size differs from the output's")
        arr[i] = _Layer(_rect(im.pvp), _rect(im.roi), im.pitch, _ptr(im.color))
    rc = lib().orc_assemble_tiles(arr, len(images), bpp, _rect(out_pvp), out.shape[1] if out.ndim > 1 else 0,
                                  _ptr(out) if out.size else None)
    if rc:
        raise OracleError(rc, "assemble_tiles")
    return out


def assemble_pixels(srcs: Sequence[np.ndarray], offsets, kernel, out: np.ndarray, out_pvp) -> np.ndarray:
    """Pixel-compound assembly: source k ([h_k][pitch_k](...)) holds the destination
    pixels at offsets (kx + i*nx, ky + j*ny); returns the assembled copy of out."""
    out = np.ascontiguousarray(out).copy()
    bpp = _pixel_bytes(out)
    n = len(srcs)
    for a in srcs:
        _check_c(a, "source")
    ptrs = (C.c_void_p * max(1, n))(*[_ptr(a) for a in srcs])
    pitches = (C.c_int32 * max(1, n))(*[int(a.shape[1]) for a in srcs])
    kx = (C.c_int32 * max(1, n))(*[int(o[0]) for o in offsets])
    ky = (C.c_int32 * max(1, n))(*[int(o[1]) for o in offsets])
    rc = lib().orc_assemble_pixels(ptrs, pitches, kx, ky, n, int(kernel[0]), int(kernel[1]), bpp,
                                   _rect(out_pvp), out.shape[1], _ptr(out) if out.size else None)
    if rc:
        raise OracleError(rc, "assemble_pixels")
    return out


def average(images: Sequence[Image], out_pvp, fmt: int) -> np.ndarray:
    """Subpixel-compound assembly: per-pixel average of the sources whose roi holds
    it.  fmt 0 (RGBA8): uint32 [h][w] with integer rounding; fmt 1/2 (float32 /
    float16 storage): float64 [h][w][4]."""
    W, H = max(out_pvp[2], 0), max(out_pvp[3], 0)
    arr = (_Layer * max(1, len(images)))()
    for i, im in enumerate(images):
        _check_c(im.color, "color")
        arr[i] = _Layer(_rect(im.pvp), _rect(im.roi), im.pitch, _ptr(im.color))
    out = np.zeros((H, W), dtype=np.uint32) if fmt == 0 else np.zeros((H, W, 4), dtype=np.float64)
    rc = lib().orc_average(arr, len(images), int(fmt), _rect(out_pvp), W, _ptr(out) if out.size else None)
    if rc:
        raise OracleError(rc, "average")
    return out


def detect_roi(pvp, search, pitch: int, fmt: int, color: Optional[np.ndarray] = None,
               depth: Optional[np.ndarray] = None, tile: int = 64):
    """Automatic ROI (thesis 5.3): bounding box of the data pixels of the
    examined region, and the tile occupancy grid.  color: [pvp.h][pitch] uint32
    (RGBA8), [..][4] float32 or [..][4] uint16 half bits; depth: float32."""
    gw, gh = -(-max(pvp[2], 0) // tile), -(-max(pvp[3], 0) // tile)
    # the grid, then a guard region that must stay zero: the oracle never writes
    # there, a planted indexing mistake that does is caught instead of
    # corrupting the process's heap
    guard = 65536 + gw * max(gw, gh)
    buf = np.zeros(gh * gw + guard, dtype=np.uint8)
    occ = buf[:gh * gw].reshape(gh, gw)
    c = None if color is None else np.ascontiguousarray(color)
    d = None if depth is None else np.ascontiguousarray(depth, dtype=np.float32)
    out = Rect()
    rc = lib().orc_detect_roi(_rect(pvp), _rect(search), int(pitch), int(fmt),
                              None if c is None else _ptr(c), None if d is None else _ptr(d),
                              int(tile), _ptr(buf) if occ.size else None, C.byref(out))
    if rc:
        raise OracleError(rc, "detect_roi")
    if buf[gh * gw:].any():
        raise OracleError(EINVAL, "detect_roi wrote past the occupancy grid")
    return (out.x, out.y, out.w, out.h), occ.copy()


def rle_max_size(w: int, h: int) -> int:
    return int(lib().orc_rle_max_size(int(w), int(h)))


def swizzle(v: int) -> int:
    return int(lib().orc_swizzle(int(v) & 0xFFFFFFFF))


def unswizzle(v: int) -> int:
    return int(lib().orc_unswizzle(int(v) & 0xFFFFFFFF))


def rle_compress(src: np.ndarray, mode: int, w: Optional[int] = None) -> bytes:
    """Compress a [h][pitch] array of 4-byte elements (the first w columns)."""
    if src.itemsize != 4 or src.ndim != 2:
        raise ValueError("src must be a 2-D array of 4-byte elements")
    _check_c(src, "src")
    h, pitch = src.shape
    w = pitch if w is None else int(w)
    cap = rle_max_size(w, h)
    # a guard region past the declared capacity: the oracle never writes there,
    # but a planted mistake that overruns is caught as a wrong size instead of
    # corrupting the process's heap
    dst = np.zeros(max(cap, 1) + 65536, dtype=np.uint8)
    n = lib().orc_rle_compress(_ptr(src), w, h, pitch, int(mode), _ptr(dst), cap)
    if n < 0:
        raise OracleError(-n, "rle_compress")
    if n > cap:
        raise OracleError(ECAP, "rle_compress wrote past its capacity")
    return dst[:n].tobytes()


def yuv_encode(src: np.ndarray, w: Optional[int] = None) -> np.ndarray:
    """Lossy YUV conversion with 2x2 chroma subsampling (thesis 5.5.3) of a
    [h][pitch] RGBA8 (uint32) image: returns the packed [2*ceil(h/2)][ceil(w/2)]
    uint32 image (luma words, then chroma words)."""
    if src.dtype != np.uint32 or src.ndim != 2:
        raise ValueError("src must be a [h][pitch] uint32 array")
    _check_c(src, "src")
    h, pitch = src.shape
    w = pitch if w is None else int(w)
    out = np.zeros((2 * ((h + 1) // 2), (w + 1) // 2), dtype=np.uint32)
    rc = lib().orc_yuv_encode(_ptr(src), w, h, pitch, _ptr(out))
    if rc:
        raise OracleError(rc, "yuv_encode")
    return out


def yuv_decode(packed: np.ndarray, w: int, h: int) -> np.ndarray:
    """Inverse of yuv_encode up to its loss: a [h][w] RGBA8 (uint32) image."""
    packed = np.ascontiguousarray(packed, dtype=np.uint32)
    if packed.shape != (2 * ((h + 1) // 2), (w + 1) // 2):
        raise ValueError("packed image has the wrong shape")
    out = np.zeros((h, w), dtype=np.uint32)
    rc = lib().orc_yuv_decode(_ptr(packed), w, h, _ptr(out), w)
    if rc:
        raise OracleError(rc, "yuv_decode")
    return out


def rle_decompress(buf: bytes, w: int, h: int, pitch: Optional[int] = None,
                   dtype=np.uint32) -> np.ndarray:
    pitch = w if pitch is None else int(pitch)
    src = np.frombuffer(bytes(buf), dtype=np.uint8).copy()
    dst = np.zeros((h, pitch), dtype=dtype)
    rc = lib().orc_rle_decompress(_ptr(src) if len(src) else None, len(src), _ptr(dst), w, h,
                                  pitch)
    if rc:
        raise OracleError(rc, "rle_decompress")
    return dst


def rle_decompress_status(buf: bytes, w: int, h: int) -> int:
    """Return code of decoding ``buf`` (0 = valid stream)."""
    src = np.frombuffer(bytes(buf), dtype=np.uint8).copy()
    dst = np.zeros((max(h, 1), max(w, 1)), dtype=np.uint32)
    return int(lib().orc_rle_decompress(_ptr(src) if len(src) else None, len(src), _ptr(dst),
                                        w, h, max(w, 1)))
