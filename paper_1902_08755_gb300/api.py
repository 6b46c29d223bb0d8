"""Python binding of libec: the C ABI of include/ec.h over torch tensors.

Argument marshalling only -- every step runs in the CUDA kernels behind the C
ABI.  Tensors must live on the context's CUDA device; the functions enqueue
work on the current torch stream (or the one given) and return at once.
Names follow the C ABI without its ``ec_`` prefix.

Tensor layouts (pitch = row stride in pixels, taken from the tensor's stride):
  RGBA8    uint32 [h][pitch]          (R in the low byte)
  RGBA32F  float32 [h][pitch][4]
  RGBA16F  float16 [h][pitch][4]
  depth    float32 [h][pitch], same pitch as the colour
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass
from typing import List, Optional, Sequence, Tuple

import torch

from . import _abi as A
from ._abi import EcError, check, ec_image, ec_rect, ec_rle_job, ec_target

Rect = Tuple[int, int, int, int]


def _lib():
    return A.load()


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Context:
    """An ec_ctx: device status word and codec scratch memory on one device."""

    def __init__(self, device: Optional[int] = None):
        if not torch.cuda.is_available():
            raise RuntimeError("libec needs a CUDA device")
        self.device = torch.cuda.current_device() if device is None else int(device)
        h = C.c_void_p()
        check(_lib().ec_create(C.byref(h), self.device), "ec_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            _lib().ec_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def status_sync(self, stream=None) -> int:
        """Wait for the stream; return and clear the first device-side error."""
        return int(_lib().ec_status_sync(self.h, _stream_handle(stream)))

    def check_status(self, stream=None, what: str = "device"):
        check(self.status_sync(stream), what)


_default_ctx = {}


def default_context(device: Optional[int] = None) -> Context:
    dev = torch.cuda.current_device() if device is None else int(device)
    if dev not in _default_ctx:
        _default_ctx[dev] = Context(dev)
    return _default_ctx[dev]


@dataclass
class Image:
    """One input frame: colour (and depth) buffers, pixel viewport and ROI."""
    color: torch.Tensor
    depth: Optional[torch.Tensor] = None
    pvp: Optional[Rect] = None
    roi: Optional[Rect] = None


def pixel_layout(t: torch.Tensor) -> Tuple[int, int, int, int]:
    """(format, pitch, width, height) of a colour tensor."""
    if t.dim() == 2 and t.dtype in (torch.uint32, torch.int32):
        if t.stride(1) != 1:
            raise ValueError("RGBA8 tensor needs unit column stride")
        return A.EC_RGBA8, t.stride(0), t.shape[1], t.shape[0]
    if t.dim() == 3 and t.shape[2] == 4 and t.dtype in (torch.float32, torch.float16):
        if t.stride(2) != 1 or t.stride(1) != 4 or t.stride(0) % 4:
            raise ValueError("RGBA float tensor needs strides (4*pitch, 4, 1)")
        fmt = A.EC_RGBA32F if t.dtype == torch.float32 else A.EC_RGBA16F
        return fmt, t.stride(0) // 4, t.shape[1], t.shape[0]
    raise ValueError(f"unsupported colour tensor {t.dtype} {tuple(t.shape)}")


def _rect(r) -> ec_rect:
    return ec_rect(*[int(v) for v in r])


def _on_device(t: Optional[torch.Tensor], dev: int, what: str):
    if t is None:
        return
    if not t.is_cuda or t.device.index != dev:
        raise ValueError(f"{what} must be a CUDA tensor on device {dev}")


def _image_struct(im: Image, dev: int, need_depth: bool) -> ec_image:
    fmt, pitch, w, h = pixel_layout(im.color)
    _on_device(im.color, dev, "colour")
    pvp = tuple(im.pvp) if im.pvp is not None else (0, 0, w, h)
    roi = tuple(im.roi) if im.roi is not None else pvp
    if pvp[2] > w or pvp[3] > h:
        raise ValueError("pvp larger than the colour tensor")
    dptr = None
    if need_depth:
        if im.depth is None:
            raise ValueError("depth compositing needs depth buffers")
        _on_device(im.depth, dev, "depth")
        d = im.depth
        if d.dtype != torch.float32 or d.dim() != 2 or d.stride(1) != 1 or d.stride(0) != pitch \
                or d.shape[0] < pvp[3] or d.shape[1] < pvp[2]:
            raise ValueError("depth must be float32 [h][pitch] with the colour's pitch")
        dptr = d.data_ptr()
    return ec_image(_rect(pvp), _rect(roi), pitch, fmt, im.color.data_ptr(), dptr)


def _target(color: torch.Tensor, depth: Optional[torch.Tensor], pvp, dev: int) -> ec_target:
    fmt, pitch, w, h = pixel_layout(color)
    _on_device(color, dev, "output colour")
    pvp = tuple(pvp) if pvp is not None else (0, 0, w, h)
    if pvp[2] > w or pvp[3] > h:
        raise ValueError("output pvp larger than the output tensor")
    dptr = None
    if depth is not None:
        _on_device(depth, dev, "output depth")
        if depth.dtype != torch.float32 or depth.stride(0) != pitch or depth.stride(1) != 1:
            raise ValueError("output depth must be float32 with the colour's pitch")
        dptr = depth.data_ptr()
    return ec_target(_rect(pvp), pitch, fmt, color.data_ptr(), dptr)


def _dense(t: Optional[torch.Tensor], shape, dtype, dev: int, what: str) -> Optional[int]:
    if t is None:
        return None
    _on_device(t, dev, what)
    if t.dtype != dtype or not t.is_contiguous() or t.numel() < int(torch.tensor(shape).prod()):
        raise ValueError(f"{what} must be a contiguous {dtype} tensor of shape {shape}")
    return t.data_ptr()


def composite_depth(images: Sequence[Image], out_color: torch.Tensor,
                    out_depth: Optional[torch.Tensor] = None, out_pvp: Optional[Rect] = None,
                    winner: Optional[torch.Tensor] = None, ctx: Optional[Context] = None,
                    stream=None) -> Rect:
    """ec_composite_depth: per-pixel depth-test merge.  Returns the merged ROI."""
    ctx = ctx or default_context(out_color.device.index)
    dev = ctx.device
    arr = (ec_image * max(1, len(images)))(*[_image_struct(im, dev, True) for im in images])
    tgt = _target(out_color, out_depth, out_pvp, dev)
    wp = _dense(winner, (tgt.pvp.h, tgt.pvp.w), torch.int16, dev, "winner")
    roi = ec_rect()
    check(_lib().ec_composite_depth(ctx.h, arr, len(images), C.byref(tgt), wp, C.byref(roi),
                                    _stream_handle(stream)), "ec_composite_depth")
    return roi.tup()


def _order(order, n):
    if order is None:
        return None
    o = (C.c_int32 * max(1, n))(*[int(v) for v in order])
    if len(order) != n:
        raise ValueError("order needs one entry per layer")
    return o


def composite_alpha(layers: Sequence[Image], out: torch.Tensor, order=None,
                    out_pvp: Optional[Rect] = None, t_final: Optional[torch.Tensor] = None,
                    ctx: Optional[Context] = None, stream=None) -> Rect:
    """ec_composite_alpha: front-to-back premultiplied 'over'.  Returns the merged ROI."""
    ctx = ctx or default_context(out.device.index)
    dev = ctx.device
    arr = (ec_image * max(1, len(layers)))(*[_image_struct(im, dev, False) for im in layers])
    tgt = _target(out, None, out_pvp, dev)
    tp = _dense(t_final, (tgt.pvp.h, tgt.pvp.w), torch.float32, dev, "t_final")
    roi = ec_rect()
    check(_lib().ec_composite_alpha(ctx.h, arr, _order(order, len(layers)), len(layers),
                                    C.byref(tgt), tp, C.byref(roi), _stream_handle(stream)),
          "ec_composite_alpha")
    return roi.tup()


def composite_alpha_backward(layers: Sequence[Image], out_pvp: Rect, grad_out: torch.Tensor,
                             grads: Sequence[torch.Tensor], order=None,
                             ctx: Optional[Context] = None, stream=None):
    """ec_composite_alpha_backward: dL/dlayer for L = sum(grad_out * out)."""
    ctx = ctx or default_context(grad_out.device.index)
    dev = ctx.device
    n = len(layers)
    arr = (ec_image * max(1, n))(*[_image_struct(im, dev, False) for im in layers])
    gp = _dense(grad_out, (out_pvp[3], out_pvp[2], 4), torch.float32, dev, "grad_out")
    gfmt = _grad_format(grads, layers, dev)
    ptrs = (C.c_void_p * max(1, n))(*[g.data_ptr() for g in grads])
    check(_lib().ec_composite_alpha_backward(ctx.h, arr, _order(order, n), n, _rect(out_pvp), gp,
                                             ptrs, gfmt, _stream_handle(stream)),
          "ec_composite_alpha_backward")


def _grad_format(grads, layers, dev) -> int:
    if len(grads) != len(layers):
        raise ValueError("one gradient buffer per layer")
    fmt = None
    for g, im in zip(grads, layers):
        _on_device(g, dev, "gradient")
        f, pitch, w, h = pixel_layout(g)
        if f == A.EC_RGBA8 or pitch != pixel_layout(im.color)[1] or g.shape[:2] != im.color.shape[:2]:
            raise ValueError("gradients must have their layer's shape and pitch (float32/float16)")
        if fmt is not None and f != fmt:
            raise ValueError("all gradients share one format")
        fmt = f
    return A.EC_RGBA32F if fmt is None else fmt


def composite_alpha_fwd_bwd(layers: Sequence[Image], out: torch.Tensor, w: torch.Tensor,
                            grads: Sequence[torch.Tensor], order=None,
                            out_pvp: Optional[Rect] = None, t_final: Optional[torch.Tensor] = None,
                            ctx: Optional[Context] = None, stream=None) -> Rect:
    """ec_composite_alpha_fwd_bwd: forward and gradients of sum(w * out) in one pass."""
    ctx = ctx or default_context(out.device.index)
    dev = ctx.device
    n = len(layers)
    arr = (ec_image * max(1, n))(*[_image_struct(im, dev, False) for im in layers])
    tgt = _target(out, None, out_pvp, dev)
    tp = _dense(t_final, (tgt.pvp.h, tgt.pvp.w), torch.float32, dev, "t_final")
    wp = _dense(w, (tgt.pvp.h, tgt.pvp.w, 4), torch.float32, dev, "w")
    gfmt = _grad_format(grads, layers, dev)
    ptrs = (C.c_void_p * max(1, n))(*[g.data_ptr() for g in grads])
    roi = ec_rect()
    check(_lib().ec_composite_alpha_fwd_bwd(ctx.h, arr, _order(order, n), n, C.byref(tgt), tp, wp,
                                            ptrs, gfmt, C.byref(roi), _stream_handle(stream)),
          "ec_composite_alpha_fwd_bwd")
    return roi.tup()


def assemble_tiles(images: Sequence[Image], out: torch.Tensor, out_pvp: Optional[Rect] = None,
                   ctx: Optional[Context] = None, stream=None):
    """ec_assemble_tiles: copy every image's roi into out (later images win)."""
    ctx = ctx or default_context(out.device.index)
    dev = ctx.device
    n = len(images)
    arr = (ec_image * max(1, n))(*[_image_struct(im, dev, False) for im in images])
    tgt = _target(out, None, out_pvp, dev)
    check(_lib().ec_assemble_tiles(ctx.h, arr, n, C.byref(tgt), _stream_handle(stream)), "ec_assemble_tiles")


def average(images: Sequence[Image], out: torch.Tensor, out_pvp: Optional[Rect] = None,
            ctx: Optional[Context] = None, stream=None):
    """ec_average: per-pixel average of the images whose roi holds the pixel."""
    ctx = ctx or default_context(out.device.index)
    dev = ctx.device
    n = len(images)
    arr = (ec_image * max(1, n))(*[_image_struct(im, dev, False) for im in images])
    tgt = _target(out, None, out_pvp, dev)
    check(_lib().ec_average(ctx.h, arr, n, C.byref(tgt), _stream_handle(stream)), "ec_average")


def assemble_pixels(sources: Sequence[torch.Tensor], offsets, kernel, out: torch.Tensor,
                    out_pvp: Optional[Rect] = None, ctx: Optional[Context] = None, stream=None):
    """ec_assemble_pixels: sources[k] holds the pixels at offsets (kx + i*nx, ky + j*ny)."""
    ctx = ctx or default_context(out.device.index)
    dev = ctx.device
    n = len(sources)
    structs = []
    for t in sources:
        fmt, pitch, w, h = pixel_layout(t)
        _on_device(t, dev, "source")
        structs.append(ec_image(_rect((0, 0, w, h)), _rect((0, 0, w, h)), pitch, fmt, t.data_ptr(), None))
    arr = (ec_image * max(1, n))(*structs)
    kx = (C.c_int32 * max(1, n))(*[int(o[0]) for o in offsets])
    ky = (C.c_int32 * max(1, n))(*[int(o[1]) for o in offsets])
    tgt = _target(out, None, out_pvp, dev)
    check(_lib().ec_assemble_pixels(ctx.h, arr, kx, ky, n, int(kernel[0]), int(kernel[1]), C.byref(tgt),
                                    _stream_handle(stream)), "ec_assemble_pixels")


def detect_roi(images: Sequence[Image], tile: int = 64, occupancy: bool = True,
               ctx: Optional[Context] = None, stream=None):
    """ec_detect_roi: bounding box of each image's data pixels inside its roi
    (depth < 1.0 when a depth buffer is given, else a non-zero colour), and
    optionally its tile occupancy grid (holes are the 0 tiles).

    Returns (rois, grids): rois is an int32 [n][4] device tensor of (x, y, w, h)
    in destination coordinates ((0,0,0,0) when nothing is found); grids is a list
    of uint8 [ceil(pvp.h/tile)][ceil(pvp.w/tile)] device tensors, or None."""
    n = len(images)
    dev = (ctx.device if ctx else (images[0].color.device.index if n else torch.cuda.current_device()))
    ctx = ctx or default_context(dev)
    dev = ctx.device
    structs = []
    for im in images:
        fmt, pitch, w, h = pixel_layout(im.color)
        _on_device(im.color, dev, "colour")
        pvp = tuple(im.pvp) if im.pvp is not None else (0, 0, w, h)
        roi = tuple(im.roi) if im.roi is not None else pvp
        if pvp[2] > w or pvp[3] > h:
            raise ValueError("pvp larger than the colour tensor")
        dptr = None
        if im.depth is not None:
            _on_device(im.depth, dev, "depth")
            dd = im.depth
            if dd.dtype != torch.float32 or dd.dim() != 2 or dd.stride(1) != 1 or dd.stride(0) != pitch \
                    or dd.shape[0] < pvp[3] or dd.shape[1] < pvp[2]:
                raise ValueError("depth must be float32 [h][pitch] with the colour's pitch")
            dptr = dd.data_ptr()
        structs.append(ec_image(_rect(pvp), _rect(roi), pitch, fmt, im.color.data_ptr(), dptr))
    arr = (ec_image * max(1, n))(*structs)
    rois = torch.zeros((max(n, 1), 4), dtype=torch.int32, device=f"cuda:{dev}")[:n]
    grids, occ = None, None
    if occupancy:
        grids = [torch.empty((-(-s.pvp.h // tile), -(-s.pvp.w // tile)), dtype=torch.uint8, device=f"cuda:{dev}")
                 for s in structs]
        occ = (C.c_void_p * max(1, n))(*[g.data_ptr() if g.numel() else None for g in grids])
    check(_lib().ec_detect_roi(ctx.h, arr, n, int(tile), occ, rois.data_ptr() if n else None,
                               _stream_handle(stream)), "ec_detect_roi")
    return rois, grids


def composite_depth_backward(winner: torch.Tensor, out_pvp: Rect, grad_out: torch.Tensor,
                             images: Sequence[Image], grads: Sequence[torch.Tensor],
                             ctx: Optional[Context] = None, stream=None):
    """ec_composite_depth_backward: route grad_out to each pixel's winning input."""
    ctx = ctx or default_context(grad_out.device.index)
    dev = ctx.device
    n = len(images)
    wp = _dense(winner, (out_pvp[3], out_pvp[2]), torch.int16, dev, "winner")
    gp = _dense(grad_out, (out_pvp[3], out_pvp[2], 4), torch.float32, dev, "grad_out")
    pvps, pitches = [], []
    for im, g in zip(images, grads):
        f, pitch, w, h = pixel_layout(im.color)
        gf, gpitch, _, _ = pixel_layout(g)
        if gf != A.EC_RGBA32F or gpitch != pitch:
            raise ValueError("depth gradients are float32 [h][pitch][4] with the input's pitch")
        _on_device(g, dev, "gradient")
        pvps.append(_rect(im.pvp if im.pvp is not None else (0, 0, w, h)))
        pitches.append(pitch)
    rp = (ec_rect * max(1, n))(*pvps)
    pp = (C.c_int32 * max(1, n))(*pitches)
    ptrs = (C.c_void_p * max(1, n))(*[g.data_ptr() for g in grads])
    check(_lib().ec_composite_depth_backward(ctx.h, wp, _rect(out_pvp), gp, n, rp, pp, ptrs,
                                             _stream_handle(stream)),
          "ec_composite_depth_backward")


def yuv_packed_shape(w: int, h: int) -> Tuple[int, int]:
    """(rows, words) of the packed image of a w x h frame."""
    return 2 * ((h + 1) // 2), (w + 1) // 2


def yuv_encode(src: torch.Tensor, w: Optional[int] = None, out: Optional[torch.Tensor] = None,
               ctx: Optional[Context] = None, stream=None) -> torch.Tensor:
    """ec_yuv_encode: lossy YUV with 2x2 chroma blocks (thesis 5.5.3) of a
    [h][pitch] RGBA8 (uint32/int32) image; returns the packed uint32 image."""
    ctx = ctx or default_context(src.device.index)
    pitch, wt, h = _elem_layout(src)
    w = wt if w is None else int(w)
    rows, words = yuv_packed_shape(w, h)
    if out is None:
        out = torch.empty((rows, words), dtype=torch.int32, device=src.device).view(torch.uint32)
    opitch, ow, oh = _elem_layout(out)
    if ow < words or oh < rows:
        raise ValueError("packed output too small")
    check(_lib().ec_yuv_encode(ctx.h, src.data_ptr(), w, h, pitch, out.data_ptr(), opitch,
                               _stream_handle(stream)), "ec_yuv_encode")
    return out


def yuv_decode(packed: torch.Tensor, w: int, h: int, out: Optional[torch.Tensor] = None,
               ctx: Optional[Context] = None, stream=None) -> torch.Tensor:
    """ec_yuv_decode: RGBA8 [h][w] (or into out, any pitch) from a packed image."""
    ctx = ctx or default_context(packed.device.index)
    spitch, sw, sh = _elem_layout(packed)
    rows, words = yuv_packed_shape(w, h)
    if sw < words or sh < rows:
        raise ValueError("packed image too small")
    if out is None:
        out = torch.empty((h, w), dtype=torch.int32, device=packed.device).view(torch.uint32)
    pitch, ow, oh = _elem_layout(out)
    if ow < w or oh < h:
        raise ValueError("output too small")
    check(_lib().ec_yuv_decode(ctx.h, packed.data_ptr(), spitch, w, h, out.data_ptr(), pitch,
                               _stream_handle(stream)), "ec_yuv_decode")
    return out


def yuv_batch(jobs, encode: bool, ctx: Optional[Context] = None, stream=None):
    """ec_yuv_encode_batch / ec_yuv_decode_batch over [(src, dst, w, h)]: encode
    reads RGBA8 src and writes packed dst, decode the reverse (one launch)."""
    prepare_yuv_batch(jobs, encode, ctx).run(stream)


def prepare_yuv_batch(jobs, encode: bool, ctx: Optional[Context] = None) -> "Prepared":
    """Prepared ec_yuv_encode_batch / ec_yuv_decode_batch."""
    ctx = ctx or default_context(jobs[0][0].device.index)
    arr = (A.ec_yuv_job * max(1, len(jobs)))()
    for i, (src, dst, w, h) in enumerate(jobs):
        rgba, packed = (src, dst) if encode else (dst, src)
        pitch, rw, rh = _elem_layout(rgba)
        ppitch, pw, ph = _elem_layout(packed)
        rows, words = yuv_packed_shape(w, h)
        if rw < w or rh < h or pw < words or ph < rows:
            raise ValueError("yuv job: tensors too small")
        arr[i] = A.ec_yuv_job(src.data_ptr(), dst.data_ptr(), int(w), int(h), pitch, ppitch)
    fn = _lib().ec_yuv_encode_batch if encode else _lib().ec_yuv_decode_batch
    return Prepared(fn, ctx, arr, len(jobs), "ec_yuv_batch", list(jobs))


def rle_max_size(w: int, h: int) -> int:
    return int(_lib().ec_rle_max_size(int(w), int(h)))


def _elem_layout(t: torch.Tensor) -> Tuple[int, int, int]:
    """(pitch, w, h) of a 2-D tensor of 4-byte elements."""
    if t.dim() != 2 or t.element_size() != 4:
        raise ValueError("codec images are 2-D tensors of 4-byte elements")
    if t.numel() == 0:
        return t.shape[1], t.shape[1], t.shape[0]
    if t.stride(1) != 1:
        raise ValueError("codec images need unit column stride")
    return t.stride(0), t.shape[1], t.shape[0]


def rle_compress(src: torch.Tensor, mode: int, w: Optional[int] = None,
                 dst: Optional[torch.Tensor] = None, d_size: Optional[torch.Tensor] = None,
                 ctx: Optional[Context] = None, stream=None):
    """ec_rle_compress.  Returns (dst uint8 buffer, d_size uint64[1] device tensor)."""
    ctx = ctx or default_context(src.device.index)
    jobs = [(src, mode, w, dst, d_size)]
    out = rle_compress_batch(jobs, ctx=ctx, stream=stream)
    return out[0]


class Prepared:
    """A batched call whose argument array is built once; run() only enqueues
    it (for frame loops and for timing the kernels rather than the marshalling).
    The tensors named by the jobs must stay alive and in place."""

    def __init__(self, fn, ctx, arr, n, what, keep):
        self.fn, self.ctx, self.arr, self.n, self.what, self._keep = fn, ctx, arr, n, what, keep

    def run(self, stream=None):
        check(self.fn(self.ctx.h, self.arr, self.n, _stream_handle(stream)), self.what)


def prepare_rle_compress_batch(jobs, ctx: Optional[Context] = None):
    """Prepared ec_rle_compress_batch; returns (Prepared, [(dst, d_size)])."""
    ctx = ctx or default_context(jobs[0][0].device.index)
    arr, outs = _rle_compress_jobs(jobs, ctx)
    return Prepared(_lib().ec_rle_compress_batch, ctx, arr, len(jobs), "ec_rle_compress_batch",
                    [jobs, outs]), outs


def prepare_rle_decompress_batch(jobs, ctx: Optional[Context] = None):
    """Prepared ec_rle_decompress_batch; returns (Prepared, [dst])."""
    ctx = ctx or default_context(jobs[0][0].device.index)
    arr, outs = _rle_decompress_jobs(jobs, ctx)
    return Prepared(_lib().ec_rle_decompress_batch, ctx, arr, len(jobs), "ec_rle_decompress_batch",
                    [jobs, outs]), outs


def rle_compress_batch(jobs, ctx: Optional[Context] = None, stream=None):
    """ec_rle_compress_batch over [(src, mode, w|None, dst|None, d_size|None)].
    Returns [(dst, d_size)]."""
    ctx = ctx or default_context(jobs[0][0].device.index)
    arr, outs = _rle_compress_jobs(jobs, ctx)
    check(_lib().ec_rle_compress_batch(ctx.h, arr, len(jobs), _stream_handle(stream)),
          "ec_rle_compress_batch")
    return outs


def _rle_compress_jobs(jobs, ctx):
    dev = ctx.device
    arr = (ec_rle_job * max(1, len(jobs)))()
    outs = []
    for i, (src, mode, w, dst, d_size) in enumerate(jobs):
        _on_device(src, dev, "codec source")
        pitch, tw, h = _elem_layout(src)
        w = tw if w is None else int(w)
        cap = rle_max_size(w, h)
        if dst is None:
            dst = torch.empty(max(cap, 16), dtype=torch.uint8, device=src.device)
        if d_size is None:
            d_size = torch.zeros(1, dtype=torch.uint64, device=src.device)
        _on_device(dst, dev, "codec destination")
        arr[i] = ec_rle_job(src.data_ptr(), dst.data_ptr(), dst.numel() * dst.element_size(),
                            d_size.data_ptr(), w, h, pitch, int(mode))
        outs.append((dst, d_size))
    return arr, outs


def rle_decompress(src: torch.Tensor, w: int, h: int, dst: Optional[torch.Tensor] = None,
                   src_size: Optional[int] = None, ctx: Optional[Context] = None, stream=None):
    """ec_rle_decompress into a uint32 [h][w] tensor (or the given dst)."""
    ctx = ctx or default_context(src.device.index)
    return rle_decompress_batch([(src, w, h, dst, src_size)], ctx=ctx, stream=stream)[0]


def rle_decompress_batch(jobs, ctx: Optional[Context] = None, stream=None):
    """ec_rle_decompress_batch over [(src, w, h, dst|None, src_size|None)]."""
    ctx = ctx or default_context(jobs[0][0].device.index)
    arr, outs = _rle_decompress_jobs(jobs, ctx)
    check(_lib().ec_rle_decompress_batch(ctx.h, arr, len(jobs), _stream_handle(stream)),
          "ec_rle_decompress_batch")
    return outs


def _rle_decompress_jobs(jobs, ctx):
    dev = ctx.device
    arr = (ec_rle_job * max(1, len(jobs)))()
    outs = []
    for i, (src, w, h, dst, src_size) in enumerate(jobs):
        _on_device(src, dev, "codec stream")
        if dst is None:
            dst = torch.empty((h, w), dtype=torch.uint32, device=src.device)
        _on_device(dst, dev, "codec destination")
        pitch, dw, dh = _elem_layout(dst)
        if dw < w or dh < h:
            raise ValueError("destination smaller than the image")
        size = src.numel() * src.element_size() if src_size is None else int(src_size)
        arr[i] = ec_rle_job(src.data_ptr(), dst.data_ptr(), size, None, int(w), int(h), pitch, 0)
        outs.append(dst)
    return arr, outs


# ------------------------------------------------------------------ batches


@dataclass
class Job:
    """One composite of a batch: mode 'depth' or 'alpha', inputs, destination."""
    mode: str
    images: Sequence[Image]
    out_color: torch.Tensor
    out_depth: Optional[torch.Tensor] = None
    out_pvp: Optional[Rect] = None
    order: Optional[Sequence[int]] = None
    winner: Optional[torch.Tensor] = None
    t_final: Optional[torch.Tensor] = None


class Batch:
    """ec_batch: many composites in one persistent, graph-captured launch.

    ``config=None`` autotunes the tile shapes on the jobs themselves (running
    them, so the destinations are written during construction).  The tensors
    must stay alive and in place while the batch exists."""

    def __init__(self, jobs: Sequence[Job], config: Optional[dict] = None,
                 ctx: Optional[Context] = None):
        self.ctx = ctx or default_context(jobs[0].out_color.device.index if jobs else None)
        dev = self.ctx.device
        self._keep = []
        arr = (A.ec_job * max(1, len(jobs)))()
        for k, jb in enumerate(jobs):
            depth = jb.mode == "depth"
            imgs = (ec_image * max(1, len(jb.images)))(*[_image_struct(im, dev, depth) for im in jb.images])
            order = None if depth else _order(jb.order, len(jb.images))
            tgt = _target(jb.out_color, jb.out_depth if depth else None, jb.out_pvp, dev)
            wp = _dense(jb.winner, (tgt.pvp.h, tgt.pvp.w), torch.int16, dev, "winner") if depth else None
            tp = None if depth else _dense(jb.t_final, (tgt.pvp.h, tgt.pvp.w), torch.float32, dev, "t_final")
            self._keep += [imgs, order, jb]
            arr[k] = A.ec_job(A.EC_JOB_DEPTH if depth else A.EC_JOB_ALPHA, len(jb.images),
                              C.cast(imgs, C.c_void_p), None if order is None else C.cast(order, C.c_void_p),
                              tgt, wp, tp)
        cfg = None
        if config is not None:
            cfg = A.ec_batch_config(config.get("depth_tile_w", 128), config.get("depth_tile_h", 8),
                                    config.get("alpha32_tile_w", 32), config.get("alpha32_tile_h", 8),
                                    config.get("alpha16_tile_w", 64), config.get("alpha16_tile_h", 8),
                                    config.get("ctas_per_sm", 0))
        h = C.c_void_p()
        check(_lib().ec_batch_plan(self.ctx.h, arr, len(jobs), C.byref(cfg) if cfg else None,
                                   C.byref(h)), "ec_batch_plan")
        self.h = h

    def run(self, stream=None):
        check(_lib().ec_batch_run(self.h, _stream_handle(stream)), "ec_batch_run")

    @property
    def config(self) -> dict:
        cfg = A.ec_batch_config()
        n = C.c_int32()
        g = C.c_int32()
        check(_lib().ec_batch_get_config(self.h, C.byref(cfg), C.byref(n), C.byref(g)), "ec_batch_get_config")
        d = {f: getattr(cfg, f) for f, _ in cfg._fields_}
        d["n_items"] = n.value
        d["grid"] = g.value
        return d

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            _lib().ec_batch_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


SCHEDULES = {"stream": A.EC_SCHED_STREAM, "direct_send": A.EC_SCHED_DIRECT_SEND,
             "binary_swap": A.EC_SCHED_BINARY_SWAP, "two_three_swap": A.EC_SCHED_TWO_THREE_SWAP}


def schedule_geometry(algorithm: str, rois, frame):
    """ec_schedule_geometry (host only): ([(level, sender, receiver, (x, y, w, h))],
    n_levels, [final region per resource]) of a schedule over resources whose
    data lies in rois (frame coordinates)."""
    n = len(rois)
    arr = (ec_rect * max(1, n))(*[_rect(r) for r in rois])
    regions = (ec_rect * max(1, n))()
    nm, nl = C.c_int32(), C.c_int32()
    code = _lib().ec_schedule_geometry(SCHEDULES[algorithm], arr, n, _rect(frame), None, 0, C.byref(nm),
                                       C.byref(nl), regions)
    if code not in (A.EC_OK, A.EC_ERR_CAPACITY):
        check(code, "ec_schedule_geometry")
    msgs = (A.ec_sched_message * max(1, nm.value))()
    check(_lib().ec_schedule_geometry(SCHEDULES[algorithm], arr, n, _rect(frame), msgs, nm.value, C.byref(nm),
                                      C.byref(nl), regions), "ec_schedule_geometry")
    return ([(m.level, m.sender, m.receiver, (m.piece.x, m.piece.y, m.piece.w, m.piece.h)) for m in msgs[:nm.value]],
            nl.value, [(r.x, r.y, r.w, r.h) for r in regions[:n]])


class Schedule:
    """ec_schedule: a multi-stage compositing schedule (thesis 5.2.2, 5.2.3)
    captured in a CUDA graph.

    ``mode`` is 'depth' or 'alpha'; ``algorithm`` one of SCHEDULES.  With
    ``rle`` the transfers travel RLE-compressed (depth, RGBA8); ``fused`` lets
    binary stages decode inside the composite.  The tensors must stay alive and
    in place while the schedule exists."""

    def __init__(self, mode: str, algorithm: str, images: Sequence[Image], out_color: torch.Tensor,
                 out_depth: Optional[torch.Tensor] = None, out_pvp: Optional[Rect] = None,
                 order=None, rle: bool = True, fused: bool = True, ctx: Optional[Context] = None):
        self.ctx = ctx or default_context(out_color.device.index)
        dev = self.ctx.device
        depth = mode == "depth"
        if not depth and mode != "alpha":
            raise ValueError("mode must be 'depth' or 'alpha'")
        imgs = (ec_image * max(1, len(images)))(*[_image_struct(im, dev, depth) for im in images])
        o = None if depth else _order(order, len(images))
        tgt = _target(out_color, out_depth if depth else None, out_pvp, dev)
        self._keep = [imgs, o, list(images), out_color, out_depth]
        flags = (A.EC_SCHED_RLE if rle else 0) | (A.EC_SCHED_FUSED if fused else 0)
        h = C.c_void_p()
        check(_lib().ec_schedule_plan(self.ctx.h, A.EC_JOB_DEPTH if depth else A.EC_JOB_ALPHA,
                                      SCHEDULES[algorithm], imgs, len(images),
                                      None if o is None else C.cast(o, C.c_void_p), C.byref(tgt), flags,
                                      C.byref(h)), "ec_schedule_plan")
        self.h = h
        self.rle = rle

    def run(self, stream=None):
        check(_lib().ec_schedule_run(self.h, _stream_handle(stream)), "ec_schedule_run")

    def info(self) -> dict:
        lv, nm, nl = C.c_int32(), C.c_int32(), C.c_int32()
        ab = C.c_uint64()
        check(_lib().ec_schedule_info(self.h, C.byref(lv), C.byref(nm), C.byref(nl), C.byref(ab)),
              "ec_schedule_info")
        return {"levels": lv.value, "messages": nm.value, "launches": nl.value, "arena_bytes": ab.value}

    def messages(self):
        """[(level, sender, receiver, fused, (x, y, w, h))] in stage order."""
        n = self.info()["messages"]
        arr = (A.ec_sched_message * max(1, n))()
        check(_lib().ec_schedule_messages(self.h, arr, n), "ec_schedule_messages")
        return [(m.level, m.sender, m.receiver, m.fused, (m.piece.x, m.piece.y, m.piece.w, m.piece.h))
                for m in arr[:n]]

    def launches(self):
        """[(level, kind, pixel bytes)] of the run's kernel launches, in order;
        kind is one of 'rle_compress', 'rle_decompress', 'fused_depth', 'composite'."""
        n = self.info()["launches"]
        arr = (A.ec_sched_launch * max(1, n))()
        check(_lib().ec_schedule_launches(self.h, arr, n), "ec_schedule_launches")
        return [(l.level, A.EC_SCHED_LAUNCH_KINDS[l.kind], int(l.bytes)) for l in arr[:n]]

    def run_launch(self, i: int, stream=None):
        """Enqueue launch i alone (in order, for timing)."""
        check(_lib().ec_schedule_run_launch(self.h, i, _stream_handle(stream)), "ec_schedule_run_launch")

    def stream_sizes(self, stream=None):
        """[(colour bytes, depth bytes)] of every transfer of the last run."""
        n = self.info()["messages"]
        arr = (C.c_uint64 * max(2, 2 * n))()
        check(_lib().ec_schedule_stream_sizes(self.h, arr, 2 * n, _stream_handle(stream)),
              "ec_schedule_stream_sizes")
        return [(int(arr[2 * i]), int(arr[2 * i + 1])) for i in range(n)]

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            _lib().ec_schedule_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
