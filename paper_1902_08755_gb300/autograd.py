"""torch.autograd.Function wrappers over the compositing entry points.

The forward and the hand-written backward both run in libec's kernels
(ec_composite_alpha / ec_composite_alpha_backward, ec_composite_depth /
ec_composite_depth_backward); this module only marshals tensors and keeps the
layer metadata (pixel viewport, ROI, order) that the backward needs.
"""
from __future__ import annotations

from typing import Optional, Sequence, Tuple

import torch

from . import api
from .api import Image

Rect = Tuple[int, int, int, int]


def _meta(images: Sequence[Image]):
    out = []
    for im in images:
        fmt, pitch, w, h = api.pixel_layout(im.color)
        pvp = tuple(im.pvp) if im.pvp is not None else (0, 0, w, h)
        roi = tuple(im.roi) if im.roi is not None else pvp
        out.append((pvp, roi, pitch))
    return out


def _grad_buffers(colors, meta, out_pvp, dtype=None):
    """Gradient tensors shaped like the layers.  The kernels write every pixel of
    pvp ∩ out_pvp; anything else (pitch padding, parts of pvp outside the
    output) must read as zero, so those buffers start zeroed."""
    grads = []
    ox, oy, ow, oh = out_pvp
    for c, (pvp, _, pitch) in zip(colors, meta):
        inside = (pvp[0] >= ox and pvp[1] >= oy and pvp[0] + pvp[2] <= ox + ow and
                  pvp[1] + pvp[3] <= oy + oh)
        full = inside and pitch == pvp[2] and c.shape[0] == pvp[3]
        t = torch.empty_like(c, dtype=dtype or c.dtype) if full else torch.zeros_like(c, dtype=dtype or c.dtype)
        grads.append(t)
    return grads


class _AlphaOver(torch.autograd.Function):
    @staticmethod
    def forward(ctx, meta, order, out_pvp, out_shape, *colors):
        imgs = [Image(color=c, pvp=m[0], roi=m[1]) for c, m in zip(colors, meta)]
        out = torch.empty(out_shape, dtype=colors[0].dtype, device=colors[0].device)
        api.composite_alpha(imgs, out, order=order, out_pvp=out_pvp)
        ctx.save_for_backward(*colors)
        ctx.meta, ctx.order, ctx.out_pvp = meta, order, out_pvp
        return out

    @staticmethod
    def backward(ctx, grad_out):
        colors = ctx.saved_tensors
        imgs = [Image(color=c, pvp=m[0], roi=m[1]) for c, m in zip(colors, ctx.meta)]
        W, H = ctx.out_pvp[2], ctx.out_pvp[3]
        g = grad_out[:H, :W].to(torch.float32).contiguous()
        grads = _grad_buffers(colors, ctx.meta, ctx.out_pvp)
        api.composite_alpha_backward(imgs, ctx.out_pvp, g, grads, order=ctx.order)
        return (None, None, None, None, *grads)


def alpha_composite(layers: Sequence[Image], order=None, out_pvp: Optional[Rect] = None,
                    out_shape=None) -> torch.Tensor:
    """Differentiable ordered 'over' (premultiplied, front to back).  Gradients
    flow to every layer's colour tensor (RGB and alpha)."""
    meta = _meta(layers)
    if out_pvp is None:
        fmt, pitch, w, h = api.pixel_layout(layers[0].color)
        out_pvp = (0, 0, w, h)
    out_shape = out_shape or (out_pvp[3], out_pvp[2], 4)
    order = None if order is None else tuple(int(v) for v in order)
    return _AlphaOver.apply(meta, order, tuple(out_pvp), tuple(out_shape), *[im.color for im in layers])


def alpha_composite_fwd_bwd(layers: Sequence[Image], w: torch.Tensor, order=None,
                            out_pvp: Optional[Rect] = None, grad_dtype=None):
    """Forward and the gradient of sum(w * out) in one kernel pass.
    Returns (out, [dL/dlayer])."""
    meta = _meta(layers)
    if out_pvp is None:
        fmt, pitch, wd, h = api.pixel_layout(layers[0].color)
        out_pvp = (0, 0, wd, h)
    out = torch.empty((out_pvp[3], out_pvp[2], 4), dtype=layers[0].color.dtype, device=w.device)
    grads = _grad_buffers([im.color for im in layers], meta, out_pvp, grad_dtype)
    api.composite_alpha_fwd_bwd(layers, out, w.to(torch.float32).contiguous(), grads, order=order,
                                out_pvp=out_pvp)
    return out, grads


class _DepthOver(torch.autograd.Function):
    @staticmethod
    def forward(ctx, meta, out_pvp, depths, *colors):
        imgs = [Image(color=c, depth=d, pvp=m[0], roi=m[1]) for c, d, m in zip(colors, depths, meta)]
        H, W = out_pvp[3], out_pvp[2]
        out = torch.empty((H, W, 4), dtype=torch.float32, device=colors[0].device)
        dep = torch.empty((H, W), dtype=torch.float32, device=colors[0].device)
        win = torch.empty((H, W), dtype=torch.int16, device=colors[0].device)
        api.composite_depth(imgs, out, dep, out_pvp=out_pvp, winner=win)
        ctx.save_for_backward(win, *colors)
        ctx.meta, ctx.out_pvp = meta, out_pvp
        ctx.mark_non_differentiable(dep)
        return out, dep

    @staticmethod
    def backward(ctx, grad_out, grad_depth):
        win, *colors = ctx.saved_tensors
        W, H = ctx.out_pvp[2], ctx.out_pvp[3]
        g = grad_out[:H, :W].to(torch.float32).contiguous()
        grads = _grad_buffers(colors, ctx.meta, ctx.out_pvp)
        imgs = [Image(color=c, pvp=m[0], roi=m[1]) for c, m in zip(colors, ctx.meta)]
        api.composite_depth_backward(win, ctx.out_pvp, g, imgs, grads)
        return (None, None, None, *grads)


def depth_composite(images: Sequence[Image], out_pvp: Optional[Rect] = None):
    """Differentiable depth merge of RGBA32F colours: returns (colour, depth);
    the colour gradient flows to each pixel's winning input only."""
    meta = _meta(images)
    if out_pvp is None:
        fmt, pitch, w, h = api.pixel_layout(images[0].color)
        out_pvp = (0, 0, w, h)
    return _DepthOver.apply(meta, tuple(out_pvp), [im.depth for im in images],
                            *[im.color for im in images])
