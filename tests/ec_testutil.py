"""Helpers shared by the GPU parity tests: hand the same seeded inputs to the
CUDA path (through its C ABI) and to the oracle, and compare."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
import paper_1902_08755_gb300 as ec


def require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")


def np_of(t: torch.Tensor) -> np.ndarray:
    """Host copy of a tensor (uint32 via an int32 view)."""
    if t.dtype == torch.uint32:
        return t.view(torch.int32).cpu().numpy().view(np.uint32)
    return t.cpu().numpy()


def depth_pair(src, device="cuda"):
    """(oracle.Image, ec.Image) for one synthetic DepthSource (same bits)."""
    o = oracle.Image(src.pvp, src.roi, np.ascontiguousarray(np_of(src.color)),
                     np.ascontiguousarray(np_of(src.depth)))
    g = ec.Image(color=src.color.to(device), depth=src.depth.to(device), pvp=src.pvp, roi=src.roi)
    return o, g


def band(img: "oracle.Image", y0: int, y1: int):
    """Crop an oracle image to destination rows [y0, y1): the oracle then computes
    exactly those output rows (every output pixel depends only on its own inputs)."""
    px, py, pw, ph = img.pvp
    a, b = max(y0, py), min(y1, py + ph)
    if b <= a:
        pvp = (px, y0, pw, 0)
        col = img.color[:0]
        dep = None if img.depth is None else img.depth[:0]
    else:
        pvp = (px, a, pw, b - a)
        col = img.color[a - py:b - py]
        dep = None if img.depth is None else img.depth[a - py:b - py]
    rx, ry, rw, rh = img.roi
    ra, rb = max(ry, pvp[1]), min(ry + rh, pvp[1] + pvp[3])
    roi = (rx, ra, rw, rb - ra) if rb > ra and rw > 0 else (pvp[0], pvp[1], 0, 0)
    return oracle.Image(pvp, roi, np.ascontiguousarray(col),
                        None if dep is None else np.ascontiguousarray(dep))


def band_of_source(src, y0: int, y1: int):
    """Oracle image of destination rows [y0, y1) of a (device) DepthSource, copying
    only those rows to the host."""
    px, py, pw, ph = src.pvp
    a, b = max(y0, py), min(y1, py + ph)
    a, b = min(max(a, py), py + ph), max(min(b, py + ph), py)
    b = max(a, b)
    col = np_of(src.color[a - py:b - py])
    dep = np_of(src.depth[a - py:b - py])
    img = oracle.Image((px, a, pw, b - a), (px, a, pw, b - a), col, dep)
    rx, ry, rw, rh = src.roi
    ra, rb = max(ry, a), min(ry + rh, b)
    img.roi = (rx, ra, rw, rb - ra) if rb > ra and rw > 0 else (px, a, 0, 0)
    return img
