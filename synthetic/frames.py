"""Seeded generators for partial framebuffers (see the package docstring).

Nothing here composites, blends or encodes: generators draw numbers from seeded
PCG64 streams and paint them into buffers on the requested device.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Tuple

import numpy as np
import torch

ROOT_SEED = 190208755

Rect = Tuple[int, int, int, int]


def rng(*key: int) -> np.random.Generator:
    """PCG64 stream for the key (cfg, source, ...)."""
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([ROOT_SEED, *key])))


def _torch_gen(device, *key: int) -> torch.Generator:
    seed = int(np.random.SeedSequence([ROOT_SEED, *key]).generate_state(1, dtype=np.uint64)[0])
    g = torch.Generator(device=device)
    g.manual_seed(seed & ((1 << 63) - 1))
    return g


@dataclass
class DepthSource:
    """One rendered partial image.  Arrays are [pvp.h][pitch] (pitch == pvp.w)."""
    pvp: Rect
    roi: Rect
    color: torch.Tensor        # uint32 RGBA8 (R in the low byte) or float32 [h][w][4]
    depth: torch.Tensor        # float32
    boxes: list = field(default_factory=list)

    @property
    def pitch(self) -> int:
        return int(self.color.shape[1])


def _pack_rgba8(r: int, g: int, b: int, a: int = 255) -> int:
    return (r | (g << 8) | (b << 16) | (a << 24)) & 0xFFFFFFFF


def _draw_boxes(r: np.random.Generator, W: int, H: int, coverage: float, clustered: bool,
                side: Tuple[float, float], quantize_depth: int, max_boxes: int = 100000):
    """Draw boxes until ``coverage`` of the W x H frame is covered.
    Returns the box list [(x, y, w, h, rgba8, depth)] and the coverage mask."""
    if clustered:
        area = min(1.0, 2.0 * coverage) * W * H
        aspect = math.exp(r.uniform(math.log(0.75), math.log(4.0 / 3.0)))
        sw = int(min(W, max(8, round(math.sqrt(area * aspect)))))
        sh = int(min(H, max(8, round(area / sw))))
        sx = int(r.integers(0, W - sw + 1))
        sy = int(r.integers(0, H - sh + 1))
        region = (sx, sy, sw, sh)
    else:
        region = (0, 0, W, H)
    rx, ry, rw, rh = region
    mask = np.zeros((H, W), dtype=bool)
    covered, target = 0, coverage * W * H
    boxes = []
    while covered < target and len(boxes) < max_boxes:
        bw = int(max(1, min(rw, round(r.uniform(side[0] * rw, side[1] * rw)))))
        bh = int(max(1, min(rh, round(r.uniform(side[0] * rh, side[1] * rh)))))
        bx = rx + int(r.integers(0, rw - bw + 1))
        by = ry + int(r.integers(0, rh - bh + 1))
        rgb = r.integers(0, 256, size=3)
        if quantize_depth:
            d = float(r.integers(0, quantize_depth)) / quantize_depth
        else:
            d = float(np.float32(r.random()))
        boxes.append((bx, by, bw, bh, _pack_rgba8(int(rgb[0]), int(rgb[1]), int(rgb[2])), d))
        sub = mask[by:by + bh, bx:bx + bw]
        covered += int(sub.size - np.count_nonzero(sub))
        sub[...] = True
    return boxes, mask


def _bbox(mask: np.ndarray) -> Rect:
    rows = np.flatnonzero(mask.any(axis=1))
    cols = np.flatnonzero(mask.any(axis=0))
    if rows.size == 0:
        return (0, 0, 0, 0)
    return (int(cols[0]), int(rows[0]), int(cols[-1] - cols[0] + 1), int(rows[-1] - rows[0] + 1))


def _u32_tensor(v: int, device) -> torch.Tensor:
    # uint32 tensors support fill but little arithmetic; paint through int32 bits
    return torch.tensor(np.array([v], dtype=np.uint32).view(np.int32)[0], dtype=torch.int32,
                        device=device)


def depth_source(W: int, H: int, coverage: float, cfg: int, source: int, *,
                 clustered: bool = False, cropped: bool = False,
                 side: Tuple[float, float] = (1 / 16, 1 / 4), quantize_depth: int = 0,
                 color_f32: bool = False, device="cpu", align: int = 4) -> DepthSource:
    """One depth-mode source (RGBA8 or RGBA32F colour + float32 depth)."""
    r = rng(cfg, source)
    boxes, mask = _draw_boxes(r, W, H, coverage, clustered, side, quantize_depth)
    roi = _bbox(mask)
    if cropped and roi[2] > 0:
        x0 = (roi[0] // align) * align
        x1 = min(W if W % align == 0 else ((W + align - 1) // align) * align,
                 ((roi[0] + roi[2] + align - 1) // align) * align)
        pvp = (x0, roi[1], x1 - x0, roi[3])
    elif cropped:
        pvp = (0, 0, 0, 0)
    else:
        pvp = (0, 0, W, H)
    ph, pw = pvp[3], pvp[2]
    depth = torch.ones((ph, pw), dtype=torch.float32, device=device)
    if color_f32:
        color = torch.zeros((ph, pw, 4), dtype=torch.float32, device=device)
    else:
        color = torch.zeros((ph, pw), dtype=torch.int32, device=device)
    for (bx, by, bw, bh, rgba, d) in boxes:
        x0, y0 = max(bx, pvp[0]), max(by, pvp[1])
        x1, y1 = min(bx + bw, pvp[0] + pw), min(by + bh, pvp[1] + ph)
        if x1 <= x0 or y1 <= y0:
            continue
        sl = (slice(y0 - pvp[1], y1 - pvp[1]), slice(x0 - pvp[0], x1 - pvp[0]))
        depth[sl] = d
        if color_f32:
            color[sl] = torch.tensor([(rgba >> (8 * k)) & 255 for k in range(4)],
                                     dtype=torch.float32, device=device) / 255.0
        else:
            color[sl] = _u32_tensor(rgba, device)
    if not color_f32:
        color = color.view(torch.uint32)
    return DepthSource(pvp=pvp, roi=roi, color=color, depth=depth, boxes=boxes)


def depth_sources(cfg: int, n: int, W: int, H: int, coverage: float, **kw) -> List[DepthSource]:
    return [depth_source(W, H, coverage, cfg, i, **kw) for i in range(n)]


def alpha_layers(cfg: int, L: int, W: int, H: int, amax: float, dtype=torch.float32,
                 device="cpu", first: int = 0) -> torch.Tensor:
    """[L][H][W][4] premultiplied RGBA, alpha ~ U[0, amax], colour = alpha * U[0, 1)."""
    out = torch.empty((L, H, W, 4), dtype=dtype, device=device)
    for k in range(L):
        if torch.device(device).type == "cpu":
            r = rng(cfg, 1000 + first + k)
            a = r.random((H, W), dtype=np.float32) * np.float32(amax)
            u = r.random((H, W, 3), dtype=np.float32)
            lay = np.empty((H, W, 4), dtype=np.float32)
            lay[..., :3] = u * a[..., None]
            lay[..., 3] = a
            out[k] = torch.from_numpy(lay).to(dtype)
        else:
            g = _torch_gen(device, cfg, 1000 + first + k)
            a = torch.rand((H, W), generator=g, device=device, dtype=torch.float32) * amax
            u = torch.rand((H, W, 3), generator=g, device=device, dtype=torch.float32)
            out[k, ..., :3] = (u * a[..., None]).to(dtype)
            out[k, ..., 3] = a.to(dtype)
    return out


def grad_weights(cfg: int, W: int, H: int, device="cpu") -> torch.Tensor:
    """Upstream weights w ~ U[-1, 1] of shape [H][W][4] for L = sum(w * out)."""
    if torch.device(device).type == "cpu":
        r = rng(cfg, 999)
        return torch.from_numpy((r.random((H, W, 4), dtype=np.float32) * 2 - 1).astype(np.float32))
    g = _torch_gen(device, cfg, 999)
    return torch.rand((H, W, 4), generator=g, device=device, dtype=torch.float32) * 2 - 1


@dataclass
class Tile:
    """One sub-image of the batched workload: L layers of w x h, full-tile ROI."""
    mode: str                  # "depth" or "alpha"
    w: int
    h: int
    L: int
    color: Optional[torch.Tensor] = None   # depth: uint32 [L][h][w]; alpha: f32 [L][h][w][4]
    depth: Optional[torch.Tensor] = None   # depth: float32 [L][h][w]


def uneven_tiles(cfg: int, n: int, *, min_side: int = 16, max_side: int = 1024,
                 lmin: int = 2, lmax: int = 64, coverage: float = 0.3, amax: float = 0.3,
                 device="cpu", materialize: bool = True) -> List[Tile]:
    """n tiles with w, h log-uniform in [min_side, max_side] and L ~ U{lmin..lmax};
    even tiles are depth mode (RGBA8 + float32), odd tiles alpha mode (FP32)."""
    r = rng(cfg, 0)
    tiles = []
    for t in range(n):
        w = int(round(math.exp(r.uniform(math.log(min_side), math.log(max_side)))))
        h = int(round(math.exp(r.uniform(math.log(min_side), math.log(max_side)))))
        L = int(r.integers(lmin, lmax + 1))
        tiles.append(Tile("depth" if t % 2 == 0 else "alpha", w, h, L))
    if not materialize:
        return tiles
    for t, tile in enumerate(tiles):
        if tile.mode == "depth":
            col = np.zeros((tile.L, tile.h, tile.w), dtype=np.uint32)
            dep = np.ones((tile.L, tile.h, tile.w), dtype=np.float32)
            for k in range(tile.L):
                boxes, _ = _draw_boxes(rng(cfg, 1 + t, k), tile.w, tile.h, coverage, False,
                                       (1 / 8, 1 / 3), 0)
                for (bx, by, bw, bh, rgba, d) in boxes:
                    col[k, by:by + bh, bx:bx + bw] = rgba
                    dep[k, by:by + bh, bx:bx + bw] = d
            tile.color = torch.from_numpy(col.view(np.int32)).to(device).view(torch.uint32)
            tile.depth = torch.from_numpy(dep).to(device)
        else:
            tile.color = alpha_layers(cfg, tile.L, tile.w, tile.h, amax, torch.float32,
                                      device, first=100000 * (t + 1))
    return tiles


def smooth_image(W: int, H: int, cfg: int = 0) -> np.ndarray:
    """Smoothly shaded RGBA8 image (uint32 [H][W]): low-frequency gradients plus a
    few flat regions, the kind of colour content the swizzle preconditioner targets."""
    r = rng(cfg, 77)
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    ph = r.uniform(0, 2 * np.pi, size=3)
    R = 127.5 + 127.5 * np.sin(x / W * 2.1 + ph[0]) * np.cos(y / H * 1.3)
    G = 127.5 + 127.5 * np.sin(y / H * 2.7 + ph[1])
    B = 127.5 + 127.5 * np.cos((x + y) / (W + H) * 3.1 + ph[2])
    rgb = np.stack([R, G, B], axis=-1).astype(np.uint32)
    for _ in range(4):
        bw, bh = int(r.integers(W // 8, W // 3)), int(r.integers(H // 8, H // 3))
        bx, by = int(r.integers(0, W - bw)), int(r.integers(0, H - bh))
        rgb[by:by + bh, bx:bx + bw] = r.integers(0, 256, size=3)
    return (rgb[..., 0] | (rgb[..., 1] << 8) | (rgb[..., 2] << 16) | (255 << 24)).astype(np.uint32)
