"""Oracle for multi-stage compositing schedules (test infrastructure).

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` and ``bench.py``'s CPU legs,
never by the product package.

Thesis 5.2.2 (direct send and binary swap, with 2-3 swap named as the extension
to any number of sources) and 5.2.3 (streaming sort-last compositing): the
sources' partial images are exchanged between compositing resources in stages;
every stage composites, per pixel and in index order, what its resource holds
with what it receives; the resources end up owning disjoint parts of the frame
(or, for the stream, one resource owns all of it) and those parts are placed
into the destination.  Transfers carry only the sender's ROI within the region
sent (thesis 5.3) and are RLE-compressed (thesis 5.5.1).

The planner works on geometry alone (regions and ROIs), so it is separate from
the executor, which moves pixels with the oracle's own codec and depth merge.

Readings of the thesis taken here (it prints no algorithm for the splits):
  * a "region" is a rectangle of the frame; ``bands(R, k)`` cuts R into k row
    bands, band j holding rows [R.y + floor(j R.h / k), R.y + floor((j+1) R.h / k));
  * stream: stage l (l = 0 .. n-2) sends resource l's whole partial frame to
    resource l+1, which composites it in front of its own image;
  * direct send: one stage; resource i owns band i of the frame and receives
    every other resource's pixels there;
  * binary swap (n a power of two): stage l pairs resource u = a + j with
    v = u + 2^l (a a multiple of 2^(l+1)); both hold the same region R, which is
    halved across its longer side (rows when R.h >= R.w; the first half has
    floor(len/2) rows or columns); u keeps the first half, v the second;
  * 2-3 swap: the current units (initially the single resources) are grouped
    consecutively in pairs, the last group a triple when their number is odd;
    a group's resources are ordered by the first row of the region they hold
    (then by unit order), the frame is cut into that many row bands in that
    order, and each resource receives from every resource of the group the
    part of its new band that the sender holds.  With 2^k resources this is
    binary swap over row bands.
A stage's inputs at a receiver are composited unit by unit in index order;
within a unit the pieces are disjoint.  A partial's ROI is the bounding box of
its pieces' ROIs.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

from . import Image, composite_depth, rle_compress, rle_decompress

Rect = Tuple[int, int, int, int]
EMPTY: Rect = (0, 0, 0, 0)

CHAIN, DIRECT_SEND, BINARY_SWAP, TWO_THREE_SWAP = 0, 1, 2, 3
NAMES = {CHAIN: "chain", DIRECT_SEND: "direct_send", BINARY_SWAP: "binary_swap",
         TWO_THREE_SWAP: "two_three_swap"}


def is_empty(r: Rect) -> bool:
    return r[2] <= 0 or r[3] <= 0


def intersect(a: Rect, b: Rect) -> Rect:
    x0, y0 = max(a[0], b[0]), max(a[1], b[1])
    x1, y1 = min(a[0] + a[2], b[0] + b[2]), min(a[1] + a[3], b[1] + b[3])
    if x1 <= x0 or y1 <= y0:
        return EMPTY
    return (x0, y0, x1 - x0, y1 - y0)


def bbox(rects: Sequence[Rect]) -> Rect:
    rs = [r for r in rects if not is_empty(r)]
    if not rs:
        return EMPTY
    x0, y0 = min(r[0] for r in rs), min(r[1] for r in rs)
    x1, y1 = max(r[0] + r[2] for r in rs), max(r[1] + r[3] for r in rs)
    return (x0, y0, x1 - x0, y1 - y0)


def bands(R: Rect, k: int) -> List[Rect]:
    """Row bands of R, band j = rows [y + floor(j h / k), y + floor((j+1) h / k))."""
    x, y, w, h = R
    out = []
    for j in range(k):
        a, b = y + (j * h) // k, y + ((j + 1) * h) // k
        out.append((x, a, w, b - a))
    return out


def halves(R: Rect) -> Tuple[Rect, Rect]:
    """Split R across its longer side (rows when h >= w); the first part is floor(len/2)."""
    x, y, w, h = R
    if h >= w:
        m = h // 2
        return (x, y, w, m), (x, y + m, w, h - m)
    m = w // 2
    return (x, y, m, h), (x + m, y, w - m, h)


@dataclass
class Message:
    level: int
    sender: int
    receiver: int
    piece: Rect           # frame coordinates, inside the sender's ROI and the receiver's new region


@dataclass
class Stage:
    """One receiver's composite in one level: pieces in compositing order."""
    receiver: int
    region: Rect                        # the receiver's new region
    units: List[List[int]]              # senders grouped by unit, units in index order
    pieces: List[Tuple[int, Rect]]      # (sender, piece) in compositing order
    roi: Rect                           # bounding box of the pieces (the partial's ROI)


@dataclass
class Level:
    stages: List[Stage] = field(default_factory=list)
    messages: List[Message] = field(default_factory=list)   # sender != receiver only


@dataclass
class Plan:
    algorithm: int
    n: int
    frame: Rect
    levels: List[Level]
    region: List[Rect]          # final region of every resource
    roi: List[Rect]             # final ROI of every resource


def _level(levels: List[Level], units_of: List[List[List[int]]], new_region: Dict[int, Rect],
           region: List[Rect], roi: List[Rect]):
    """Build one level from groups of units and the receivers' new regions;
    update region/roi in place.  units_of: one entry per group, a list of units."""
    lv = Level()
    li = len(levels)
    new_roi = {}
    for group in units_of:
        members = [m for u in group for m in u]
        for r in members:
            R = new_region[r]
            pieces = []
            for u in group:
                for m in u:
                    p = intersect(intersect(region[m], R), roi[m])
                    if is_empty(p):
                        continue
                    pieces.append((m, p))
                    if m != r:
                        lv.messages.append(Message(li, m, r, p))
            st = Stage(r, R, [list(u) for u in group], pieces, bbox([p for _, p in pieces]))
            lv.stages.append(st)
            new_roi[r] = st.roi
    for r, R in new_region.items():
        region[r] = R
        roi[r] = new_roi.get(r, EMPTY)
    levels.append(lv)


def plan(algorithm: int, frame: Rect, rois: Sequence[Rect]) -> Plan:
    """Plan a schedule for len(rois) resources whose images hold data inside
    rois[i] (frame coordinates; clipped to the frame here)."""
    n = len(rois)
    frame = tuple(int(v) for v in frame)
    if n < 1:
        raise ValueError("at least one resource")
    region = [frame] * n
    roi = [intersect(tuple(int(v) for v in r), frame) for r in rois]
    levels: List[Level] = []
    if algorithm == CHAIN:
        for l in range(n - 1):
            _level(levels, [[[l], [l + 1]]], {l: EMPTY, l + 1: frame}, region, roi)
    elif algorithm == DIRECT_SEND:
        if n > 1:
            b = bands(frame, n)
            _level(levels, [[[i] for i in range(n)]], {i: b[i] for i in range(n)}, region, roi)
    elif algorithm == BINARY_SWAP:
        if n & (n - 1):
            raise ValueError("binary swap needs a power-of-two number of resources")
        s = 1
        while s < n:
            groups, nr = [], {}
            for a in range(0, n, 2 * s):
                groups.append([list(range(a, a + s)), list(range(a + s, a + 2 * s))])
                for j in range(s):
                    u, v = a + j, a + s + j
                    assert region[u] == region[v]
                    nr[u], nr[v] = halves(region[u])
            _level(levels, groups, nr, region, roi)
            s *= 2
    elif algorithm == TWO_THREE_SWAP:
        units = [[i] for i in range(n)]
        while len(units) > 1:
            k = len(units)
            sizes = [2] * (k // 2)
            if k % 2:
                sizes[-1] = 3
            groups, nr, merged, at = [], {}, [], 0
            for sz in sizes:
                g = units[at:at + sz]
                at += sz
                order = sorted(((region[m][1], ui, pos, m) for ui, u in enumerate(g)
                                for pos, m in enumerate(u)))
                members = [t[3] for t in order]
                for m, B in zip(members, bands(frame, len(members))):
                    nr[m] = B
                groups.append(g)
                merged.append(sorted(members))
            _level(levels, groups, nr, region, roi)
            units = merged
    else:
        raise ValueError("unknown algorithm")
    return Plan(algorithm, n, frame, levels, list(region), list(roi))


# ------------------------------------------------------------------ executor

@dataclass
class _Partial:
    roi: Rect
    color: np.ndarray     # [h][w] uint32 over roi
    depth: np.ndarray     # [h][w] float32


def _slice(p: _Partial, r: Rect):
    ox, oy = r[0] - p.roi[0], r[1] - p.roi[1]
    return (np.ascontiguousarray(p.color[oy:oy + r[3], ox:ox + r[2]]),
            np.ascontiguousarray(p.depth[oy:oy + r[3], ox:ox + r[2]]))


def run_depth(pl: Plan, sources: Sequence[Image], compress: bool = True, map=map):
    """Execute a depth-compositing schedule (RGBA8 colour + float32 depth).

    Returns (color [H][W] uint32, depth [H][W] float32, sizes) where sizes maps
    (level, sender, receiver) -> (colour stream bytes, depth stream bytes) of
    every transfer when ``compress`` (else raw bytes, 4 per pixel and stream).
    ``map`` runs the stages of one level (they are independent); a thread
    pool's map spreads them over host cores."""
    if len(sources) != pl.n:
        raise ValueError("one source per resource")
    parts: List[Optional[_Partial]] = []
    for i, s in enumerate(sources):
        r = intersect(intersect(tuple(s.roi), tuple(s.pvp)), pl.frame)
        if is_empty(r):
            parts.append(None)
            continue
        ox, oy = r[0] - s.pvp[0], r[1] - s.pvp[1]
        parts.append(_Partial(r, np.ascontiguousarray(s.color[oy:oy + r[3], ox:ox + r[2]]),
                              np.ascontiguousarray(s.depth[oy:oy + r[3], ox:ox + r[2]])))
        assert parts[-1].color.dtype == np.uint32 and parts[-1].depth.dtype == np.float32
    sizes: Dict[Tuple[int, int, int], Tuple[int, int]] = {}

    def stage(li, st):
        imgs, sz = [], {}
        for m, p in st.pieces:
            c, d = _slice(parts[m], p)
            if m != st.receiver:
                if compress:
                    cs = rle_compress(c, 2)
                    ds = rle_compress(d.view(np.uint32), 1)
                    sz[(li, m, st.receiver)] = (len(cs), len(ds))
                    c = rle_decompress(cs, p[2], p[3])
                    d = rle_decompress(ds, p[2], p[3]).view(np.float32)
                else:
                    sz[(li, m, st.receiver)] = (4 * p[2] * p[3], 4 * p[2] * p[3])
            imgs.append(Image(p, p, c, d))
        if is_empty(st.roi):
            return st.receiver, None, sz
        color, depth, _, _ = composite_depth(imgs, st.roi)
        return st.receiver, _Partial(st.roi, color, depth), sz

    for li, lv in enumerate(pl.levels):
        done = list(map(lambda st: stage(li, st), lv.stages))
        for r, v, sz in done:
            parts[r] = v
            sizes.update(sz)
    fx, fy, W, H = pl.frame
    color = np.zeros((H, W), np.uint32)
    depth = np.ones((H, W), np.float32)
    for i in range(pl.n):
        if is_empty(pl.region[i]) or parts[i] is None or is_empty(pl.roi[i]):
            continue
        if pl.levels:   # the final partials are clean: place them
            r = pl.roi[i]
            color[r[1] - fy:r[1] - fy + r[3], r[0] - fx:r[0] - fx + r[2]] = parts[i].color
            depth[r[1] - fy:r[1] - fy + r[3], r[0] - fx:r[0] - fx + r[2]] = parts[i].depth
    if not pl.levels:   # one resource: its image against the background
        c, d, _, _ = composite_depth(list(sources), pl.frame)
        color, depth = c, d
    return color, depth, sizes
