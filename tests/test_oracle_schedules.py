"""Pins for the schedule oracle (thesis 5.2.2 direct send / binary swap / 2-3
swap, 5.2.3 streaming compositing).

What the thesis and the mathematics fix, independent of how a schedule is
planned:
  * depth compositing is associative and commutative once ties go to the lower
    source index (thesis 3.6, 5.2.1), so every schedule's frame equals the
    single-pass merge of all sources, bit for bit -- scenes here are built
    with many exact depth ties, NaN, depths >= 1 and empty ROIs, so that any
    compositing-order, tie or background mistake shows;
  * the final regions of a parallel schedule partition the frame (each pixel
    owned exactly once), the stream's last resource owns all of it;
  * with every ROI covering the frame, the number of transfers and the pixels
    they carry have closed forms: direct send n(n-1) transfers, binary swap
    n log2 n, the stream n-1; each moves (n-1) frames of pixels in all;
  * direct send with ROIs moves exactly sum_i |roi_i| - |roi_i ∩ band_i| pixels
    (counted here with numpy masks).
"""
import math

import numpy as np
import pytest

import oracle
from oracle import schedules as S

ALGOS = [S.CHAIN, S.DIRECT_SEND, S.BINARY_SWAP, S.TWO_THREE_SWAP]


def _ns(algo):
    return [1, 2, 4, 8, 16] if algo == S.BINARY_SWAP else [1, 2, 3, 4, 5, 6, 7, 9, 13]


def scene(n, W, H, seed, frame_origin=(0, 0), empty_every=0):
    """n depth sources with boxes of quantised depth (ties everywhere), odd
    values (NaN, 1.0, 2.0, -0.0) and pvps/ROIs that overhang the frame."""
    r = np.random.default_rng(seed)
    fx, fy = frame_origin
    srcs = []
    for i in range(n):
        pw, ph = int(r.integers(W // 2, W + 8)), int(r.integers(H // 2, H + 8))
        px, py = fx + int(r.integers(-4, W // 2)), fy + int(r.integers(-4, H // 2))
        pitch = pw + int(r.integers(0, 5))
        color = r.integers(0, 2**32, size=(ph, pitch), dtype=np.uint64).astype(np.uint32)
        depth = r.choice(np.array([0.25, 0.5, 0.75, 1.0, 2.0, -0.0, 0.0, np.nan], np.float32),
                         size=(ph, pitch), p=[.25, .25, .2, .1, .05, .05, .05, .05]).astype(np.float32)
        rx, ry = int(r.integers(0, pw // 2)), int(r.integers(0, ph // 2))
        rw, rh = int(r.integers(1, pw - rx + 1)), int(r.integers(1, ph - ry + 1))
        if empty_every and i % empty_every == empty_every - 1:
            rw = 0
        srcs.append(oracle.Image((px, py, pw, ph), (px + rx, py + ry, rw, rh), color, depth))
    return srcs


def rois_of(srcs):
    return [S.intersect(tuple(s.roi), tuple(s.pvp)) for s in srcs]


@pytest.mark.parametrize("algo", ALGOS)
@pytest.mark.parametrize("compress", [True, False])
def test_schedule_equals_single_pass(algo, compress):
    W, H = 37, 29
    frame = (3, -2, W, H)
    for n in _ns(algo):
        srcs = scene(n, W, H, 1000 * algo + n, frame_origin=frame[:2], empty_every=4)
        pl = S.plan(algo, frame, rois_of(srcs))
        c, d, _ = S.run_depth(pl, srcs, compress=compress)
        ec, ed, _, _ = oracle.composite_depth(srcs, frame)
        assert np.array_equal(c, ec), (S.NAMES[algo], n)
        assert np.array_equal(d.view(np.uint32), ed.view(np.uint32)), (S.NAMES[algo], n)


def test_compositing_order_matters_in_these_scenes():
    """The scenes really constrain order: reversing the sources changes the frame."""
    srcs = scene(6, 37, 29, 5)
    a = oracle.composite_depth(srcs, (0, 0, 37, 29))[0]
    b = oracle.composite_depth(srcs[::-1], (0, 0, 37, 29))[0]
    assert not np.array_equal(a, b)


@pytest.mark.parametrize("algo", ALGOS)
def test_final_regions_partition_the_frame(algo):
    W, H = 40, 33
    for n in _ns(algo):
        pl = S.plan(algo, (0, 0, W, H), [(0, 0, W, H)] * n)
        cover = np.zeros((H, W), np.int32)
        for i, (x, y, w, h) in enumerate(pl.region):
            cover[y:y + h, x:x + w] += 1
            if algo == S.CHAIN:
                assert (w * h == W * H) == (i == n - 1)
        assert (cover == 1).all(), (S.NAMES[algo], n)
        if algo != S.CHAIN:
            areas = sorted(w * h for (_, _, w, h) in pl.region)
            assert areas[-1] - areas[0] <= max(W, H), "balanced to within one row or column"


FULL_FRAME_COUNTS = [(S.CHAIN, lambda n: n - 1),
                     (S.DIRECT_SEND, lambda n: n * (n - 1)),
                     (S.BINARY_SWAP, lambda n: n * int(math.log2(n))),
                     (S.TWO_THREE_SWAP, None)]


@pytest.mark.parametrize("algo,count", FULL_FRAME_COUNTS)
def test_full_frame_transfers(algo, count):
    W, H = 48, 64
    for n in _ns(algo):
        pl = S.plan(algo, (0, 0, W, H), [(0, 0, W, H)] * n)
        msgs = [m for lv in pl.levels for m in lv.messages]
        px = sum(m.piece[2] * m.piece[3] for m in msgs)
        if count is not None:
            assert len(msgs) == count(n), (S.NAMES[algo], n)
        if algo != S.TWO_THREE_SWAP or n & (n - 1) == 0:
            assert px == (n - 1) * W * H, (S.NAMES[algo], n)
        if algo == S.TWO_THREE_SWAP and n & (n - 1) == 0 and n > 1:
            bs = S.plan(S.BINARY_SWAP, (0, 0, W, H), [(0, 0, W, H)] * n)
            assert len(msgs) == sum(len(lv.messages) for lv in bs.levels)
        for m in msgs:
            assert m.sender != m.receiver


def test_two_three_swap_of_three_is_direct_send():
    """A single group of three exchanges bands exactly like direct send among three."""
    rois = [(0, 0, 30, 30)] * 3
    a = S.plan(S.TWO_THREE_SWAP, (0, 0, 30, 30), rois)
    b = S.plan(S.DIRECT_SEND, (0, 0, 30, 30), rois)
    key = lambda pl: sorted((m.sender, m.receiver, m.piece) for lv in pl.levels for m in lv.messages)
    assert key(a) == key(b)


def test_direct_send_moves_only_roi_pixels():
    W, H, n = 50, 41, 7
    r = np.random.default_rng(3)
    rois = []
    for _ in range(n):
        x, y = int(r.integers(-5, W)), int(r.integers(-5, H))
        rois.append((x, y, int(r.integers(0, 30)), int(r.integers(0, 30))))
    pl = S.plan(S.DIRECT_SEND, (0, 0, W, H), rois)
    moved = sum(m.piece[2] * m.piece[3] for m in pl.levels[0].messages)
    expect = 0
    for i, (x, y, w, h) in enumerate(rois):
        mask = np.zeros((H, W), bool)
        mask[max(y, 0):max(y + h, 0), max(x, 0):max(x + w, 0)] = True
        lo, hi = (i * H) // n, ((i + 1) * H) // n
        expect += int(mask.sum()) - int(mask[lo:hi].sum())
    assert moved == expect


def test_binary_swap_rejects_other_counts():
    with pytest.raises(ValueError):
        S.plan(S.BINARY_SWAP, (0, 0, 8, 8), [(0, 0, 8, 8)] * 6)


def test_compressed_transfer_sizes_are_the_codec_sizes():
    """Each recorded stream size is the size of the piece's own RLE coding."""
    srcs = scene(4, 37, 29, 11)
    pl = S.plan(S.CHAIN, (0, 0, 37, 29), rois_of(srcs))
    _, _, sizes = S.run_depth(pl, srcs, compress=True)
    m = pl.levels[0].messages[0]
    x, y, w, h = m.piece
    s = srcs[0]
    c = np.ascontiguousarray(s.color[y - s.pvp[1]:y - s.pvp[1] + h, x - s.pvp[0]:x - s.pvp[0] + w])
    assert sizes[(0, 0, 1)][0] == len(oracle.rle_compress(c, 2))
