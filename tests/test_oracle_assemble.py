"""Pins of the oracle's compound assembly operations (thesis 4.2: sort-first
and tile compounds copy complete pixels into place, pixel compounds interleave
them, subpixel compounds average every pixel's samples).  Decompositions made
with numpy slicing must reassemble to the original frame, and averages match
numpy's mean of the stacked samples."""
import numpy as np
import pytest

import oracle

F32, F16 = 1, 2


def _frame(r, h, w, kind):
    if kind == "rgba8":
        return r.integers(0, 2 ** 32, (h, w), dtype=np.uint64).astype(np.uint32)
    if kind == "f32":
        return r.random((h, w, 4), dtype=np.float32)
    return r.random((h, w, 4)).astype(np.float16)


@pytest.mark.parametrize("kind", ["rgba8", "f32", "f16"])
def test_tiles_partitioning_the_frame_reassemble_it(orc, kind):
    r = np.random.default_rng(31)
    H, W = 37, 53
    frame = _frame(r, H, W, kind)
    xs = sorted(set([0, W] + list(r.integers(1, W, 4))))
    ys = sorted(set([0, H] + list(r.integers(1, H, 3))))
    tiles = []
    for y0, y1 in zip(ys, ys[1:]):
        for x0, x1 in zip(xs, xs[1:]):
            px = int(r.integers(0, 3))                      # stored with a pitch larger than the tile
            t = np.zeros((y1 - y0, x1 - x0 + px) + frame.shape[2:], dtype=frame.dtype)
            t[:, :x1 - x0] = frame[y0:y1, x0:x1]
            rect = (100 + x0, 50 + y0, x1 - x0, y1 - y0)
            tiles.append(orc.Image(rect, rect, np.ascontiguousarray(t)))
    r.shuffle(tiles)                                      # a partition: the order does not matter
    out = orc.assemble_tiles(tiles, np.zeros_like(frame), (100, 50, W, H))
    assert np.array_equal(out.view(np.uint8), frame.view(np.uint8))


def test_tile_order_roi_and_untouched_pixels(orc):
    a = np.full((4, 4), 7, dtype=np.uint32)
    b = np.full((4, 4), 9, dtype=np.uint32)
    out0 = np.full((6, 6), 1, dtype=np.uint32)
    out = orc.assemble_tiles([orc.Image((0, 0, 4, 4), (0, 0, 4, 4), a),
                              orc.Image((2, 2, 4, 4), (3, 2, 3, 2), b)], out0, (0, 0, 6, 6))
    want = out0.copy()
    want[0:4, 0:4] = 7
    want[2:4, 3:6] = 9                                    # later source wins, only inside its roi
    assert np.array_equal(out, want)
    # clipped to out_pvp; pixels outside it are not written
    out = orc.assemble_tiles([orc.Image((-2, -1, 4, 4), (-2, -1, 4, 4), a)], out0, (1, 1, 4, 4))
    want = out0.copy()
    want[0:2, 0:1] = 7
    assert np.array_equal(out, want)


@pytest.mark.parametrize("kind", ["rgba8", "f32", "f16"])
@pytest.mark.parametrize("kernel", [(2, 2), (3, 1), (4, 3), (1, 1)])
def test_pixel_decomposition_reassembles(orc, kind, kernel):
    r = np.random.default_rng(hash(kernel) % 1000)
    nx, ny = kernel
    H, W = 29, 41
    frame = _frame(r, H, W, kind)
    offs, srcs = [], []
    for ky in range(ny):
        for kx in range(nx):
            sub = frame[ky::ny, kx::nx]                  # numpy's strided view of the offset's pixels
            pad = int(r.integers(0, 3))
            s = np.zeros((sub.shape[0], sub.shape[1] + pad) + frame.shape[2:], dtype=frame.dtype)
            s[:, :sub.shape[1]] = sub
            offs.append((kx, ky))
            srcs.append(np.ascontiguousarray(s))
    order = r.permutation(len(srcs))
    out = orc.assemble_pixels([srcs[i] for i in order], [offs[i] for i in order], kernel,
                              np.zeros_like(frame), (5, 7, W, H))
    assert np.array_equal(out.view(np.uint8), frame.view(np.uint8))
    # a missing offset leaves its pixels unchanged
    if len(srcs) > 1:
        out = orc.assemble_pixels(srcs[1:], offs[1:], kernel, np.full_like(frame, 3), (5, 7, W, H))
        got = np.ascontiguousarray(out[0::ny, 0::nx]).view(np.uint8)
        assert np.array_equal(got, np.ascontiguousarray(np.full_like(frame, 3)[0::ny, 0::nx]).view(np.uint8))


def test_average_of_equal_samples_is_the_sample(orc):
    r = np.random.default_rng(3)
    f = _frame(r, 9, 11, "f32")
    imgs = [orc.Image((0, 0, 11, 9), (0, 0, 11, 9), f) for _ in range(7)]
    assert np.array_equal(orc.average(imgs, (0, 0, 11, 9), F32), f.astype(np.float64))
    c = _frame(r, 9, 11, "rgba8")
    imgs = [orc.Image((0, 0, 11, 9), (0, 0, 11, 9), c) for _ in range(5)]
    assert np.array_equal(orc.average(imgs, (0, 0, 11, 9), 0), c)


@pytest.mark.parametrize("kind,fmt", [("f32", F32), ("f16", F16)])
def test_float_average_matches_numpy_mean(orc, kind, fmt):
    r = np.random.default_rng(11)
    samples = [_frame(r, 13, 17, kind) for _ in range(6)]
    imgs = [orc.Image((2, 3, 17, 13), (2, 3, 17, 13), s) for s in samples]
    got = orc.average(imgs, (2, 3, 17, 13), fmt)
    want = np.mean(np.stack([s.astype(np.float64) for s in samples]), axis=0)
    assert np.max(np.abs(got - want)) <= 1e-12


def test_rgba8_average_rounding_and_coverage(orc):
    a = np.array([[0x01020304, 0xFF000000]], dtype=np.uint32)
    b = np.array([[0x02020306, 0xFF000001]], dtype=np.uint32)
    out = orc.average([orc.Image((0, 0, 2, 1), (0, 0, 2, 1), a), orc.Image((0, 0, 2, 1), (0, 0, 1, 1), b)],
                      (0, 0, 3, 1), 0)
    # channel means: (4+6)/2=5, (3+3)/2=3, (2+2)/2=2, (1+2)/2=1.5 -> 2 (half up); pixel 1: only a; pixel 2: none
    assert out.tolist() == [[0x02020305, 0xFF000000, 0]]
    samples = [np.full((1, 1), v, dtype=np.uint32) for v in (1, 1, 2)]
    out = orc.average([orc.Image((0, 0, 1, 1), (0, 0, 1, 1), s) for s in samples], (0, 0, 1, 1), 0)
    assert out[0, 0] == 1                                 # 4/3 = 1.33 rounds down
