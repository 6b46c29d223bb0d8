"""Pins for the oracle's lossy YUV compressor (thesis 5.5.3: a colour-space
conversion and chroma subsampling in front of the RLE compressor, which then
codes the Y, U and V channels).

The thesis prints no formulas; the oracle's reading is full-range BT.601
(JFIF) in 8-bit fixed point with 2x2 chroma blocks.  What pins it here, without
repeating its integer arithmetic: the textbook floating-point transform
(luma within 1, block chroma within 1.5 of the mean of the pixels' chroma),
exact round trips of grey, the alpha mean, the bound on the round-trip error
of uniform blocks, the packed layout at odd sizes, and the compression gain
over coding the RGBA pixels.
"""
import numpy as np
import pytest

import synthetic as S


def bt601(img):
    """Floating-point full-range BT.601: Y, Cb, Cr of every pixel."""
    R = (img & 0xFF).astype(np.float64)
    G = ((img >> 8) & 0xFF).astype(np.float64)
    B = ((img >> 16) & 0xFF).astype(np.float64)
    Y = 0.299 * R + 0.587 * G + 0.114 * B
    Cb = 128 - 0.168736 * R - 0.331264 * G + 0.5 * B
    Cr = 128 + 0.5 * R - 0.418688 * G - 0.081312 * B
    return Y, np.clip(Cb, 0, 255), np.clip(Cr, 0, 255)


def unpack(packed, w, h):
    """Per-pixel Y and per-block (U, V, A) from the packed layout."""
    bw, bh = (w + 1) // 2, (h + 1) // 2
    luma, chroma = packed[:bh], packed[bh:]
    Y = np.zeros((h, w), np.int64)
    for k in range(4):
        dx, dy = k & 1, k >> 1
        byte = (luma >> (8 * k)) & 0xFF
        Y[dy::2, dx::2] = byte[:(h - dy + 1) // 2, :(w - dx + 1) // 2]
    return Y, chroma & 0xFF, (chroma >> 8) & 0xFF, (chroma >> 16) & 0xFF


def rgba(r, g, b, a):
    return (np.asarray(r, np.uint32) | (np.asarray(g, np.uint32) << 8) | (np.asarray(b, np.uint32) << 16)
            | (np.asarray(a, np.uint32) << 24))


def rand_img(h, w, seed):
    return np.random.default_rng(seed).integers(0, 2**32, size=(h, w), dtype=np.uint64).astype(np.uint32)


@pytest.mark.parametrize("h,w", [(8, 8), (5, 7), (1, 1), (3, 2), (33, 64)])
def test_luma_and_chroma_follow_the_float_transform(orc, h, w):
    img = rand_img(h, w, h * 100 + w)
    packed = orc.yuv_encode(img)
    assert packed.shape == (2 * ((h + 1) // 2), (w + 1) // 2)
    Y, U, V, A = unpack(packed, w, h)
    fy, fu, fv = bt601(img)
    assert np.abs(Y - fy).max() <= 1.0
    for by in range((h + 1) // 2):
        for bx in range((w + 1) // 2):
            sl = (slice(2 * by, 2 * by + 2), slice(2 * bx, 2 * bx + 2))
            assert abs(U[by, bx] - fu[sl].mean()) <= 1.5
            assert abs(V[by, bx] - fv[sl].mean()) <= 1.5
            a = (img[sl] >> 24).astype(np.int64)
            assert A[by, bx] == (a.sum() + a.size // 2) // a.size        # rounded mean, half up


def test_missing_pixels_of_edge_blocks_are_zero(orc):
    img = np.full((3, 5), rgba(200, 100, 50, 255), np.uint32)
    packed = orc.yuv_encode(img)
    luma = packed[:2]
    assert (luma[1, :] >> 16 == 0).all()          # block row 1 has no second pixel row
    assert luma[0, 2] & 0xFF00FF00 == 0           # block column 2 has no second column


def test_grey_round_trips_exactly(orc):
    r = np.random.default_rng(2)
    h, w = 10, 12
    g = np.repeat(np.repeat(r.integers(0, 256, size=(h // 2, w // 2)), 2, 0), 2, 1)
    a = np.repeat(np.repeat(r.integers(0, 256, size=(h // 2, w // 2)), 2, 0), 2, 1)
    img = rgba(g, g, g, a)
    packed = orc.yuv_encode(img)
    _, U, V, _ = unpack(packed, w, h)
    assert (U == 128).all() and (V == 128).all()
    assert np.array_equal(orc.yuv_decode(packed, w, h), img)


def test_uniform_blocks_round_trip_within_bound(orc):
    """A uniform 2x2 block loses only the rounding of Y, U and V: every channel
    comes back within 3, and the decode equals the float inverse of the stored
    (Y, U, V) within 1."""
    r = np.random.default_rng(3)
    n = 4096
    c = r.integers(0, 256, size=(n, 4))
    img = np.repeat(np.repeat(rgba(c[:, 0], c[:, 1], c[:, 2], c[:, 3]).reshape(64, 64), 2, 0), 2, 1)
    packed = orc.yuv_encode(img)
    out = orc.yuv_decode(packed, 128, 128)
    for ch in range(4):
        d = np.abs(((out >> (8 * ch)) & 0xFF).astype(np.int64) - ((img >> (8 * ch)) & 0xFF).astype(np.int64))
        assert d.max() <= (0 if ch == 3 else 3), ch
    Y, U, V, _ = unpack(packed, 128, 128)
    Uf = np.repeat(np.repeat(U, 2, 0), 2, 1).astype(np.float64) - 128
    Vf = np.repeat(np.repeat(V, 2, 0), 2, 1).astype(np.float64) - 128
    fR = np.clip(Y + 1.402 * Vf, 0, 255)
    fG = np.clip(Y - 0.344136 * Uf - 0.714136 * Vf, 0, 255)
    fB = np.clip(Y + 1.772 * Uf, 0, 255)
    for ch, f in enumerate((fR, fG, fB)):
        assert np.abs(((out >> (8 * ch)) & 0xFF) - f).max() <= 1.0, ch


def test_odd_sizes_and_empty(orc):
    for h, w in ((0, 0), (1, 1), (1, 5), (7, 1), (9, 13)):
        img = rand_img(h, w, 7)
        packed = orc.yuv_encode(img) if h * w else np.zeros((2 * ((h + 1) // 2), (w + 1) // 2), np.uint32)
        out = orc.yuv_decode(packed, w, h)
        assert out.shape == (h, w)


def test_yuv_then_rle_codes_colour_smaller(orc):
    """Thesis 5.5.3: subsampling and per-channel RLE together code colour frames
    smaller than RLE of the RGBA pixels alone: the packed image holds 2 bytes
    per pixel instead of 4 (smooth colour: ~0.73 of the swizzled RGBA coding;
    flat boxes, which RLE already codes well: ~0.93)."""
    for img in (S.smooth_image(256, 192), S.depth_source(400, 300, 0.4, 42, 0).color.numpy()):
        yuv = orc.rle_compress(orc.yuv_encode(img), 1)
        assert len(yuv) < len(orc.rle_compress(img, 2))
