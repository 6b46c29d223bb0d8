"""Pins of the oracle's automatic ROI (thesis 5.3: the ROI found by analysing
the frame buffer, with holes detected).  The bounding box and the tile
occupancy are checked against numpy's own reductions of the data mask, and
against the generator's ROI, which it takes from the mask of the boxes it drew
(never from the pixels)."""
import numpy as np
import pytest

import synthetic as S

F_RGBA8, F_RGBA32F, F_RGBA16F = 0, 1, 2


def _np_bbox(mask, pvp):
    ys, xs = np.nonzero(mask)
    if ys.size == 0:
        return (0, 0, 0, 0)
    return (pvp[0] + int(xs.min()), pvp[1] + int(ys.min()), int(xs.max() - xs.min() + 1), int(ys.max() - ys.min() + 1))


def _np_occ(mask, tile):
    h, w = mask.shape
    gh, gw = -(-h // tile), -(-w // tile)
    pad = np.zeros((gh * tile, gw * tile), dtype=bool)
    pad[:h, :w] = mask
    return pad.reshape(gh, tile, gw, tile).any(axis=(1, 3)).astype(np.uint8)


def _random_image(r, fmt, w, h, pitch, p_data):
    """Return (color, depth, mask) with data exactly where mask is set."""
    mask = r.random((h, w)) < p_data
    if fmt == "depth":
        d = np.ones((h, pitch), dtype=np.float32)
        d[:, w:] = r.random((h, pitch - w)).astype(np.float32)       # padding may hold anything
        d[:h, :w][mask] = r.random(int(mask.sum())).astype(np.float32) * np.float32(0.999)
        d[:h, :w][~mask & (r.random((h, w)) < 0.2)] = np.nan          # NaN depth is background
        return None, d, mask
    if fmt == F_RGBA8:
        c = np.zeros((h, pitch), dtype=np.uint32)
        c[:, w:] = r.integers(0, 2 ** 32, (h, pitch - w), dtype=np.uint64).astype(np.uint32)
        v = r.integers(1, 2 ** 32, int(mask.sum()), dtype=np.uint64).astype(np.uint32)
        c[:h, :w][mask] = v
        return c, None, mask
    if fmt == F_RGBA32F:
        c = np.zeros((h, pitch, 4), dtype=np.float32)
        c[:h, :w][~mask & (r.random((h, w)) < 0.3)] = -0.0             # negative zero is no data
        ch = r.integers(0, 4, int(mask.sum()))
        vals = np.zeros((int(mask.sum()), 4), dtype=np.float32)
        vals[np.arange(ch.size), ch] = r.uniform(-1, 1, ch.size).astype(np.float32) + np.float32(2.0)
        c[:h, :w][mask] = vals
        return c, None, mask
    c = np.zeros((h, pitch, 4), dtype=np.uint16)                       # RGBA16F bits
    c[:h, :w][~mask & (r.random((h, w)) < 0.3)] = 0x8000               # -0.0
    ch = r.integers(0, 4, int(mask.sum()))
    vals = np.zeros((int(mask.sum()), 4), dtype=np.uint16)
    vals[np.arange(ch.size), ch] = r.integers(1, 0x7FFF, ch.size).astype(np.uint16) | (r.integers(0, 2, ch.size) << 15).astype(np.uint16)
    c[:h, :w][mask] = vals
    return c, None, mask


@pytest.mark.parametrize("fmt", ["depth", F_RGBA8, F_RGBA32F, F_RGBA16F])
@pytest.mark.parametrize("seed", range(4))
def test_matches_numpy_reductions(orc, fmt, seed):
    r = np.random.default_rng(500 + seed)
    w, h = int(r.integers(1, 90)), int(r.integers(1, 70))
    pitch = w + int(r.integers(0, 5))
    tile = int(r.choice([1, 2, 8, 16, 64]))
    pvp = (int(r.integers(-50, 50)), int(r.integers(-50, 50)), w, h)
    c, d, mask = _random_image(r, fmt, w, h, pitch, float(r.choice([0.0, 0.001, 0.05, 0.5])))
    roi, occ = orc.detect_roi(pvp, pvp, pitch, 0 if fmt == "depth" else fmt, color=c, depth=d, tile=tile)
    assert roi == _np_bbox(mask, pvp)
    assert np.array_equal(occ, _np_occ(mask, tile))


def test_search_region_limits_the_scan(orc):
    r = np.random.default_rng(7)
    w, h, pitch, pvp = 40, 30, 44, (100, 200, 40, 30)
    _, d, mask = _random_image(r, "depth", w, h, pitch, 0.02)   # padding holds depths < 1
    # clipped above (y < 200) and on the right (x >= 140, inside the padding)
    search = (108, 195, 35, 22)
    sub = np.zeros_like(mask)
    sub[0:17, 8:40] = mask[0:17, 8:40]
    roi, occ = orc.detect_roi(pvp, search, pitch, 0, depth=d, tile=8)
    assert roi == _np_bbox(sub, pvp)
    assert np.array_equal(occ, _np_occ(sub, 8))


def test_special_values(orc):
    pvp = (0, 0, 4, 1)
    d = np.array([[1.0, np.nan, 0.9999999, np.inf]], dtype=np.float32)
    assert orc.detect_roi(pvp, pvp, 4, 0, depth=d, tile=4)[0] == (2, 0, 1, 1)
    c = np.array([[0, 0, 1, 0]], dtype=np.uint32)
    assert orc.detect_roi(pvp, pvp, 4, F_RGBA8, color=c, tile=4)[0] == (2, 0, 1, 1)
    f = np.zeros((1, 4, 4), dtype=np.float32)
    f[0, 0] = [-0.0, 0.0, -0.0, 0.0]
    f[0, 3, 3] = np.nan
    assert orc.detect_roi(pvp, pvp, 4, F_RGBA32F, color=f, tile=4)[0] == (3, 0, 1, 1)
    hb = np.zeros((1, 4, 4), dtype=np.uint16)
    hb[0, 0] = [0x8000, 0, 0x8000, 0]
    hb[0, 1, 2] = 0x0001                              # smallest subnormal
    assert orc.detect_roi(pvp, pvp, 4, F_RGBA16F, color=hb, tile=4)[0] == (1, 0, 1, 1)


def test_empty_cases(orc):
    roi, occ = orc.detect_roi((5, 5, 0, 0), (5, 5, 0, 0), 0, 0, depth=np.ones((0, 0), np.float32), tile=8)
    assert roi == (0, 0, 0, 0) and occ.size == 0
    d = np.ones((9, 9), dtype=np.float32)
    roi, occ = orc.detect_roi((0, 0, 9, 9), (0, 0, 9, 9), 9, 0, depth=d, tile=4)
    assert roi == (0, 0, 0, 0) and occ.shape == (3, 3) and not occ.any()
    d[4, 4] = 0.5
    assert orc.detect_roi((0, 0, 9, 9), (0, 0, 0, 0), 9, 0, depth=d, tile=4)[0] == (0, 0, 0, 0)


@pytest.mark.parametrize("cfg,source", [(1, 0), (1, 3), (2, 5), (2, 11)])
def test_generator_roi_is_detected(orc, cfg, source):
    """The generator's ROI is the bbox of the box mask it painted; detection on
    either the depth or the colour buffer must find exactly it."""
    W, H = (640, 480) if cfg == 1 else (1920, 1080)
    s = S.depth_source(W, H, 0.4 if cfg == 1 else 0.3, cfg, source, clustered=cfg == 2)
    d = s.depth.numpy()
    c = s.color.numpy().view(np.uint32)
    pvp = (0, 0, W, H)
    roi_d, occ_d = orc.detect_roi(pvp, pvp, W, 0, depth=d, tile=64)
    roi_c, occ_c = orc.detect_roi(pvp, pvp, W, F_RGBA8, color=c, tile=64)
    assert roi_d == tuple(s.roi) and roi_c == tuple(s.roi)
    assert np.array_equal(occ_d, occ_c) and occ_d.any()
