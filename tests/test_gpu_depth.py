"""GPU parity of ec_composite_depth against the oracle: bit-exact colour, depth and
winner on every pixel (thesis 5.2.1 depth-sorted compositing, 5.3 ROI).

Sizes span many 128x4 tiles with ragged right/bottom edges; the full-size
workloads (4 x 640x480, 16 x 1920x1080 cropped) are compared on every pixel,
the 64 x 7680x4320 one on sampled row bands."""
import numpy as np
import pytest
import torch

import oracle
import paper_1902_08755_gb300 as ec
import synthetic as S
from ec_testutil import band_of_source, depth_pair, np_of, require_gpu

pytestmark = pytest.mark.gpu


def _run_gpu(gimgs, W, H, out_pvp=None, pitch=None, fmt=torch.uint32, winner=True):
    pitch = pitch or W
    if fmt == torch.uint32:
        col = torch.full((H, pitch), 0x7F7F7F7F, dtype=torch.int32, device="cuda").view(torch.uint32)
    else:
        col = torch.full((H, pitch, 4), 7.0, dtype=torch.float32, device="cuda")
    dep = torch.full((H, pitch), 7.0, dtype=torch.float32, device="cuda")
    win = torch.full((H, W), 99, dtype=torch.int16, device="cuda") if winner else None
    roi = ec.composite_depth(gimgs, col, dep, out_pvp=out_pvp or (0, 0, W, H), winner=win)
    ec.default_context().check_status()
    return col, dep, win, roi


def _compare(oimgs, gimgs, W, H, out_pvp=None, pitch=None, fmt=torch.uint32):
    col, dep, win, roi = _run_gpu(gimgs, W, H, out_pvp, pitch, fmt)
    ec_, ed, ew, eroi = oracle.composite_depth(oimgs, out_pvp or (0, 0, W, H))
    gc = np_of(col)[:, :W]
    assert np.array_equal(gc.view(np.uint32), np.ascontiguousarray(ec_[:, :W]).view(np.uint32))
    assert np.array_equal(np_of(dep)[:, :W].view(np.uint32), ed[:, :W].view(np.uint32))
    assert np.array_equal(np_of(win), ew)
    assert roi == eroi


def test_cfg1_four_sources_640x480():
    require_gpu()
    pairs = [depth_pair(s) for s in S.depth_sources(1, 4, 640, 480, 0.4)]
    _compare([p[0] for p in pairs], [p[1] for p in pairs], 640, 480)


def test_cfg2_sixteen_cropped_sources_1080p():
    require_gpu()
    pairs = [depth_pair(s) for s in S.depth_sources(2, 16, 1920, 1080, 0.3, clustered=True, cropped=True)]
    assert any(p[0].pvp[0] % 4 == 0 and p[0].pvp[2] < 1920 for p in pairs)
    _compare([p[0] for p in pairs], [p[1] for p in pairs], 1920, 1080)


def _tiny(r, W, H, qlevels=4, nan_p=0.05):
    x0, y0 = int(r.integers(-3, W)), int(r.integers(-3, H))
    pvp = (x0, y0, int(r.integers(1, W + 4)), int(r.integers(1, H + 4)))
    rx = pvp[0] + int(r.integers(0, pvp[2] + 1))
    ry = pvp[1] + int(r.integers(0, pvp[3] + 1))
    roi = (rx, ry, int(r.integers(0, pvp[0] + pvp[2] - rx + 1)), int(r.integers(0, pvp[1] + pvp[3] - ry + 1)))
    pitch = pvp[2] + int(r.integers(0, 9))
    depth = (r.integers(0, qlevels + 1, size=(pvp[3], pitch)) / qlevels).astype(np.float32)
    depth[r.random(depth.shape) < nan_p] = np.nan
    depth[r.random(depth.shape) < 0.02] = -0.0
    color = r.integers(0, 2**32, size=(pvp[3], pitch), dtype=np.uint64).astype(np.uint32)
    o = oracle.Image(pvp, roi, color, depth)
    g = ec.Image(color=torch.from_numpy(color.view(np.int32)).cuda().view(torch.uint32),
                 depth=torch.from_numpy(depth).cuda(), pvp=pvp, roi=roi)
    return o, g


@pytest.mark.parametrize("seed", range(12))
def test_random_ragged_ties_nan_scalar_and_vector_paths(seed):
    require_gpu()
    r = np.random.default_rng(1000 + seed)
    W, H = int(r.integers(1, 300)), int(r.integers(1, 40))
    n = int(r.integers(0, 20)) if seed != 5 else 100     # 100 > 64: large source list
    pairs = [_tiny(r, W, H) for _ in range(n)]
    out_pvp = (int(r.integers(-2, 3)), int(r.integers(-2, 3)), W, H)
    pitch = W + int(r.integers(0, 3)) * 4 if seed % 2 else W + int(r.integers(0, 3))
    _compare([p[0] for p in pairs], [p[1] for p in pairs], W, H, out_pvp=out_pvp, pitch=pitch)


def test_unaligned_pointers_take_scalar_path():
    require_gpu()
    src = S.depth_source(130, 33, 0.5, 9, 0)
    big_c = torch.zeros((33, 133), dtype=torch.int32, device="cuda")
    big_d = torch.ones((33, 133), dtype=torch.float32, device="cuda")
    big_c[:, 1:131] = src.color.view(torch.int32).cuda()
    big_d[:, 1:131] = src.depth.cuda()
    g = ec.Image(color=big_c.view(torch.uint32)[:, 1:], depth=big_d[:, 1:], pvp=src.pvp, roi=src.roi)
    o = oracle.Image(src.pvp, src.roi, np_of(src.color), np_of(src.depth))
    _compare([o, o], [g, g], 130, 33)


def test_no_sources_writes_background():
    require_gpu()
    col, dep, win, roi = _run_gpu([], 45, 17)
    assert np.all(np_of(col) == 0) and np.all(np_of(dep) == 1.0) and np.all(np_of(win) == -1)
    assert roi == (0, 0, 0, 0)


def test_rgba32f_colour_variant():
    require_gpu()
    r = np.random.default_rng(7)
    W, H = 77, 21
    oimgs, gimgs = [], []
    for i in range(5):
        s = S.depth_source(W, H, 0.5, 70, i, color_f32=True, cropped=bool(i % 2))
        oimgs.append(oracle.Image(s.pvp, s.roi, np_of(s.color), np_of(s.depth)))
        gimgs.append(ec.Image(color=s.color.cuda(), depth=s.depth.cuda(), pvp=s.pvp, roi=s.roi))
    _compare(oimgs, gimgs, W, H, fmt=torch.float32)


def test_quantised_depth_ties_across_sources():
    require_gpu()
    srcs = [S.depth_source(257, 63, 0.6, 71, i, quantize_depth=8) for i in range(6)]
    pairs = [depth_pair(s) for s in srcs]
    _compare([p[0] for p in pairs], [p[1] for p in pairs], 257, 63)


def test_invalid_arguments_rejected():
    require_gpu()
    s = S.depth_source(64, 16, 0.4, 72, 0)
    o, g = depth_pair(s)
    col = torch.zeros((16, 64), dtype=torch.int32, device="cuda").view(torch.uint32)
    bad = ec.Image(color=g.color, depth=g.depth, pvp=(0, 0, 64, 16), roi=(60, 0, 8, 4))
    with pytest.raises(ec.EcError) as e:
        ec.composite_depth([bad], col)
    assert e.value.code == 1
    with pytest.raises(ec.EcError):
        ec.composite_depth([ec.Image(color=g.color, depth=g.depth)] * 513, col)


@pytest.mark.slow
def test_cfg5_64_sources_8k_sampled_rows():
    require_gpu()
    W, H = 7680, 4320
    srcs = S.depth_sources(5, 64, W, H, 0.25, clustered=True, cropped=True, device="cuda")
    gimgs = [ec.Image(color=s.color, depth=s.depth, pvp=s.pvp, roi=s.roi) for s in srcs]
    col = torch.empty((H, W), dtype=torch.int32, device="cuda").view(torch.uint32)
    dep = torch.empty((H, W), dtype=torch.float32, device="cuda")
    win = torch.empty((H, W), dtype=torch.int16, device="cuda")
    ec.composite_depth(gimgs, col, dep, winner=win)
    ec.default_context().check_status()
    for y0 in (0, 1111, 2160, 3333, 4312):
        y1 = y0 + 8
        ob = [band_of_source(s, y0, y1) for s in srcs]
        ec_, ed, ew, _ = oracle.composite_depth(ob, (0, y0, W, y1 - y0))
        assert np.array_equal(np_of(col[y0:y1]), ec_)
        assert np.array_equal(np_of(dep[y0:y1]).view(np.uint32), ed.view(np.uint32))
        assert np.array_equal(np_of(win[y0:y1]), ew)
