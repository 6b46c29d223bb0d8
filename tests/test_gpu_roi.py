"""GPU parity of the automatic ROI (ec_detect_roi, thesis 5.3) with the oracle:
bounding boxes and occupancy grids must be identical, for every pixel kind,
odd sizes, pitches, origins, search regions, tile sizes, unaligned buffers
(element-wise loads), batches spanning several launches, and the full-size
1080p sources of the depth pipeline."""
import numpy as np
import pytest
import torch

import oracle
import paper_1902_08755_gb300 as ec
import synthetic as S
from ec_testutil import require_gpu
from test_oracle_roi import _random_image

pytestmark = pytest.mark.gpu

KINDS = ["depth", 0, 1, 2]


def _to_torch(kind, c, d, w, h, pitch, offset):
    """Device tensors with the given data; offset elements shift the base (unaligned path)."""
    if kind == "depth":
        flat = torch.ones(h * pitch + offset + 4, dtype=torch.float32, device="cuda")
        dd = flat[offset:offset + h * pitch].view(h, pitch)
        dd.copy_(torch.from_numpy(d))
        color = torch.zeros((h, pitch), dtype=torch.int32, device="cuda").view(torch.uint32)
        return ec.Image(color=color[:, :w] if w else color, depth=dd[:, :w] if w else dd), dd
    if kind == 0:
        flat = torch.zeros(h * pitch + offset + 4, dtype=torch.int32, device="cuda")
        cc = flat[offset:offset + h * pitch].view(h, pitch)
        cc.copy_(torch.from_numpy(c.view(np.int32)))
        return ec.Image(color=cc.view(torch.uint32)[:, :w]), cc
    dt = torch.float32 if kind == 1 else torch.float16
    flat = torch.zeros((h * pitch + 4) * 4 + offset, dtype=dt, device="cuda")
    cc = flat[offset:offset + 4 * h * pitch].view(h, pitch, 4)   # offset in channels: 4 / 2 bytes
    src = torch.from_numpy(c) if kind == 1 else torch.from_numpy(c.view(np.int16)).view(torch.float16)
    cc.copy_(src)
    return ec.Image(color=cc[:, :w]), cc


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("seed", range(6))
def test_matches_oracle(kind, seed):
    require_gpu()
    r = np.random.default_rng(900 + seed)
    w, h = int(r.integers(1, 300)), int(r.integers(1, 200))
    pitch = w + int(r.integers(0, 9))
    if seed % 2 == 0:
        pitch = -(-pitch // 4) * 4                     # 16-byte rows for 4-byte pixels
    offset = int(r.integers(1, 3)) if seed == 5 else 0
    tile = [8, 16, 32, 64][seed % 4]
    pvp = (int(r.integers(-300, 300)), int(r.integers(-300, 300)), w, h)
    sx0, sy0 = int(r.integers(0, w)), int(r.integers(0, h))
    search = pvp if seed % 3 else (pvp[0] + sx0, pvp[1] + sy0, int(r.integers(0, w - sx0 + 1)),
                                   int(r.integers(0, h - sy0 + 1)))
    c, d, _ = _random_image(r, kind, w, h, pitch, float(r.choice([0.0, 0.0005, 0.02, 0.4])))
    img, _ = _to_torch(kind, c, d, w, h, pitch, offset)
    img.pvp, img.roi = pvp, search
    rois, grids = ec.detect_roi([img], tile=tile)
    ec.default_context().check_status()
    want_roi, want_occ = oracle.detect_roi(pvp, search, pitch, 0 if kind == "depth" else kind,
                                           color=c, depth=d, tile=tile)
    assert tuple(rois[0].tolist()) == want_roi
    assert np.array_equal(grids[0].cpu().numpy(), want_occ)


def test_batch_across_launches_and_empties():
    require_gpu()
    r = np.random.default_rng(77)
    imgs, want = [], []
    for i in range(300):                                # more images than one launch carries
        kind = KINDS[i % 4]
        w, h = int(r.integers(0, 70)), int(r.integers(0, 70))
        pitch = max(w, 1) + int(r.integers(0, 3))
        c, d, _ = _random_image(r, kind, w, h, pitch, 0.01) if w and h else (None, None, None)
        if w and h:
            img, _ = _to_torch(kind, c, d, w, h, pitch, 0)
        else:
            img = ec.Image(color=torch.zeros((h, max(w, 1)), dtype=torch.int32, device="cuda").view(torch.uint32)[:, :w])
            kind = 0
            c = np.zeros((h, max(w, 1)), dtype=np.uint32)
            pitch = max(w, 1)
        pvp = (int(r.integers(-50, 50)), int(r.integers(-50, 50)), w, h)
        img.pvp, img.roi = pvp, pvp
        imgs.append(img)
        want.append(oracle.detect_roi(pvp, pvp, pitch, 0 if kind == "depth" else kind, color=c, depth=d, tile=16))
    rois, grids = ec.detect_roi(imgs, tile=16)
    ec.default_context().check_status()
    for i, (roi, occ) in enumerate(want):
        assert tuple(rois[i].tolist()) == roi, i
        assert np.array_equal(grids[i].cpu().numpy(), occ), i


def test_full_size_sources_match_generator():
    """16 uncropped 1920x1080 sources: the detected ROI is the generator's ROI
    (the bbox of the boxes it drew), from depth and from colour alike."""
    require_gpu()
    srcs = S.depth_sources(2, 16, 1920, 1080, 0.3, clustered=True, device="cuda")
    imgs_d = [ec.Image(color=s.color, depth=s.depth) for s in srcs]
    imgs_c = [ec.Image(color=s.color) for s in srcs]
    rd, gd = ec.detect_roi(imgs_d, tile=64)
    rc, gc = ec.detect_roi(imgs_c, tile=64)
    for i, s in enumerate(srcs):
        assert tuple(rd[i].tolist()) == tuple(s.roi) and tuple(rc[i].tolist()) == tuple(s.roi)
        assert torch.equal(gd[i], gc[i])
    # occupancy of two sources against the oracle
    for i in (0, 9):
        _, occ = oracle.detect_roi((0, 0, 1920, 1080), (0, 0, 1920, 1080), 1920, 0,
                                   depth=srcs[i].depth.cpu().numpy(), tile=64)
        assert np.array_equal(gd[i].cpu().numpy(), occ)


def test_bad_arguments():
    require_gpu()
    img = ec.Image(color=torch.zeros((8, 8), dtype=torch.int32, device="cuda").view(torch.uint32))
    with pytest.raises(ec.EcError):
        ec.detect_roi([img], tile=12)
    img.roi = (4, 4, 8, 8)                              # not inside pvp
    with pytest.raises(ec.EcError):
        ec.detect_roi([img], tile=8)
    rois, grids = ec.detect_roi([], tile=8)
    assert rois.shape == (0, 4) and grids == []
