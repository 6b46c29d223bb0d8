"""GPU parity of the compound assembly operations (thesis 4.2) with the oracle:
tile assembly and pixel-compound interleaving bit for bit, subpixel averages
bit for bit for RGBA8 and within FP32 summation / FP16 rounding error for
float formats; unaligned layouts take the per-pixel path."""
import numpy as np
import pytest
import torch

import oracle
import paper_1902_08755_gb300 as ec
from ec_testutil import np_of, require_gpu

pytestmark = pytest.mark.gpu

KINDS = {"rgba8": (torch.int32, ()), "f32": (torch.float32, (4,)), "f16": (torch.float16, (4,))}


def _host(r, kind, h, w):
    if kind == "rgba8":
        return r.integers(0, 2 ** 32, (h, w), dtype=np.uint64).astype(np.uint32)
    if kind == "f32":
        return r.random((h, w, 4), dtype=np.float32)
    return r.random((h, w, 4)).astype(np.float16)


def _dev(a, pitch=None, offset=0):
    """Device copy of a [h][w](4) array stored with the given pitch and a base
    offset of `offset` pixels (0 keeps 16-byte alignment)."""
    h, w = a.shape[:2]
    pitch = w if pitch is None else pitch
    inner = a.shape[2:]
    if a.dtype == np.uint32:
        flat = torch.zeros((h * pitch + offset + 4) * (int(np.prod(inner)) if inner else 1), dtype=torch.int32, device="cuda")
        t = flat[offset:offset + h * pitch].view(h, pitch)
        t[:, :w].copy_(torch.from_numpy(a.view(np.int32)))
        return t.view(torch.uint32)[:, :w]
    dt = torch.float32 if a.dtype == np.float32 else torch.float16
    flat = torch.zeros((h * pitch + offset + 4) * 4, dtype=dt, device="cuda")
    t = flat[4 * offset:4 * (offset + h * pitch)].view(h, pitch, 4)
    t[:, :w].copy_(torch.from_numpy(a))
    return t[:, :w]


def _bits(t):
    a = np_of(t)
    return np.ascontiguousarray(a).view(np.uint8)


@pytest.mark.parametrize("kind", list(KINDS))
@pytest.mark.parametrize("seed", range(3))
def test_tiles_match_oracle(kind, seed):
    require_gpu()
    r = np.random.default_rng(1200 + seed)
    W, H = int(r.integers(20, 400)), int(r.integers(10, 200))
    out_pvp = (int(r.integers(-50, 50)), int(r.integers(-50, 50)), W, H)
    base = _host(r, kind, H, W)
    imgs_o, imgs_g = [], []
    for i in range(int(r.integers(1, 12))):
        w, h = int(r.integers(1, W + 30)), int(r.integers(1, H + 30))
        pvp = (out_pvp[0] + int(r.integers(-20, W)), out_pvp[1] + int(r.integers(-20, H)), w, h)
        rx, ry = int(r.integers(0, w)), int(r.integers(0, h))
        roi = (pvp[0] + rx, pvp[1] + ry, int(r.integers(0, w - rx + 1)), int(r.integers(0, h - ry + 1)))
        a = _host(r, kind, h, w)
        imgs_o.append(oracle.Image(pvp, roi, a))
        aligned = seed != 2
        t = _dev(a, pitch=w + (0 if aligned else 1), offset=0 if aligned else 1)
        imgs_g.append(ec.Image(color=t, pvp=pvp, roi=roi))
    out = _dev(base)
    ec.assemble_tiles(imgs_g, out, out_pvp=out_pvp)
    ec.default_context().check_status()
    want = oracle.assemble_tiles(imgs_o, base, out_pvp)
    assert np.array_equal(_bits(out), np.ascontiguousarray(want).view(np.uint8))


@pytest.mark.parametrize("case", ["many_sources", "wide_frame"])
def test_tiles_without_tile_masks(case):
    """More than 64 sources, or a frame wider than 128 CTA tiles: the CTAs list
    their sources themselves instead of reading the host's tile masks."""
    require_gpu()
    r = np.random.default_rng(1300 + len(case))
    W, H = (300, 120) if case == "many_sources" else (16500, 9)
    n = 80 if case == "many_sources" else 6
    base = _host(r, "rgba8", H, W)
    imgs_o, imgs_g = [], []
    for i in range(n):
        w, h = int(r.integers(1, min(W, 4000))), int(r.integers(1, H + 5))
        pvp = (int(r.integers(-10, W)), int(r.integers(-5, H)), w, h)
        roi = (pvp[0], pvp[1], w, h)
        a = _host(r, "rgba8", h, w)
        imgs_o.append(oracle.Image(pvp, roi, a))
        imgs_g.append(ec.Image(color=_dev(a), pvp=pvp, roi=roi))
    out = _dev(base)
    ec.assemble_tiles(imgs_g, out, out_pvp=(0, 0, W, H))
    ec.default_context().check_status()
    want = oracle.assemble_tiles(imgs_o, base, (0, 0, W, H))
    assert np.array_equal(_bits(out), np.ascontiguousarray(want).view(np.uint8))


@pytest.mark.parametrize("kind", list(KINDS))
@pytest.mark.parametrize("kernel", [(2, 2), (3, 1), (4, 3), (16, 16)])
def test_pixels_match_oracle(kind, kernel):
    require_gpu()
    r = np.random.default_rng(sum(kernel))
    nx, ny = kernel
    W, H = int(r.integers(17, 300)), int(r.integers(17, 120))
    frame = _host(r, kind, H, W)
    offs, srcs_h, srcs_d = [], [], []
    for ky in range(ny):
        for kx in range(nx):
            if r.random() < 0.15:
                continue                                   # an offset nobody owns stays untouched
            sub = np.ascontiguousarray(frame[ky::ny, kx::nx])
            offs.append((kx, ky))
            srcs_h.append(sub)
            srcs_d.append(_dev(sub, pitch=sub.shape[1] + int(r.integers(0, 3))))
    base = _host(r, kind, H, W)
    out = _dev(base)
    ec.assemble_pixels(srcs_d, offs, kernel, out, out_pvp=(3, 9, W, H))
    ec.default_context().check_status()
    want = oracle.assemble_pixels(srcs_h, offs, kernel, base, (3, 9, W, H))
    assert np.array_equal(_bits(out), np.ascontiguousarray(want).view(np.uint8))


@pytest.mark.parametrize("kind,fmt,tol", [("rgba8", 0, 0.0), ("f32", 1, 2e-6), ("f16", 2, 1e-3)])
@pytest.mark.parametrize("seed", range(3))
def test_average_matches_oracle(kind, fmt, tol, seed):
    require_gpu()
    r = np.random.default_rng(1300 + seed)
    W, H = int(r.integers(10, 300)), int(r.integers(5, 150))
    imgs_o, imgs_g = [], []
    for i in range(int(r.integers(1, 17))):
        full = r.random() < 0.6
        pvp = (0, 0, W, H) if full else (int(r.integers(-10, W)), int(r.integers(-10, H)),
                                          int(r.integers(1, W + 10)), int(r.integers(1, H + 10)))
        a = _host(r, kind, pvp[3], pvp[2])
        imgs_o.append(oracle.Image(pvp, pvp, a))
        imgs_g.append(ec.Image(color=_dev(a, offset=0 if seed else 1), pvp=pvp, roi=pvp))
    dt, inner = KINDS[kind]
    out = torch.full((H, W) + inner, 7, dtype=dt, device="cuda")
    if kind == "rgba8":
        out = out.view(torch.uint32)
    ec.average(imgs_g, out)
    ec.default_context().check_status()
    want = oracle.average(imgs_o, (0, 0, W, H), fmt)
    got = np_of(out)
    if fmt == 0:
        assert np.array_equal(got, want)
    else:
        assert np.max(np.abs(got.astype(np.float64) - want)) <= tol


def test_subpixel_average_full_frame():
    """16 jittered samples of a 1920x1080 RGBA8 frame, as a subpixel compound
    produces them; every row of a sample band against the oracle."""
    require_gpu()
    r = np.random.default_rng(5)
    samples = [_host(r, "rgba8", 1080, 1920) for _ in range(16)]
    out = torch.empty((1080, 1920), dtype=torch.int32, device="cuda").view(torch.uint32)
    ec.average([ec.Image(color=_dev(s)) for s in samples], out)
    got = np_of(out)
    band = [oracle.Image((0, 0, 1920, 16), (0, 0, 1920, 16), np.ascontiguousarray(s[500:516])) for s in samples]
    assert np.array_equal(got[500:516], oracle.average(band, (0, 0, 1920, 16), 0))


def test_bad_arguments():
    require_gpu()
    out = torch.zeros((8, 8), dtype=torch.int32, device="cuda").view(torch.uint32)
    f = torch.zeros((8, 8, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(ec.EcError):
        ec.assemble_tiles([ec.Image(color=f)], out)           # format differs from the output
    with pytest.raises(ec.EcError):
        ec.assemble_pixels([out[:4, :4]], [(2, 0)], (2, 2), out)   # offset outside the kernel
    with pytest.raises(ec.EcError):
        ec.assemble_pixels([out], [(0, 0)], (17, 1), out)     # kernel larger than 16


def test_rgba8_average_of_many_bright_samples():
    """300 samples with channels near 255 (the 16-bit lane sums are folded every
    256 sources) and per-pixel counts from 1 to 300: exact integer rounding."""
    require_gpu()
    r = np.random.default_rng(17)
    W, H = 37, 9
    imgs_o, imgs_g = [], []
    for i in range(300):
        w = int(r.integers(1, W + 1))
        pvp = (0, 0, w, H)                                 # pixel x is held by every sample wider than x
        a = (0xFFFFFFFF - r.integers(0, 0x03030303, (H, w), dtype=np.uint64)).astype(np.uint32)
        imgs_o.append(oracle.Image(pvp, pvp, a))
        imgs_g.append(ec.Image(color=_dev(a), pvp=pvp, roi=pvp))
    out = torch.empty((H, W), dtype=torch.int32, device="cuda").view(torch.uint32)
    ec.average(imgs_g, out)
    ec.default_context().check_status()
    assert np.array_equal(np_of(out), oracle.average(imgs_o, (0, 0, W, H), 0))


def test_asm4k_workload():
    """The 3840x2160 RGBA8 workloads the bench times: a sort-first frame from an
    8 x 8 grid of tiles and a 2 x 2 pixel compound (every pixel, bit for bit),
    and the average of 8 samples (sampled row bands, bit for bit)."""
    require_gpu()
    W, H, nt = 3840, 2160, 8
    r = np.random.default_rng(4321)
    tw, th = -(-W // nt), -(-H // nt)
    base = _host(r, "rgba8", H, W)
    imgs_o, imgs_g = [], []
    for j in range(nt):
        for i in range(nt):
            rect = (i * tw, j * th, min(tw, W - i * tw), min(th, H - j * th))
            a = _host(r, "rgba8", rect[3], rect[2])
            imgs_o.append(oracle.Image(rect, rect, a))
            imgs_g.append(ec.Image(color=_dev(a), pvp=rect, roi=rect))
    out = _dev(base)
    ec.assemble_tiles(imgs_g, out, out_pvp=(0, 0, W, H))
    ec.default_context().check_status()
    assert np.array_equal(np_of(out), oracle.assemble_tiles(imgs_o, base, (0, 0, W, H)))

    frame = _host(r, "rgba8", H, W)
    offs = [(kx, ky) for ky in range(2) for kx in range(2)]
    subs = [np.ascontiguousarray(frame[ky::2, kx::2]) for kx, ky in offs]
    out2 = _dev(base)
    ec.assemble_pixels([_dev(s) for s in subs], offs, (2, 2), out2, out_pvp=(0, 0, W, H))
    ec.default_context().check_status()
    got = np_of(out2)
    assert np.array_equal(got, oracle.assemble_pixels(subs, offs, (2, 2), base, (0, 0, W, H)))
    assert np.array_equal(got, frame)              # the four sources rebuild the frame

    samples = [_host(r, "rgba8", H, W) for _ in range(8)]
    out3 = torch.empty((H, W), dtype=torch.int32, device="cuda").view(torch.uint32)
    ec.average([ec.Image(color=_dev(s)) for s in samples], out3)
    ec.default_context().check_status()
    got = np_of(out3)
    for y0 in (0, 1000, 2144):
        band = [oracle.Image((0, 0, W, 16), (0, 0, W, 16), np.ascontiguousarray(s[y0:y0 + 16])) for s in samples]
        assert np.array_equal(got[y0:y0 + 16], oracle.average(band, (0, 0, W, 16), 0))
