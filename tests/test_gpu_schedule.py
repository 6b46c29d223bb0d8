"""GPU parity of the multi-stage compositing schedules (ec_schedule_*, thesis
5.2.2 direct send / binary swap / 2-3 swap, 5.2.3 streaming compositing)
against the oracle.

Depth: the frame is compared bit for bit with the oracle's schedule (itself
pinned to the single-pass merge), the transfers (stage, sender, receiver,
piece) with the oracle planner's, and every RLE stream size with the size of
the oracle's coding of the same piece -- for the fused stages, the unfused
ones and raw (uncompressed) transfers.  Scenes are full of depth ties, NaN and
depths >= 1 so that order, tie and background mistakes show.

Alpha: partials travel raw and are composited with "over" in FP32 (or stored
as FP16 between stages).  The frame is compared with the FP64 oracle within
2e-6 (FP32 layers) or (stages + 1) * 2^-12 + 1e-6 (FP16 layers: every stage
rounds the partial to half once more, at most half an ulp of a value below 1).
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1902_08755_gb300 as ec
import synthetic as SY
from oracle import schedules as OS
from ec_testutil import depth_pair, np_of, require_gpu
from test_oracle_schedules import scene

pytestmark = pytest.mark.gpu

NAME = {OS.CHAIN: "stream", OS.DIRECT_SEND: "direct_send", OS.BINARY_SWAP: "binary_swap",
        OS.TWO_THREE_SWAP: "two_three_swap"}
VARIANTS = {"fused": dict(rle=True, fused=True), "rle": dict(rle=True, fused=False),
            "raw": dict(rle=False, fused=False)}


def _gpu_image(o):
    c = torch.from_numpy(np.ascontiguousarray(o.color).view(np.int32)).cuda().view(torch.uint32)
    d = torch.from_numpy(np.ascontiguousarray(o.depth)).cuda()
    return ec.Image(color=c, depth=d, pvp=o.pvp, roi=o.roi)


def _target(frame, pitch_pad=3):
    H, P = frame[3], frame[2] + pitch_pad
    col = torch.full((H, P), 0x7F7F7F7F, dtype=torch.int32, device="cuda").view(torch.uint32)
    dep = torch.full((H, P), 7.0, dtype=torch.float32, device="cuda")
    return col, dep


def _run_depth(algo, srcs, frame, variant):
    gimgs = [_gpu_image(s) for s in srcs]
    col, dep = _target(frame)
    sch = ec.Schedule("depth", NAME[algo], gimgs, col, dep, out_pvp=frame, **VARIANTS[variant])
    sch.run()
    ec.default_context().check_status()
    torch.cuda.synchronize()
    return sch, np_of(col)[:, :frame[2]].view(np.uint32), np_of(dep)[:, :frame[2]].view(np.uint32)


def _check_depth(algo, srcs, frame, variant):
    pl = OS.plan(algo, frame, [OS.intersect(tuple(s.roi), tuple(s.pvp)) for s in srcs])
    ec_, ed, sizes = OS.run_depth(pl, srcs, compress=True)
    sch, c, d = _run_depth(algo, srcs, frame, variant)
    assert np.array_equal(c, ec_), (NAME[algo], variant, len(srcs))
    assert np.array_equal(d, ed.view(np.uint32)), (NAME[algo], variant, len(srcs))
    msgs = sch.messages()
    omsgs = [(li, m.sender, m.receiver, m.piece) for li, lv in enumerate(pl.levels) for m in lv.messages]
    assert sorted((m[0], m[1], m[2], m[4]) for m in msgs) == sorted(omsgs)
    info = sch.info()
    assert info["levels"] == len(pl.levels) and info["messages"] == len(omsgs)
    if variant != "raw":
        got = {(m[0], m[1], m[2]): s for m, s in zip(msgs, sch.stream_sizes())}
        assert got == sizes
    fused = [m[3] for m in msgs]
    if variant == "fused" and algo in (OS.CHAIN, OS.BINARY_SWAP):
        assert all(fused)
    if variant != "fused":
        assert not any(fused)
    sch.close()


def _ns(algo):
    return [1, 2, 4, 8, 16] if algo == OS.BINARY_SWAP else [1, 2, 3, 5, 6, 7, 12]


@pytest.mark.parametrize("variant", list(VARIANTS))
@pytest.mark.parametrize("algo", [OS.CHAIN, OS.DIRECT_SEND, OS.BINARY_SWAP, OS.TWO_THREE_SWAP])
def test_depth_schedules_match_oracle(algo, variant):
    """Frames of several 4096-element chunks per piece with ragged tails."""
    require_gpu()
    W, H = 301, 170
    frame = (5, -3, W, H)
    for n in _ns(algo):
        srcs = scene(n, W, H, 7000 + 100 * algo + n, frame_origin=frame[:2], empty_every=5)
        _check_depth(algo, srcs, frame, variant)


@pytest.mark.parametrize("algo", [OS.DIRECT_SEND, OS.BINARY_SWAP, OS.TWO_THREE_SWAP])
def test_more_resources_than_rows(algo):
    """Empty bands and halves: some resources end up owning nothing."""
    require_gpu()
    W, H = 41, 5
    n = 8
    srcs = scene(n, W, H, 99 + algo)
    _check_depth(algo, srcs, (0, 0, W, H), "fused")
    _check_depth(algo, srcs, (0, 0, W, H), "rle")


def test_sources_outside_the_frame_and_empty():
    require_gpu()
    W, H = 64, 48
    srcs = scene(4, W, H, 5)
    far = oracle.Image((500, 500, 8, 8), (500, 500, 8, 8), srcs[0].color[:8, :8].copy(),
                       srcs[0].depth[:8, :8].copy())
    empty = oracle.Image((0, 0, 8, 8), (0, 0, 0, 0), srcs[1].color[:8, :8].copy(), srcs[1].depth[:8, :8].copy())
    for algo in (OS.CHAIN, OS.BINARY_SWAP, OS.TWO_THREE_SWAP, OS.DIRECT_SEND):
        _check_depth(algo, [far, srcs[0], empty, srcs[1]], (0, 0, W, H), "fused")


def _cfg2():
    return [depth_pair(s) for s in SY.depth_sources(2, 16, 1920, 1080, 0.3, clustered=True, cropped=True)]


@pytest.mark.parametrize("algo,variant", [(OS.BINARY_SWAP, "fused"), (OS.BINARY_SWAP, "rle"),
                                          (OS.DIRECT_SEND, "rle"), (OS.TWO_THREE_SWAP, "fused"),
                                          (OS.CHAIN, "fused"), (OS.BINARY_SWAP, "raw")])
def test_full_size_sixteen_1080p_sources(algo, variant):
    """The 16 x 1920x1080 cropped workload: the schedule's frame equals the
    oracle's single-pass merge on every pixel, the transfers the planner's."""
    require_gpu()
    pairs = _cfg2()
    frame = (0, 0, 1920, 1080)
    col, dep = _target(frame, 0)
    sch = ec.Schedule("depth", NAME[algo], [p[1] for p in pairs], col, dep, out_pvp=frame, **VARIANTS[variant])
    sch.run()
    ec.default_context().check_status()
    ec_, ed, _, _ = oracle.composite_depth([p[0] for p in pairs], frame)
    assert np.array_equal(np_of(col).view(np.uint32), ec_)
    assert np.array_equal(np_of(dep).view(np.uint32), ed.view(np.uint32))
    pl = OS.plan(algo, frame, [p[0].roi for p in pairs])
    omsgs = sorted((li, m.sender, m.receiver, m.piece) for li, lv in enumerate(pl.levels) for m in lv.messages)
    assert sorted((m[0], m[1], m[2], m[4]) for m in sch.messages()) == omsgs
    # a second run over the same buffers gives the same frame
    col.fill_(0)
    sch.run()
    assert np.array_equal(np_of(col).view(np.uint32), ec_)
    sch.close()


@pytest.mark.parametrize("dtype,algo", [(torch.float32, OS.BINARY_SWAP), (torch.float32, OS.TWO_THREE_SWAP),
                                        (torch.float32, OS.CHAIN), (torch.float16, OS.DIRECT_SEND),
                                        (torch.float16, OS.BINARY_SWAP), (torch.float16, OS.TWO_THREE_SWAP)])
def test_alpha_schedules_match_oracle(dtype, algo):
    require_gpu()
    L, W, H = 8, 257, 190
    lay = SY.alpha_layers(7, L, W, H, 0.6, dtype=dtype)
    r = np.random.default_rng(4)
    rois = []
    for k in range(L):
        x, y = int(r.integers(0, W // 2)), int(r.integers(0, H // 2))
        rois.append((x, y, int(r.integers(1, W - x + 1)), int(r.integers(1, H - y + 1))))
    order = [int(v) for v in r.permutation(L)]
    oimgs = [oracle.Image((0, 0, W, H), rois[k], np.ascontiguousarray(lay[k].numpy())) for k in range(L)]
    gl = lay.cuda()
    gimgs = [ec.Image(color=gl[k], pvp=(0, 0, W, H), roi=rois[k]) for k in range(L)]
    out = torch.full((H, W, 4), 9.0, dtype=dtype, device="cuda")
    sch = ec.Schedule("alpha", NAME[algo], gimgs, out, out_pvp=(0, 0, W, H), order=order, rle=False)
    sch.run()
    ec.default_context().check_status()
    ref, _, _ = oracle.composite_alpha(oimgs, (0, 0, W, H), order=order)
    levels = sch.info()["levels"]
    tol = 2e-6 if dtype == torch.float32 else (levels + 1) * 2.0 ** -12 + 1e-6
    err = np.abs(np_of(out).astype(np.float64) - ref).max()
    assert err <= tol, (err, tol)
    pl = OS.plan(algo, (0, 0, W, H), [OS.intersect(tuple(oimgs[o].roi), tuple(oimgs[o].pvp)) for o in order])
    omsgs = sorted((li, m.sender, m.receiver, m.piece) for li, lv in enumerate(pl.levels) for m in lv.messages)
    assert sorted((m[0], m[1], m[2], m[4]) for m in sch.messages()) == omsgs
    sch.close()


def test_argument_errors():
    require_gpu()
    srcs = [_gpu_image(s) for s in scene(6, 32, 32, 1)]
    col, dep = _target((0, 0, 32, 32))
    with pytest.raises(ec.EcError):
        ec.Schedule("depth", "binary_swap", srcs, col, dep, out_pvp=(0, 0, 32, 32))
    lay = torch.zeros((32, 32, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(ec.EcError):
        ec.Schedule("alpha", "stream", [ec.Image(color=lay)], lay.clone(), rle=True)


def test_alpha_binary_swap_at_full_size():
    """32 FP32 layers of 2048 x 2048 (the alpha workload's size) through binary
    swap: within 2e-6 of the FP64 oracle on every pixel."""
    require_gpu()
    L, W, H = 32, 2048, 2048
    lay = SY.alpha_layers(3, L, W, H, 0.3, dtype=torch.float32, device="cuda")
    out = torch.empty((H, W, 4), dtype=torch.float32, device="cuda")
    sch = ec.Schedule("alpha", "binary_swap", [ec.Image(color=lay[k]) for k in range(L)], out, rle=False)
    sch.run()
    ec.default_context().check_status()
    host = lay.cpu().numpy()
    ref, _, _ = oracle.composite_alpha([oracle.Image((0, 0, W, H), (0, 0, W, H), host[k]) for k in range(L)],
                                       (0, 0, W, H))
    assert np.abs(np_of(out).astype(np.float64) - ref).max() <= 2e-6
    assert sch.info()["levels"] == 5
    sch.close()
