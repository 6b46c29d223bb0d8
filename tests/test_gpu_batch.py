"""GPU checks of the batched persistent path (ec_batch_*): many uneven composites
in one graph-captured launch must give, bit for bit, what one ec_composite_depth /
ec_composite_alpha call per job gives (those are oracle-checked elsewhere), for
the autotuned and for explicitly chosen tile shapes, on every graph replay."""
import numpy as np
import pytest
import torch

import oracle
import paper_1902_08755_gb300 as ec
import synthetic as S
from ec_testutil import np_of, require_gpu
from test_gpu_alpha import _random_layers

pytestmark = pytest.mark.gpu


def _jobs_from_tiles(tiles):
    jobs = []
    for t in tiles:
        if t.mode == "depth":
            imgs = [ec.Image(color=t.color[k], depth=t.depth[k]) for k in range(t.L)]
            out = torch.empty((t.h, t.w), dtype=torch.int32, device="cuda").view(torch.uint32)
            dep = torch.empty((t.h, t.w), dtype=torch.float32, device="cuda")
            win = torch.empty((t.h, t.w), dtype=torch.int16, device="cuda")
            jobs.append(ec.Job("depth", imgs, out, out_depth=dep, winner=win))
        else:
            imgs = [ec.Image(color=t.color[k]) for k in range(t.L)]
            out = torch.empty((t.h, t.w, 4), dtype=t.color.dtype, device="cuda")
            tf = torch.empty((t.h, t.w), dtype=torch.float32, device="cuda")
            jobs.append(ec.Job("alpha", imgs, out, t_final=tf))
    return jobs


def _extra_jobs(r):
    """Jobs with cropped inputs, sub-ROIs, orders, FP16 and RGBA32F depth colour."""
    jobs = []
    for i, dtype in enumerate((torch.float16, torch.float32, torch.float16)):
        W, H = int(r.integers(30, 300)), int(r.integers(5, 60))
        n = int(r.integers(1, 20))
        _, g = _random_layers(r, n, W, H, dtype)
        out = torch.empty((H, W, 4), dtype=dtype, device="cuda")
        jobs.append(ec.Job("alpha", g, out, order=list(r.permutation(n)), out_pvp=(1, -1, W, H)))
    imgs = []
    for k in range(5):
        s = S.depth_source(133, 41, 0.5, 77, k, color_f32=True, cropped=bool(k % 2))
        imgs.append(ec.Image(color=s.color.cuda(), depth=s.depth.cuda(), pvp=s.pvp, roi=s.roi))
    out = torch.empty((41, 133, 4), dtype=torch.float32, device="cuda")
    jobs.append(ec.Job("depth", imgs, out, out_depth=torch.empty((41, 133), device="cuda")))
    return jobs


def _single_calls(jobs):
    outs = []
    for jb in jobs:
        c = torch.empty_like(jb.out_color)
        if jb.mode == "depth":
            d = None if jb.out_depth is None else torch.empty_like(jb.out_depth)
            w = None if jb.winner is None else torch.empty_like(jb.winner)
            ec.composite_depth(jb.images, c, d, out_pvp=jb.out_pvp, winner=w)
            outs.append((c, d, w))
        else:
            t = None if jb.t_final is None else torch.empty_like(jb.t_final)
            ec.composite_alpha(jb.images, c, order=jb.order, out_pvp=jb.out_pvp, t_final=t)
            outs.append((c, t))
    ec.default_context().check_status()
    return outs


def _bits(t):
    if t is None:
        return None
    return t.contiguous().view(torch.int16 if t.element_size() == 2 else torch.int32).cpu()


def _assert_same(jobs, ref):
    for jb, r in zip(jobs, ref):
        got = (jb.out_color, jb.out_depth, jb.winner) if jb.mode == "depth" else (jb.out_color, jb.t_final)
        for a, b in zip(got, r):
            if a is not None:
                assert torch.equal(_bits(a), _bits(b))


@pytest.fixture(scope="module")
def workload():
    require_gpu()
    tiles = S.uneven_tiles(40, 48, max_side=200, lmax=12, device="cuda")
    jobs = _jobs_from_tiles(tiles) + _extra_jobs(np.random.default_rng(40))
    ref = _single_calls(jobs)
    return jobs, ref


@pytest.mark.parametrize("cfg", [
    None,
    dict(depth_tile_w=128, depth_tile_h=8, alpha32_tile_w=32, alpha32_tile_h=8, alpha16_tile_w=64, alpha16_tile_h=8),
    dict(depth_tile_w=256, depth_tile_h=4, alpha32_tile_w=128, alpha32_tile_h=16, alpha16_tile_w=128, alpha16_tile_h=4),
    dict(depth_tile_w=128, depth_tile_h=32, alpha32_tile_w=64, alpha32_tile_h=2, alpha16_tile_w=64, alpha16_tile_h=32,
         ctas_per_sm=1),
])
def test_batch_bit_identical_to_single_calls(workload, cfg):
    jobs, ref = workload
    for jb in jobs:                      # poison the destinations
        jb.out_color.view(torch.uint8).fill_(0xA5)
    b = ec.Batch(jobs, config=cfg)
    for _ in range(2):                   # two graph replays
        b.run()
        ec.default_context().check_status()
        _assert_same(jobs, ref)
    c = b.config
    assert c["n_items"] > len(jobs) and c["grid"] > 0
    b.close()


def test_batch_against_oracle_sample(workload):
    jobs, ref = workload
    b = ec.Batch(jobs, config=dict(depth_tile_w=128, depth_tile_h=16, alpha32_tile_w=32, alpha32_tile_h=8,
                                   alpha16_tile_w=64, alpha16_tile_h=8))
    b.run()
    ec.default_context().check_status()
    for jb in jobs[:6]:
        if jb.mode == "depth":
            oimgs = [oracle.Image((0, 0, im.color.shape[1], im.color.shape[0]),
                                  (0, 0, im.color.shape[1], im.color.shape[0]),
                                  np_of(im.color), np_of(im.depth)) for im in jb.images]
            c, d, w, _ = oracle.composite_depth(oimgs, (0, 0, jb.out_color.shape[1], jb.out_color.shape[0]))
            assert np.array_equal(np_of(jb.out_color), c) and np.array_equal(np_of(jb.winner), w)
        else:
            H, W = jb.out_color.shape[:2]
            oimgs = [oracle.Image((0, 0, W, H), (0, 0, W, H), np_of(im.color)) for im in jb.images]
            o, t, _ = oracle.composite_alpha(oimgs, (0, 0, W, H))
            assert np.max(np.abs(np_of(jb.out_color).astype(np.float64) - o)) <= 2e-6
    b.close()


def test_empty_batch_and_bad_config():
    require_gpu()
    b = ec.Batch([], config=dict())
    b.run()
    torch.cuda.synchronize()
    b.close()
    t = S.uneven_tiles(41, 2, max_side=64, lmax=4, device="cuda")
    with pytest.raises(ec.EcError):
        ec.Batch(_jobs_from_tiles(t), config=dict(depth_tile_w=100))     # not a multiple of 128


def test_cfg4_1000_tiles_full_size():
    """The 1000-tile workload the bench times (autotuned plan, one graph launch):
    every output bit-identical to the per-tile calls, and the two largest depth
    and alpha tiles equal to the oracle."""
    require_gpu()
    tiles = S.uneven_tiles(4, 1000, device="cuda")
    jobs = _jobs_from_tiles(tiles)
    ref = _single_calls(jobs)
    for jb in jobs:
        jb.out_color.view(torch.uint8).fill_(0xA5)
    b = ec.Batch(jobs)
    b.run()
    ec.default_context().check_status()
    _assert_same(jobs, ref)
    b.close()
    for mode in ("depth", "alpha"):
        big = sorted((i for i, t in enumerate(tiles) if t.mode == mode),
                     key=lambda i: tiles[i].w * tiles[i].h * tiles[i].L)[-2:]
        for i in big:
            jb, t = jobs[i], tiles[i]
            full = (0, 0, t.w, t.h)
            if mode == "depth":
                oimgs = [oracle.Image(full, full, np_of(im.color), np_of(im.depth)) for im in jb.images]
                c, d, w, _ = oracle.composite_depth(oimgs, full)
                assert np.array_equal(np_of(jb.out_color), c) and np.array_equal(np_of(jb.winner), w)
                assert np.array_equal(np_of(jb.out_depth).view(np.uint32), d.view(np.uint32))
            else:
                oimgs = [oracle.Image(full, full, np_of(im.color)) for im in jb.images]
                o, tf, _ = oracle.composite_alpha(oimgs, full)
                assert np.max(np.abs(np_of(jb.out_color).astype(np.float64) - o)) <= 2e-6
                assert np.max(np.abs(np_of(jb.t_final) - tf)) <= 2e-6
    del jobs, ref, tiles
    torch.cuda.empty_cache()


_CACHE_CHILD = r"""
import sys, torch
sys.path.insert(0, sys.argv[1]); sys.path.insert(0, sys.argv[1] + "/tests")
import paper_1902_08755_gb300 as ec, synthetic as S
from test_gpu_batch import _jobs_from_tiles, _single_calls, _assert_same
jobs = _jobs_from_tiles(S.uneven_tiles(42, 12, max_side=160, lmax=6, device="cuda"))
ref = _single_calls(jobs)
for jb in jobs:
    jb.out_color.view(torch.uint8).fill_(0xA5)
b = ec.Batch(jobs)
b.run()
ec.default_context().check_status()
_assert_same(jobs, ref)
c = b.config
print("CFG", c["depth_tile_w"], c["depth_tile_h"], c["alpha32_tile_w"], c["alpha32_tile_h"])
"""


def _plan_in_child(tmp_path, cache):
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, EC_AUTOTUNE_CACHE=str(cache))
    r = subprocess.run([sys.executable, "-c", _CACHE_CHILD, root], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return [ln for ln in r.stdout.splitlines() if ln.startswith("CFG")][-1]


def test_autotune_cache_file_round_trip(tmp_path):
    """A plan autotuned in one process is stored in EC_AUTOTUNE_CACHE and a second
    process loads it (nothing is appended); an entry whose shape the kernel
    cannot run is ignored, and the batch is autotuned again."""
    require_gpu()
    cache = tmp_path / "tune.txt"
    first = _plan_in_child(tmp_path, cache)
    lines = cache.read_text().splitlines()
    assert len(lines) == 1 and len(lines[0].split()) == 9          # key is one token
    assert _plan_in_child(tmp_path, cache) == first
    assert cache.read_text().splitlines() == lines                  # loaded, not re-tuned
    key = lines[0].split()[0]
    cache.write_text(f"{key} 0 0 0 0 0 0 0 0\n{key} 100 8 32 8 64 8 64 8\n")   # zero sizes; width not /128
    again = _plan_in_child(tmp_path, cache)
    assert again.split()[1] in ("128", "256")
    assert len(cache.read_text().splitlines()) == 3                 # re-tuned and appended
