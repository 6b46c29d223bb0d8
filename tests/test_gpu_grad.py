"""GPU parity of the hand-written backward kernels against the FP64 oracle gradient
(itself pinned to exact central differences): alpha gradients within
1e-5 * (|y| + max|y| over that layer), FP16-stored gradients within 2e-3 of the
oracle's after casting; the fused forward+backward gives the separate
backward's gradients bit for bit and an output within the forward's tolerance;
the depth gradient is routed to the winner bit-exactly."""
import numpy as np
import pytest
import torch

import oracle
import paper_1902_08755_gb300 as ec
import synthetic as S
from ec_testutil import np_of, require_gpu
from test_gpu_alpha import _random_layers

pytestmark = pytest.mark.gpu


def _grad_close(got: np.ndarray, ref: np.ndarray, rel=1e-5):
    scale = np.max(np.abs(ref), initial=0.0)
    assert np.all(np.abs(got - ref) <= rel * (np.abs(ref) + scale) + 1e-30), \
        float(np.max(np.abs(got - ref) - rel * (np.abs(ref) + scale)))


def _bwd_case(seed, dtype, n=None, W=None, H=None, gdtype=torch.float32, odd=False):
    r = np.random.default_rng(3000 + seed)
    W = W or int(r.integers(1, 150))
    H = H or int(r.integers(1, 12))
    n = int(r.integers(1, 20)) if n is None else n
    oimgs, gimgs = _random_layers(r, n, W, H, dtype, amax=0.9 if seed % 2 else 0.3, odd=odd)
    order = r.permutation(n) if seed % 3 else None
    out_pvp = (int(r.integers(-1, 2)), int(r.integers(-1, 2)), W, H)
    g = (r.random((H, W, 4)) * 2 - 1).astype(np.float32)
    return oimgs, gimgs, order, out_pvp, g


def _run_bwd(gimgs, order, out_pvp, g, gdtype):
    grads = [torch.full_like(im.color, float("nan"), dtype=gdtype) for im in gimgs]
    ec.composite_alpha_backward(gimgs, out_pvp, torch.from_numpy(g).cuda(), grads, order=order)
    ec.default_context().check_status()
    return grads


def _check_against_oracle(oimgs, grads, order, out_pvp, g, gdtype):
    ref = oracle.composite_alpha_backward(oimgs, out_pvp, g.astype(np.float64), order=order,
                                          fill=np.nan)
    for gi, ri in zip(grads, ref):
        got = np_of(gi).astype(np.float64)
        written = ~np.isnan(ri)
        assert np.array_equal(~np.isnan(got), written)        # same elements written
        if gdtype == torch.float32:
            _grad_close(got[written], ri[written])
        else:
            assert np.max(np.abs(got[written] - ri[written].astype(np.float16)), initial=0) <= 2e-3


@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("dtype", [torch.float32, torch.float16])
def test_alpha_backward_matches_oracle(seed, dtype):
    require_gpu()
    oimgs, gimgs, order, out_pvp, g = _bwd_case(seed, dtype, odd=seed == 7)
    grads = _run_bwd(gimgs, order, out_pvp, g, torch.float32)
    _check_against_oracle(oimgs, grads, order, out_pvp, g, torch.float32)


@pytest.mark.parametrize("seed", range(3))
def test_alpha_backward_fp16_gradients(seed):
    require_gpu()
    oimgs, gimgs, order, out_pvp, g = _bwd_case(seed, torch.float16)
    grads = _run_bwd(gimgs, order, out_pvp, g, torch.float16)
    _check_against_oracle(oimgs, grads, order, out_pvp, g, torch.float16)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float16])
def test_alpha_backward_many_layers_chunked(dtype):
    """More layers than one shared-memory chunk holds (the reverse reloads chunks)."""
    require_gpu()
    oimgs, gimgs, order, out_pvp, g = _bwd_case(11, dtype, n=200, W=70, H=3)
    grads = _run_bwd(gimgs, order, out_pvp, g, torch.float32)
    _check_against_oracle(oimgs, grads, order, out_pvp, g, torch.float32)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float16])
def test_fused_gradients_equal_separate_pass_bitwise(dtype):
    require_gpu()
    oimgs, gimgs, order, out_pvp, g = _bwd_case(5, dtype, n=17, W=133, H=9)
    W, H = out_pvp[2], out_pvp[3]
    out_a = torch.empty((H, W, 4), dtype=dtype, device="cuda")
    t_a = torch.empty((H, W), device="cuda")
    ec.composite_alpha(gimgs, out_a, order=order, out_pvp=out_pvp, t_final=t_a)
    grads_a = _run_bwd(gimgs, order, out_pvp, g, torch.float32)
    out_b = torch.empty_like(out_a)
    t_b = torch.empty_like(t_a)
    grads_b = [torch.full_like(im.color, float("nan"), dtype=torch.float32) for im in gimgs]
    ec.composite_alpha_fwd_bwd(gimgs, out_b, torch.from_numpy(g).cuda(), grads_b, order=order,
                               out_pvp=out_pvp, t_final=t_b)
    ec.default_context().check_status()
    # the fused kernel composes the output from per-segment partials (another
    # rounding order): both outputs are checked against the FP64 oracle
    ref, Tref, _ = oracle.composite_alpha(oimgs, out_pvp, order=order)
    tol = 2e-6 if dtype == torch.float32 else 2e-3
    for o, t in ((out_a, t_a), (out_b, t_b)):
        assert np.max(np.abs(np_of(o).astype(np.float64) - ref)) <= tol
        assert np.max(np.abs(np_of(t) - Tref)) <= 2e-6
    for a, b in zip(grads_a, grads_b):
        assert torch.equal(a.nan_to_num(7.0).view(torch.int32), b.nan_to_num(7.0).view(torch.int32))


def test_autograd_function():
    require_gpu()
    r = np.random.default_rng(9)
    W, H, n = 40, 6, 5
    oimgs, gimgs = _random_layers(r, n, W, H, torch.float32, crop=False)
    leaves = [im.color.clone().requires_grad_(True) for im in gimgs]
    imgs = [ec.Image(color=c, pvp=im.pvp, roi=im.roi) for c, im in zip(leaves, gimgs)]
    out = ec.alpha_composite(imgs, order=[4, 2, 0, 1, 3], out_pvp=(0, 0, W, H))
    w = torch.from_numpy((r.random((H, W, 4)) * 2 - 1).astype(np.float32)).cuda()
    (out * w).sum().backward()
    ref = oracle.composite_alpha_backward(oimgs, (0, 0, W, H), w.cpu().double().numpy(),
                                          order=[4, 2, 0, 1, 3])
    for leaf, rg in zip(leaves, ref):
        _grad_close(leaf.grad.cpu().double().numpy(), rg)
    # the fused entry point gives the same gradients
    out2, grads2 = ec.alpha_composite_fwd_bwd(gimgs, w, order=[4, 2, 0, 1, 3], out_pvp=(0, 0, W, H))
    for leaf, g2 in zip(leaves, grads2):
        assert torch.equal(leaf.grad, g2)


def test_depth_backward_routes_to_winner():
    require_gpu()
    W, H = 131, 37
    oimgs, gimgs, pvps, pitches = [], [], [], []
    for i in range(6):
        s = S.depth_source(W, H, 0.5, 90, i, color_f32=True, cropped=bool(i % 2), quantize_depth=6)
        oimgs.append(oracle.Image(s.pvp, s.roi, np_of(s.color), np_of(s.depth)))
        gimgs.append(ec.Image(color=s.color.cuda(), depth=s.depth.cuda(), pvp=s.pvp, roi=s.roi))
        pvps.append(s.pvp)
        pitches.append(s.pitch)
    out = torch.empty((H, W, 4), device="cuda")
    win = torch.empty((H, W), dtype=torch.int16, device="cuda")
    ec.composite_depth(gimgs, out, winner=win)
    g = torch.randn((H, W, 4), device="cuda")
    grads = [torch.full_like(im.color, float("nan")) for im in gimgs]
    ec.composite_depth_backward(win, (0, 0, W, H), g, gimgs, grads)
    ec.default_context().check_status()
    ref = oracle.composite_depth_backward(np_of(win), (0, 0, W, H), np_of(g), pvps, pitches, fill=np.nan)
    for a, b in zip(grads, ref):
        assert np.array_equal(np_of(a).view(np.uint32), b.view(np.uint32))
    # through autograd
    leaves = [im.color.clone().requires_grad_(True) for im in gimgs]
    col, dep = ec.depth_composite([ec.Image(color=c, depth=im.depth, pvp=im.pvp, roi=im.roi)
                                   for c, im in zip(leaves, gimgs)], out_pvp=(0, 0, W, H))
    (col * g).sum().backward()
    for leaf, b in zip(leaves, ref):
        assert np.array_equal(np.nan_to_num(np_of(leaf.grad)), np.nan_to_num(b, nan=0.0))


@pytest.mark.parametrize("dtype", [torch.float32, torch.float16])
def test_cfg3_backward_2048_sampled_rows(dtype):
    require_gpu()
    L, W, H = 32, 2048, 2048
    lay = S.alpha_layers(3, L, W, H, 0.3, dtype=dtype, device="cuda")
    w = S.grad_weights(3, W, H, device="cuda")
    gimgs = [ec.Image(color=lay[k]) for k in range(L)]
    out = torch.empty((H, W, 4), dtype=dtype, device="cuda")
    grads = [torch.empty_like(lay[k], dtype=torch.float32) for k in range(L)]
    ec.composite_alpha_fwd_bwd(gimgs, out, w, grads)
    ec.default_context().check_status()
    for y0 in (0, 1500):
        rows = lay[:, y0:y0 + 4].cpu().numpy()
        oimgs = [oracle.Image((0, y0, W, 4), (0, y0, W, 4), np.ascontiguousarray(rows[k])) for k in range(L)]
        ref = oracle.composite_alpha_backward(oimgs, (0, y0, W, 4), w[y0:y0 + 4].cpu().double().numpy())
        for k in range(L):
            _grad_close(np_of(grads[k][y0:y0 + 4]).astype(np.float64), ref[k])


def test_cfg5_fused_128_fp16_layers_4k_sampled_rows():
    """The 128-layer FP16 workload at 3840x2160 in the launch configuration the
    bench times: fused forward + backward with FP16 gradients, more layers than
    the two-pixels-per-lane path takes.  Sampled row bands of the output and of
    every layer's gradient against the oracle."""
    require_gpu()
    L, W, H = 128, 3840, 2160
    lay = S.alpha_layers(5, L, W, H, 0.1, dtype=torch.float16, device="cuda")
    w = S.grad_weights(5, W, H, device="cuda")
    gimgs = [ec.Image(color=lay[k]) for k in range(L)]
    out = torch.empty((H, W, 4), dtype=torch.float16, device="cuda")
    grads = [torch.empty_like(lay[k]) for k in range(L)]
    ec.composite_alpha_fwd_bwd(gimgs, out, w, grads)
    ec.default_context().check_status()
    for y0 in (0, 1079, 2156):
        rows = lay[:, y0:y0 + 4].cpu().numpy()
        oimgs = [oracle.Image((0, y0, W, 4), (0, y0, W, 4), np.ascontiguousarray(rows[k])) for k in range(L)]
        fwd, _, _ = oracle.composite_alpha(oimgs, (0, y0, W, 4))
        assert np.max(np.abs(np_of(out[y0:y0 + 4]).astype(np.float64) - fwd)) <= 2e-3
        ref = oracle.composite_alpha_backward(oimgs, (0, y0, W, 4), w[y0:y0 + 4].cpu().double().numpy())
        for k in range(L):
            got = np_of(grads[k][y0:y0 + 4]).astype(np.float64)
            assert np.max(np.abs(got - ref[k].astype(np.float16))) <= 2e-3, k
    del lay, grads
    torch.cuda.empty_cache()


@pytest.mark.parametrize("n,pad,roi,gdtype", [
    (64, 0, None, torch.float16),
    (37, 6, (0, 0, 64, 32), torch.float16),
    (40, 2, None, torch.float32),
    (100, 4, (0, 0, 64, 32), torch.float16),
])
def test_fused_fp16_lean_tiles_every_pixel(n, pad, roi, gdtype):
    """FP16 layers that cover the frame with one pitch: tiles take the lean,
    software-pipelined row pass (the next row's loads in flight behind the
    segment exchange) over several CTA row bands and a ragged last band; layer
    counts that do and do not divide into 8-layer segments, 16 and 32 rows per
    CTA.  With `roi`, layer 5's ROI covers only the top-left tiles, so lean and
    general tiles share the launch.  Output, T_final and every gradient element
    against the oracle."""
    require_gpu()
    r = np.random.default_rng(4100 + n)
    W, H = 96, 40
    oimgs, gimgs = [], []
    for i in range(n):
        a = r.random((H, W + pad)) * 0.2
        lay = np.empty((H, W + pad, 4))
        lay[..., :3] = r.random((H, W + pad, 3)) * a[..., None]
        lay[..., 3] = a
        lay = lay.astype(np.float16)
        pvp = (0, 0, W, H)
        lroi = roi if (roi is not None and i == 5) else pvp
        oimgs.append(oracle.Image(pvp, lroi, lay))
        gimgs.append(ec.Image(color=torch.from_numpy(lay).cuda(), pvp=pvp, roi=lroi))
    w = (r.random((H, W, 4)) * 2 - 1).astype(np.float32)
    out = torch.empty((H, W, 4), dtype=torch.float16, device="cuda")
    T = torch.empty((H, W), dtype=torch.float32, device="cuda")
    grads = [torch.full_like(im.color, float("nan"), dtype=gdtype) for im in gimgs]
    ec.composite_alpha_fwd_bwd(gimgs, out, torch.from_numpy(w).cuda(), grads, t_final=T)
    ec.default_context().check_status()
    fwd, Tref, _ = oracle.composite_alpha(oimgs, (0, 0, W, H))
    assert np.max(np.abs(np_of(out).astype(np.float64) - fwd)) <= 2e-3
    assert np.max(np.abs(np_of(T).astype(np.float64) - Tref)) <= 2e-3
    _check_against_oracle(oimgs, grads, None, (0, 0, W, H), w, gdtype)
