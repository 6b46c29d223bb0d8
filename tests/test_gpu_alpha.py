"""GPU parity of ec_composite_alpha against the FP64 oracle (thesis 5.2.1 ordered
compositing): FP32 layers within 2e-6 absolute, FP16-stored layers within 2e-3
absolute (the oracle runs on the decoded FP16 inputs), remaining transmittance
within the same bounds.  Ragged sizes, ROIs, cropped and unaligned layers,
arbitrary orders; the 32 x 2048^2 and 128 x 3840x2160 FP16 workloads on
sampled row bands."""
import numpy as np
import pytest
import torch

import oracle
import paper_1902_08755_gb300 as ec
import synthetic as S
from ec_testutil import np_of, require_gpu

pytestmark = pytest.mark.gpu

TOL = {torch.float32: 2e-6, torch.float16: 2e-3}


def _random_layers(r, n, W, H, dtype, amax=0.3, crop=True, odd=False):
    oimgs, gimgs = [], []
    for i in range(n):
        if crop and i % 3:
            x0 = int(r.integers(-2, W))
            if not odd:
                x0 -= x0 % 2
            pvp = (x0, int(r.integers(-2, H)), int(r.integers(1, W + 3)), int(r.integers(1, H + 3)))
        else:
            pvp = (0, 0, W, H)
        rx = pvp[0] + int(r.integers(0, pvp[2] + 1))
        ry = pvp[1] + int(r.integers(0, pvp[3] + 1))
        roi = (rx, ry, int(r.integers(0, pvp[0] + pvp[2] - rx + 1)),
               int(r.integers(0, pvp[1] + pvp[3] - ry + 1))) if i % 4 == 1 else pvp
        pitch = pvp[2] + (int(r.integers(0, 4)) if odd else 2 * int(r.integers(0, 3)))
        a = r.random((pvp[3], pitch)) * amax
        lay = np.empty((pvp[3], pitch, 4))
        lay[..., :3] = r.random((pvp[3], pitch, 3)) * a[..., None]
        lay[..., 3] = a
        lay = lay.astype(np.float32 if dtype == torch.float32 else np.float16)
        oimgs.append(oracle.Image(pvp, roi, lay))
        gimgs.append(ec.Image(color=torch.from_numpy(lay).cuda(), pvp=pvp, roi=roi))
    return oimgs, gimgs


def _check(oimgs, gimgs, W, H, dtype, order=None, out_pvp=None, pitch=None):
    pitch = pitch or W
    out = torch.full((H, pitch, 4), 9.0, dtype=dtype, device="cuda")
    T = torch.full((H, W), 9.0, dtype=torch.float32, device="cuda")
    roi = ec.composite_alpha(gimgs, out, order=order, out_pvp=out_pvp or (0, 0, W, H), t_final=T)
    ec.default_context().check_status()
    ref, Tref, eroi = oracle.composite_alpha(oimgs, out_pvp or (0, 0, W, H), order=order)
    got = np_of(out)[:, :W].astype(np.float64)
    tol = TOL[dtype]
    assert np.max(np.abs(got - ref), initial=0.0) <= tol
    assert np.max(np.abs(np_of(T).astype(np.float64) - Tref), initial=0.0) <= max(tol, 2e-6)
    assert roi == eroi


@pytest.mark.parametrize("dtype", [torch.float32, torch.float16])
@pytest.mark.parametrize("seed", range(6))
def test_random_ragged_layers(dtype, seed):
    require_gpu()
    r = np.random.default_rng(2000 + seed)
    W, H = int(r.integers(1, 200)), int(r.integers(1, 30))
    n = int(r.integers(0, 24)) if seed != 3 else 130          # > 64 layers: large list
    oimgs, gimgs = _random_layers(r, n, W, H, dtype, amax=0.3 if seed % 2 else 0.9,
                                  odd=seed == 4)
    order = r.permutation(n) if seed % 2 else None
    out_pvp = (int(r.integers(-1, 2)), int(r.integers(-1, 2)), W, H)
    pitch = W + (2 * int(r.integers(0, 3)) if seed != 5 else 1)
    _check(oimgs, gimgs, W, H, dtype, order=order, out_pvp=out_pvp, pitch=pitch)


def test_no_layers_is_transparent():
    require_gpu()
    out = torch.full((5, 9, 4), 3.0, device="cuda")
    T = torch.zeros((5, 9), device="cuda")
    assert ec.composite_alpha([], out, t_final=T) == (0, 0, 0, 0)
    torch.cuda.synchronize()
    assert torch.all(out == 0) and torch.all(T == 1)


def test_unaligned_layer_pointer():
    require_gpu()
    r = np.random.default_rng(5)
    W, H = 50, 7
    o, g = _random_layers(r, 3, W, H, torch.float16, crop=False)
    big = torch.zeros((H, W + 1, 4), dtype=torch.float16, device="cuda")
    big[:, 1:] = g[0].color
    g[0] = ec.Image(color=big[:, 1:], pvp=(0, 0, W, H))
    _check(o, g, W, H, torch.float16)


def test_rejects_bad_order_and_mixed_formats():
    require_gpu()
    r = np.random.default_rng(6)
    o, g = _random_layers(r, 2, 8, 8, torch.float32, crop=False)
    out = torch.empty((8, 8, 4), device="cuda")
    with pytest.raises(ec.EcError):
        ec.composite_alpha(g, out, order=[0, 0])
    o2, g2 = _random_layers(r, 1, 8, 8, torch.float16, crop=False)
    with pytest.raises(ec.EcError):
        ec.composite_alpha([g[0], g2[0]], out)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float16])
def test_cfg3_32_layers_2048_sampled_rows(dtype):
    require_gpu()
    L, W, H = 32, 2048, 2048
    lay = S.alpha_layers(3, L, W, H, 0.3, dtype=dtype, device="cuda")
    gimgs = [ec.Image(color=lay[k]) for k in range(L)]
    out = torch.empty((H, W, 4), dtype=dtype, device="cuda")
    T = torch.empty((H, W), dtype=torch.float32, device="cuda")
    ec.composite_alpha(gimgs, out, t_final=T)
    ec.default_context().check_status()
    for y0 in (0, 777, 2040):
        rows = lay[:, y0:y0 + 8].cpu().numpy()
        oimgs = [oracle.Image((0, y0, W, 8), (0, y0, W, 8), np.ascontiguousarray(rows[k])) for k in range(L)]
        ref, Tref, _ = oracle.composite_alpha(oimgs, (0, y0, W, 8))
        got = np_of(out[y0:y0 + 8]).astype(np.float64)
        assert np.max(np.abs(got - ref)) <= TOL[dtype]
        assert np.max(np.abs(np_of(T[y0:y0 + 8]) - Tref)) <= 2e-6


def test_cfg5_128_fp16_layers_4k_sampled_rows():
    """The 128-layer FP16 workload at 3840x2160 in the launch configuration the
    bench times (every tile covered by every layer, so the range-test-free
    path): sampled row bands, including the last, against the oracle."""
    require_gpu()
    L, W, H = 128, 3840, 2160
    lay = S.alpha_layers(5, L, W, H, 0.1, dtype=torch.float16, device="cuda")
    gimgs = [ec.Image(color=lay[k]) for k in range(L)]
    out = torch.empty((H, W, 4), dtype=torch.float16, device="cuda")
    T = torch.empty((H, W), dtype=torch.float32, device="cuda")
    ec.composite_alpha(gimgs, out, t_final=T)
    ec.default_context().check_status()
    for y0 in (0, 1077, 2152):
        rows = lay[:, y0:y0 + 8].cpu().numpy()
        oimgs = [oracle.Image((0, y0, W, 8), (0, y0, W, 8), np.ascontiguousarray(rows[k])) for k in range(L)]
        ref, Tref, _ = oracle.composite_alpha(oimgs, (0, y0, W, 8))
        got = np_of(out[y0:y0 + 8]).astype(np.float64)
        assert np.max(np.abs(got - ref)) <= TOL[torch.float16]
        assert np.max(np.abs(np_of(T[y0:y0 + 8]) - Tref)) <= 1e-5
    del lay
    torch.cuda.empty_cache()
