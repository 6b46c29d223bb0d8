"""Pins for the ordered-compositing oracle (thesis 5.2.1 spatial sort-last compositing:
partial images blended in order, correct transparency) and its gradient.

Independent checks: closed forms for equal alpha, occlusion by an opaque front
layer, the back-to-front form of 'over' (a different recurrence that must agree
by associativity), tree == sequential, FP16 decoding against numpy's own
half-precision conversion, and exact central differences for the gradient
(L is affine in every single input, so a finite difference with dyadic inputs
and a dyadic step has no truncation error).
"""
import numpy as np
import pytest


def _layers(orc, arrs, rois=None, pvps=None):
    out = []
    for i, a in enumerate(arrs):
        H, P = a.shape[:2]
        pvp = pvps[i] if pvps else (0, 0, P, H)
        roi = rois[i] if rois else pvp
        out.append(orc.Image(pvp, roi, np.ascontiguousarray(a)))
    return out


def _rand_layers(r, n, H, W, amax=0.3, dtype=np.float32, dyadic=False):
    a = r.random((n, H, W)) * amax
    u = r.random((n, H, W, 3))
    lay = np.empty((n, H, W, 4))
    lay[..., :3] = u * a[..., None]
    lay[..., 3] = a
    if dyadic:
        lay = np.round(lay * 4096) / 4096
    return lay.astype(dtype)


@pytest.mark.parametrize("n,a", [(1, 0.25), (3, 0.1), (8, 0.3), (32, 0.125)])
def test_equal_alpha_closed_form(orc, n, a):
    H, W, k = 3, 4, 0.5
    lay = np.zeros((n, H, W, 4), np.float32)
    lay[..., :3] = np.float32(a * k)
    lay[..., 3] = np.float32(a)
    out, T, _ = orc.composite_alpha(_layers(orc, lay), (0, 0, W, H))
    af = float(np.float32(a))
    cf = float(np.float32(a * k))
    assert np.allclose(out[..., 3], 1 - (1 - af) ** n, atol=1e-14, rtol=0)
    assert np.allclose(T, (1 - af) ** n, atol=1e-14, rtol=0)
    assert np.allclose(out[..., 0], cf / af * (1 - (1 - af) ** n), atol=1e-14, rtol=0)


def test_opaque_front_hides_everything(orc):
    r = np.random.default_rng(1)
    lay = _rand_layers(r, 5, 4, 6)
    lay[0, ..., 3] = 1.0
    out, T, _ = orc.composite_alpha(_layers(orc, lay), (0, 0, 6, 4))
    assert np.array_equal(out, lay[0].astype(np.float64))
    assert np.all(T == 0.0)


def test_single_layer_is_copy(orc):
    r = np.random.default_rng(2)
    lay = _rand_layers(r, 1, 5, 3)
    out, T, _ = orc.composite_alpha(_layers(orc, lay), (0, 0, 3, 5))
    assert np.array_equal(out, lay[0].astype(np.float64))
    assert np.array_equal(T, 1.0 - lay[0, ..., 3].astype(np.float64))


@pytest.mark.parametrize("seed", range(5))
def test_back_to_front_form_agrees(orc, seed):
    """'over' evaluated from the back, C <- c_k + (1 - a_k) C, is a different
    recurrence; by associativity it must give the front-to-back result."""
    r = np.random.default_rng(10 + seed)
    n, H, W = 7, 3, 5
    lay = _rand_layers(r, n, H, W, amax=0.9)
    order = r.permutation(n)
    out, T, _ = orc.composite_alpha(_layers(orc, lay), (0, 0, W, H), order=order)
    C = np.zeros((H, W, 4))
    for k in reversed(range(n)):
        c = lay[order[k]].astype(np.float64)
        C = c + (1.0 - c[..., 3:4]) * C
    assert np.allclose(out, C, atol=1e-14, rtol=0)
    assert np.allclose(T, np.prod(1.0 - lay[order, ..., 3].astype(np.float64), axis=0),
                       atol=1e-15, rtol=0)


def test_tree_equals_sequential(orc):
    """Composite two halves on their own, then the two partial results: the
    premultiplied 'over' is associative (binary-tree compositing, thesis 5.2.2)."""
    r = np.random.default_rng(3)
    n, H, W = 6, 4, 4
    lay = _rand_layers(r, n, H, W, amax=0.5, dtype=np.float32)
    seq, _, _ = orc.composite_alpha(_layers(orc, lay), (0, 0, W, H))
    front, _, _ = orc.composite_alpha(_layers(orc, lay[:3]), (0, 0, W, H))
    back, _, _ = orc.composite_alpha(_layers(orc, lay[3:]), (0, 0, W, H))
    # feed the partials back in as FP32 layers: agreement is limited by that rounding
    tree, _, _ = orc.composite_alpha(
        _layers(orc, np.stack([front, back]).astype(np.float32)), (0, 0, W, H))
    assert np.allclose(tree, seq, atol=2e-7, rtol=0)


def test_order_matters(orc):
    r = np.random.default_rng(4)
    lay = _rand_layers(r, 2, 2, 2, amax=0.8)
    a, _, _ = orc.composite_alpha(_layers(orc, lay), (0, 0, 2, 2), order=[0, 1])
    b, _, _ = orc.composite_alpha(_layers(orc, lay), (0, 0, 2, 2), order=[1, 0])
    assert not np.allclose(a, b)
    c, _, _ = orc.composite_alpha(_layers(orc, lay[::-1].copy()), (0, 0, 2, 2))
    assert np.array_equal(b, c)


def test_fp16_layers_decoded_exactly(orc):
    r = np.random.default_rng(5)
    lay = _rand_layers(r, 1, 3, 4, dtype=np.float16)
    lay[0, 0, 0] = np.array([6.1e-5, 3e-8, 65504, -0.0], np.float16)  # normal/subnormal/max/-0
    out, _, _ = orc.composite_alpha(_layers(orc, lay), (0, 0, 4, 3))
    assert np.array_equal(out, lay[0].astype(np.float64))


def test_roi_outside_is_transparent(orc):
    r = np.random.default_rng(6)
    lay = _rand_layers(r, 3, 6, 8, amax=0.6)
    rois = [(0, 0, 8, 6), (2, 1, 3, 4), (4, 0, 0, 0)]
    out, T, roi = orc.composite_alpha(_layers(orc, lay, rois=rois), (0, 0, 8, 6))
    masked = lay.copy()
    masked[1] = 0
    masked[1, 1:5, 2:5] = lay[1, 1:5, 2:5]
    masked[2] = 0
    ref, Tref, _ = orc.composite_alpha(_layers(orc, masked), (0, 0, 8, 6))
    assert np.array_equal(out, ref) and np.array_equal(T, Tref)
    assert roi == (0, 0, 8, 6)


def test_cropped_layers_placed_by_pvp(orc):
    """A layer stored cropped (its own pvp, pitch > width) lands at its offset."""
    r = np.random.default_rng(7)
    full = _rand_layers(r, 2, 6, 8, amax=0.6)
    crop = np.zeros((3, 5, 4), np.float32)          # pitch 5, width 4
    crop[:, :4] = full[1, 2:5, 3:7]
    ims = [orc.Image((0, 0, 8, 6), (0, 0, 8, 6), np.ascontiguousarray(full[0])),
           orc.Image((3, 2, 4, 3), (3, 2, 4, 3), crop)]
    got, _, _ = orc.composite_alpha(ims, (0, 0, 8, 6))
    ref_l = full.copy()
    ref_l[1] = 0
    ref_l[1, 2:5, 3:7] = full[1, 2:5, 3:7]
    ref, _, _ = orc.composite_alpha(_layers(orc, ref_l), (0, 0, 8, 6))
    assert np.array_equal(got, ref)


def test_rejects_bad_order(orc):
    lay = np.zeros((2, 2, 2, 4), np.float32)
    with pytest.raises(orc.OracleError):
        orc.composite_alpha(_layers(orc, lay), (0, 0, 2, 2), order=[0, 0])


# ------------------------------------------------------------------ gradient


def _loss(orc, lay, g, order=None, rois=None):
    out, _, _ = orc.composite_alpha(_layers(orc, lay, rois=rois), (0, 0, lay.shape[2], lay.shape[1]),
                                    order=order)
    return float(np.sum(out * g))


@pytest.mark.parametrize("seed", range(3))
def test_gradient_matches_exact_central_differences(orc, seed):
    r = np.random.default_rng(20 + seed)
    n, H, W = 5, 2, 3
    lay = _rand_layers(r, n, H, W, amax=0.9, dyadic=True)
    g = np.round((r.random((H, W, 4)) * 2 - 1) * 4096) / 4096
    order = r.permutation(n) if seed else None
    rois = [(0, 0, W, H)] * n
    if seed == 2:
        rois[1] = (1, 0, 2, 1)
    grads = orc.composite_alpha_backward(_layers(orc, lay, rois=rois), (0, 0, W, H), g, order=order)
    h = 2.0 ** -8
    for i in range(n):
        for y in range(H):
            for x in range(W):
                for ch in range(4):
                    p, m = lay.copy(), lay.copy()
                    p[i, y, x, ch] += h
                    m[i, y, x, ch] -= h
                    fd = (_loss(orc, p, g, order, rois) - _loss(orc, m, g, order, rois)) / (2 * h)
                    assert abs(grads[i][y, x, ch] - fd) <= 1e-12 * (1 + abs(fd)), (i, y, x, ch)


def test_gradient_closed_forms(orc):
    r = np.random.default_rng(30)
    H, W = 2, 2
    g = r.random((H, W, 4)) * 2 - 1
    lay1 = _rand_layers(r, 1, H, W)
    (d,) = orc.composite_alpha_backward(_layers(orc, lay1), (0, 0, W, H), g)
    assert np.allclose(d, g, atol=0, rtol=0)           # n = 1: dc = g, da = g^A
    lay2 = _rand_layers(r, 2, H, W)
    d0, d1 = orc.composite_alpha_backward(_layers(orc, lay2), (0, 0, W, H), g)
    c1 = lay2[1].astype(np.float64)
    a0 = lay2[0, ..., 3].astype(np.float64)
    assert np.allclose(d0[..., 3], g[..., 3] - np.sum(g * c1, axis=-1), atol=1e-15)
    assert np.allclose(d1[..., :3], g[..., :3] * (1 - a0)[..., None], atol=1e-15)
    assert np.allclose(d1[..., 3], (1 - a0) * g[..., 3], atol=1e-15)


def test_gradient_region_written(orc):
    """Gradients are written over pvp_i inside the output viewport (zero outside
    roi_i); the rest of the buffer is left alone."""
    r = np.random.default_rng(31)
    lay = _rand_layers(r, 2, 4, 4)
    ims = [orc.Image((0, 0, 4, 4), (1, 1, 2, 2), lay[0]), orc.Image((0, 0, 4, 4), (0, 0, 4, 4), lay[1])]
    g = r.random((3, 3, 4))
    d0, d1 = orc.composite_alpha_backward(ims, (1, 0, 3, 3), g, fill=np.nan)
    assert np.all(np.isnan(d0[:, 0])) and np.all(np.isnan(d0[3]))
    assert np.all(d0[0, 1:] == 0) and np.all(d0[1:3, 3] == 0)
    assert np.all(np.isfinite(d0[1:3, 1:3]))
    assert np.all(np.isfinite(d1[:3, 1:]))
