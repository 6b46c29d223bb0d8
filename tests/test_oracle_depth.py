"""Pins for the depth-compositing oracle (thesis 5.2.1 z-sorted sort-last, 3.6 unordered
compositing, 5.3 region of interest).

The oracle is checked against things other than itself: an independent numpy
formulation (argmin over a stacked candidate array, which is numpy's own first-
minimum rule), order invariance, contiguous-tree equality, idempotence and the
closed forms of the degenerate cases.
"""
import itertools

import numpy as np
import pytest

import synthetic as S


def _tiny_source(r, W, H, crop, qlevels=4, nan_p=0.0, zero_p=0.0):
    """Random tiny source: per-pixel quantised depths (many ties), random ROI."""
    if crop:
        x0, y0 = int(r.integers(0, W)), int(r.integers(0, H))
        pvp = (x0, y0, int(r.integers(1, W - x0 + 1)), int(r.integers(1, H - y0 + 1)))
    else:
        pvp = (0, 0, W, H)
    rx = pvp[0] + int(r.integers(0, pvp[2] + 1))
    ry = pvp[1] + int(r.integers(0, pvp[3] + 1))
    roi = (rx, ry, int(r.integers(0, pvp[0] + pvp[2] - rx + 1)),
           int(r.integers(0, pvp[1] + pvp[3] - ry + 1)))
    pitch = pvp[2] + int(r.integers(0, 3))
    depth = (r.integers(0, qlevels + 1, size=(pvp[3], pitch)) / qlevels).astype(np.float32)
    depth[r.random(depth.shape) < nan_p] = np.nan
    z = r.random(depth.shape) < zero_p
    depth[z] = np.where(r.random(depth.shape) < 0.5, np.float32(0.0), np.float32(-0.0))[z]
    color = r.integers(0, 2**32, size=(pvp[3], pitch), dtype=np.uint64).astype(np.uint32)
    return pvp, roi, color, depth


def _numpy_merge(srcs, out_pvp):
    """Independent formulation: candidate depth stack with the background first,
    +inf where a source has no data (outside its ROI) or NaN, then np.argmin
    (first minimum: background wins ties, then the lower source index)."""
    ox, oy, W, H = out_pvp
    D = np.full((len(srcs) + 1, H, W), np.inf, dtype=np.float64)
    Cst = np.zeros((len(srcs) + 1, H, W), dtype=np.uint32)
    D[0] = 1.0
    for i, (pvp, roi, color, depth) in enumerate(srcs):
        for y in range(H):
            for x in range(W):
                px, py = ox + x, oy + y
                if roi[0] <= px < roi[0] + roi[2] and roi[1] <= py < roi[1] + roi[3]:
                    d = depth[py - pvp[1], px - pvp[0]]
                    D[i + 1, y, x] = np.inf if np.isnan(d) else d
                    Cst[i + 1, y, x] = color[py - pvp[1], px - pvp[0]]
    # -0.0 and +0.0 compare equal in argmin, as in IEEE '<'
    win = np.argmin(D, axis=0)
    color = np.take_along_axis(Cst, win[None], 0)[0]
    dep = np.where(win == 0, np.float32(1.0), 0).astype(np.float32)
    for i, (pvp, roi, c, depth) in enumerate(srcs):
        m = win == i + 1
        ys, xs = np.nonzero(m)
        dep[ys, xs] = depth[ys + oy - pvp[1], xs + ox - pvp[0]]
    return color, dep, (win - 1).astype(np.int16)


def _run(orc, srcs, out_pvp):
    ims = [orc.Image(p, r, c, d) for (p, r, c, d) in srcs]
    return orc.composite_depth(ims, out_pvp)


@pytest.mark.parametrize("seed", range(60))
def test_matches_independent_argmin(orc, seed):
    r = np.random.default_rng(seed)
    W, H = 4, 4
    n = int(r.integers(0, 5))
    srcs = [_tiny_source(r, W, H, crop=bool(seed % 2), nan_p=0.1 if seed % 3 == 0 else 0.0,
                         zero_p=0.2 if seed % 5 == 0 else 0.0) for _ in range(n)]
    out_pvp = (0, 0, W, H) if seed % 4 else (1, 0, 3, 4)
    col, dep, win, _ = _run(orc, srcs, out_pvp)
    ec, ed, ew = _numpy_merge(srcs, out_pvp)
    assert np.array_equal(col[:, :out_pvp[2]], ec)
    assert np.array_equal(dep[:, :out_pvp[2]].view(np.uint32), ed.view(np.uint32))
    assert np.array_equal(win, ew)


@pytest.mark.parametrize("seed", range(10))
def test_order_invariant_without_ties(orc, seed):
    """Unordered compositing (thesis 3.6): with distinct depths any arrival order
    gives the same frame."""
    r = np.random.default_rng(100 + seed)
    W, H, n = 4, 4, 4
    depths = r.permutation(n * W * H + 1)[:n * W * H].reshape(n, H, W) / (n * W * H + 2)
    srcs = []
    for i in range(n):
        c = r.integers(0, 2**32, size=(H, W), dtype=np.uint64).astype(np.uint32)
        srcs.append(((0, 0, W, H), (0, 0, W, H), c, depths[i].astype(np.float32)))
    ref = _run(orc, srcs, (0, 0, W, H))
    for perm in itertools.permutations(range(n)):
        got = _run(orc, [srcs[i] for i in perm], (0, 0, W, H))
        assert np.array_equal(got[0], ref[0])
        assert np.array_equal(got[1], ref[1])
        # winner indices are relabelled by the permutation
        inv = {p: k for k, p in enumerate(perm)}
        mapped = np.vectorize(lambda w: -1 if w < 0 else inv[int(w)])(ref[2])
        assert np.array_equal(got[2], mapped)


@pytest.mark.parametrize("seed", range(10))
def test_contiguous_tree_equals_sequential(orc, seed):
    """merge(merge(A,B), merge(C,D)) == merge(A,B,C,D): a tree over contiguous
    ranges keeps the lower-index tie rule (thesis 5.2.2 binary-tree compositing)."""
    r = np.random.default_rng(200 + seed)
    W, H = 6, 5
    srcs = [_tiny_source(r, W, H, crop=True) for _ in range(4)]
    full = (0, 0, W, H)
    seq = _run(orc, srcs, full)
    left = _run(orc, srcs[:2], full)
    right = _run(orc, srcs[2:], full)
    tree = _run(orc, [(full, full, left[0], left[1]), (full, full, right[0], right[1])], full)
    assert np.array_equal(tree[0], seq[0])
    assert np.array_equal(tree[1].view(np.uint32), seq[1].view(np.uint32))


def test_idempotent_and_identity(orc):
    src = S.depth_source(64, 48, 0.4, 11, 0)
    a = (src.pvp, src.roi, src.color.numpy(), src.depth.numpy())
    one = _run(orc, [a], (0, 0, 64, 48))
    two = _run(orc, [a, a], (0, 0, 64, 48))
    assert np.array_equal(one[0], two[0]) and np.array_equal(one[1], two[1])
    # an empty-ROI source contributes nothing, wherever it sits in the order
    empty = ((0, 0, 64, 48), (5, 5, 0, 0), np.full((48, 64), 7, np.uint32),
             np.zeros((48, 64), np.float32))
    for lst in ([empty, a], [a, empty]):
        got = _run(orc, lst, (0, 0, 64, 48))
        assert np.array_equal(got[0], one[0]) and np.array_equal(got[1], one[1])


def test_single_source_is_masked_copy(orc):
    """N = 1: inside the ROI the source shows where its depth is below the cleared
    1.0; everything else is background (RGBA 0, depth 1.0)."""
    src = S.depth_source(40, 30, 0.5, 12, 0, clustered=True, cropped=True)
    c, d = src.color.numpy(), src.depth.numpy()
    col, dep, win, roi = _run(orc, [(src.pvp, src.roi, c, d)], (0, 0, 40, 30))
    exp_c = np.zeros((30, 40), np.uint32)
    exp_d = np.ones((30, 40), np.float32)
    px, py, pw, ph = src.pvp
    sub_d = d[:, :pw]
    mask = sub_d < 1.0
    rx, ry, rw, rh = src.roi
    roimask = np.zeros_like(mask)
    roimask[ry - py:ry - py + rh, rx - px:rx - px + rw] = True
    mask &= roimask
    exp_c[py:py + ph, px:px + pw][mask] = c[:, :pw][mask]
    exp_d[py:py + ph, px:px + pw][mask] = sub_d[mask]
    assert np.array_equal(col, exp_c) and np.array_equal(dep, exp_d)
    assert roi == src.roi


def test_out_roi_is_bbox_union(orc):
    """Thesis 5.3: the output ROI is the merge of the input ROIs, clipped to the
    destination viewport; empty union -> {0,0,0,0}."""
    W, H = 20, 10
    z = np.ones((H, W), np.float32)
    c = np.zeros((H, W), np.uint32)
    srcs = [((0, 0, W, H), (2, 3, 4, 2), c, z), ((0, 0, W, H), (10, 1, 5, 8), c, z),
            ((0, 0, W, H), (7, 7, 0, 3), c, z)]
    assert _run(orc, srcs, (0, 0, W, H))[3] == (2, 1, 13, 8)
    assert _run(orc, srcs, (3, 0, 10, 10))[3] == (3, 1, 10, 8)
    assert _run(orc, srcs[2:], (0, 0, W, H))[3] == (0, 0, 0, 0)
    assert _run(orc, [], (0, 0, W, H))[3] == (0, 0, 0, 0)


def test_wide_colour_is_bit_copied(orc):
    """RGBA32F colour (the differentiable depth variant) is copied bit for bit."""
    r = np.random.default_rng(5)
    W, H = 5, 3
    srcs = []
    for i in range(3):
        col = r.standard_normal((H, W, 4)).astype(np.float32)
        dep = r.random((H, W)).astype(np.float32)
        srcs.append(((0, 0, W, H), (0, 0, W, H), col, dep))
    col, dep, win, _ = _run(orc, srcs, (0, 0, W, H))
    stack = np.stack([s[3] for s in srcs])
    w = np.argmin(stack, axis=0)
    assert np.array_equal(win, w.astype(np.int16))
    for y in range(H):
        for x in range(W):
            assert np.array_equal(col[y, x].view(np.uint32), srcs[w[y, x]][2][y, x].view(np.uint32))


def test_rejects_bad_rects(orc):
    z = np.ones((4, 4), np.float32)
    c = np.zeros((4, 4), np.uint32)
    with pytest.raises(orc.OracleError):
        _run(orc, [((0, 0, 4, 4), (2, 2, 3, 1), c, z)], (0, 0, 4, 4))  # roi outside pvp
    with pytest.raises(orc.OracleError):
        orc.composite_depth([orc.Image((0, 0, 4, 4), (0, 0, 4, 4), c, z)], (0, 0, -1, 4))
