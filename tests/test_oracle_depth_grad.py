"""Pin for the depth-compositing gradient oracle: the output colour of a pixel is a
copy of its winner's colour (thesis 5.2.1), so dL/dcolor_i = g where source i
won and 0 elsewhere -- checked by brute force against the forward's winners
and against a finite difference of the forward with RGBA32F colour."""
import numpy as np


def test_depth_grad_routes_to_winner(orc):
    r = np.random.default_rng(3)
    W, H, n = 7, 5, 4
    ims, pvps, rois, pitches = [], [], [], []
    for i in range(n):
        pvp = (int(r.integers(0, 3)), int(r.integers(0, 2)), 0, 0)
        pvp = (pvp[0], pvp[1], W - pvp[0] - int(r.integers(0, 2)), H - pvp[1])
        roi = (pvp[0] + 1, pvp[1], pvp[2] - 1, pvp[3] - 1) if i % 2 else pvp
        pitch = pvp[2] + 1
        col = r.standard_normal((pvp[3], pitch, 4)).astype(np.float32)
        dep = (r.integers(0, 4, size=(pvp[3], pitch)) / 4).astype(np.float32)
        ims.append(orc.Image(pvp, roi, col, dep))
        pvps.append(pvp); rois.append(roi); pitches.append(pitch)
    out_pvp = (0, 0, W, H)
    col, dep, win, _ = orc.composite_depth(ims, out_pvp)
    g = r.standard_normal((H, W, 4)).astype(np.float32)
    grads = orc.composite_depth_backward(win, out_pvp, g, pvps, pitches, fill=np.nan)
    for i in range(n):
        px, py, pw, ph = pvps[i]
        for y in range(ph):
            for x in range(pw):
                X, Y = px + x, py + y
                exp = g[Y, X] if win[Y, X] == i else np.zeros(4, np.float32)
                assert np.array_equal(grads[i][y, x], exp)
                # colour perturbation moves the loss by g exactly where i won
                c2 = [im.color.copy() for im in ims]
                c2[i][y, x] += 1.0
                ims2 = [orc.Image(im.pvp, im.roi, c, im.depth) for im, c in zip(ims, c2)]
                col2 = orc.composite_depth(ims2, out_pvp)[0]
                dl = np.sum((col2.astype(np.float64) - col) * g, axis=(0, 1))
                assert np.allclose(dl, grads[i][y, x], atol=1e-5)
        assert np.all(np.isnan(grads[i][:, pw:]))       # pitch padding untouched
