"""Pins of the L-ORB oracle (FAST-9 + Harris + NMS + top-N + BRIEF, Sec. 4.1): hand-made corner
images, and an independent NumPy/SciPy formulation of every step compared exactly (all integer
arithmetic)."""
import numpy as np
import pytest
from scipy.signal import convolve2d

import oracle
import synth

MARGIN = 18
CIRCLE = [(0, -3), (1, -3), (2, -2), (3, -1), (3, 0), (3, 1), (2, 2), (1, 3), (0, 3), (-1, 3), (-2, 2), (-3, 1),
          (-3, 0), (-3, -1), (-2, -2), (-1, -3)]
B5 = np.array([1, 4, 6, 4, 1], np.int64)


def _gray(frame):
    f = frame.astype(np.int64)
    return (77 * f[..., 0] + 150 * f[..., 1] + 29 * f[..., 2] + 128) >> 8


def _numpy_lorb(frame, areas, pattern, fast_t, harris_t, max_points):
    g = _gray(frame)
    H, W = g.shape
    mask = np.zeros((H, W), bool)
    for x0, y0, x1, y1 in areas:
        mask[max(y0, MARGIN):min(y1, H - MARGIN), max(x0, MARGIN):min(x1, W - MARGIN)] = True
    # FAST-9: runs of 9 along the doubled circle (dense formulation over the whole image)
    pad = np.pad(g, 3)
    ring = np.stack([pad[3 + dy:3 + dy + H, 3 + dx:3 + dx + W] for dx, dy in CIRCLE])
    brighter = ring > g[None] + fast_t
    darker = ring < g[None] - fast_t
    def has_run(b):
        bb = np.concatenate([b, b], axis=0).astype(np.int32)
        run = np.zeros((H, W), np.int32)
        best = np.zeros((H, W), np.int32)
        for k in range(32):
            run = (run + 1) * bb[k]
            best = np.maximum(best, run)
        return best >= 9
    fast = has_run(brighter) | has_run(darker)
    # structure tensor with the unnormalised binomial, and R' = 25 det - tr^2
    ix = np.zeros_like(g)
    iy = np.zeros_like(g)
    ix[:, 1:-1] = g[:, 2:] - g[:, :-2]
    iy[1:-1, :] = g[2:, :] - g[:-2, :]
    k2 = np.outer(B5, B5)
    A = convolve2d(ix * ix, k2, mode="same")
    Bm = convolve2d(iy * iy, k2, mode="same")
    C = convolve2d(ix * iy, k2, mode="same")
    R = 25 * (A * Bm - C * C) - (A + Bm) ** 2
    cand = mask & fast & (R > harris_t)
    Rm = np.where(cand, R, np.iinfo(np.int64).min)
    idx = np.arange(H * W).reshape(H, W)
    keep = cand.copy()
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            if dx == 0 and dy == 0:
                continue
            nr = np.roll(np.roll(Rm, -dy, 0), -dx, 1)
            ni = np.roll(np.roll(idx, -dy, 0), -dx, 1)
            ncand = np.roll(np.roll(cand, -dy, 0), -dx, 1)
            beats = (Rm > nr) | ((Rm == nr) & (idx < ni))
            keep &= ~ncand | beats
    ys, xs = np.nonzero(keep)
    order = np.lexsort((idx[ys, xs], -R[ys, xs]))[:max_points]
    ys, xs = ys[order], xs[order]
    S = convolve2d(g, k2, mode="same")
    desc = np.zeros((len(xs), 32), np.uint8)
    for b in range(256):
        px, py, qx, qy = (int(v) for v in pattern[b])
        bit = S[ys + py, xs + px] > S[ys + qy, xs + qx]
        desc[:, b >> 3] |= (bit.astype(np.uint8) << (b & 7))
    return np.stack([xs, ys], 1), R[ys, xs], desc, np.where(cand, R, np.iinfo(np.int64).min)


def test_square_corners_are_fast_corners_and_edges_are_not():
    img = np.full((80, 80, 3), 20, np.uint8)
    img[30:50, 30:50] = 200
    pat = synth.brief_pattern()
    r = oracle.lorb(img, [(0, 0, 80, 80)], pat, fast_t=20, max_points=50, debug=True)
    pts = {tuple(p) for p in r["xy"]}
    assert pts == {(30, 30), (49, 30), (30, 49), (49, 49)}, pts
    # a pixel in the middle of an edge is not a FAST-9 corner
    assert r["resp_map"][30, 40] == np.iinfo(np.int64).min


def test_flat_image_has_no_features_and_areas_restrict():
    img = np.full((60, 90, 3), 77, np.uint8)
    pat = synth.brief_pattern()
    assert len(oracle.lorb(img, [(0, 0, 90, 60)], pat)["xy"]) == 0
    img[25:35, 25:35] = 250
    assert len(oracle.lorb(img, [(0, 0, 90, 60)], pat)["xy"]) == 4
    assert len(oracle.lorb(img, [(40, 0, 90, 60)], pat)["xy"]) == 0


@pytest.mark.parametrize("fast_t,harris_t,max_points", [(20, 0, 300), (10, 10 ** 12, 1000), (35, 0, 40)])
def test_matches_independent_numpy_formulation(fast_t, harris_t, max_points):
    cfg = synth.config_4x1080p(scale=0.25, frames=1)
    frame = cfg.frame(0)[1]
    H, W = frame.shape[:2]
    areas = [(0, 0, W // 2, H), (W // 3, H // 4, W, H)]
    pat = synth.brief_pattern(3)
    r = oracle.lorb(frame, areas, pat, fast_t, harris_t, max_points, debug=True)
    xy, resp, desc, rmap = _numpy_lorb(frame, areas, pat, fast_t, harris_t, max_points)
    assert len(xy) > 10
    np.testing.assert_array_equal(r["resp_map"], rmap)
    np.testing.assert_array_equal(r["xy"], xy)
    np.testing.assert_array_equal(r["resp"], resp)
    np.testing.assert_array_equal(r["desc"], desc)
