"""Pins of the FP64 oracle against facts fixed independently of its code (CPU only).

Each test names the property it checks.  The paper prints no worked example and no intermediate
values for the stitching path, so the pins are closed forms of the operators, invariants of the
method (identity, integer translation, telescoping collapse, constants, weights summing to one),
an independent dense-matrix formulation on tiny sizes, an independent NumPy formulation of the
whole forward path on a small blended rig, and finite differences for the gradient.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from synth import Camera
from tests import dense_ref

RNG = np.random.default_rng(12345)


def _T(tx, ty):
    return np.array([[1.0, 0, tx], [0, 1.0, ty], [0, 0, 1.0]])


def _rand_frame(h, w, seed=0):
    return np.random.default_rng(seed).integers(0, 256, (h, w, 3), dtype=np.uint8)


# ---------------------------------------------------------------------------------------------
# P6: closed forms of REDUCE / EXPAND


def test_reduce_impulse_response_polyphase():
    """An impulse at an even fine index 2a reduces to (1,6,1)/16 per axis around a; at an odd
    index 2a+1 to (4,4)/16 on a, a+1 (columns of the REDUCE operator)."""
    n = 21
    for a in (4, 5):
        img = np.zeros((n, n))
        img[2 * a, 2 * a + 1] = 1.0
        out = oracle.reduce(img)
        ey = np.zeros(11); ey[a - 1:a + 2] = [1 / 16, 6 / 16, 1 / 16]
        ex = np.zeros(11); ex[a:a + 2] = [4 / 16, 4 / 16]
        np.testing.assert_allclose(out, np.outer(ey, ex), atol=1e-15)


def test_reduce_row_is_5tap_kernel():
    """Output k of REDUCE weighs fine samples 2k-2..2k+2 by [1,4,6,4,1]/16 (a row of the operator)."""
    n = 19
    k = 4
    row = np.zeros(n)
    for i in range(n):
        img = np.zeros((1, n))
        img[0, i] = 1.0
        row[i] = oracle.reduce(img)[0, k]
    expect = np.zeros(n)
    expect[2 * k - 2:2 * k + 3] = np.array([1, 4, 6, 4, 1]) / 16
    np.testing.assert_allclose(row, expect, atol=1e-15)


def test_expand_impulse_is_kernel_times_two():
    """A coarse impulse at k expands to (1,4,6,4,1)/8 on fine 2k-2..2k+2 per axis."""
    img = np.zeros((9, 9))
    img[4, 3] = 1.0
    out = oracle.expand(img, (17, 17))
    ey = np.zeros(17); ey[6:11] = np.array([1, 4, 6, 4, 1]) / 8
    ex = np.zeros(17); ex[4:9] = np.array([1, 4, 6, 4, 1]) / 8
    np.testing.assert_allclose(out, np.outer(ey, ex), atol=1e-15)


@pytest.mark.parametrize("shape", [(1, 1), (1, 7), (2, 2), (5, 3), (8, 9), (16, 33)])
def test_constants_preserved(shape):
    """REDUCE and EXPAND preserve constants everywhere, borders included (reflect-101)."""
    img = np.full(shape + (3,), 0.37)
    r = oracle.reduce(img)
    np.testing.assert_allclose(r, 0.37, atol=1e-15)
    np.testing.assert_allclose(oracle.expand(r, shape), 0.37, atol=1e-15)


def test_linear_ramp_interior_and_border_values():
    """Away from borders a ramp f(x)=x reduces to f(2k) and a coarse ramp g(k)=k expands to x/2.
    At the border reflect-101 gives G(0) = (2+4+0+4+2)/16 = 0.75 (plain reflection would give 7/16)."""
    n = 32
    img = np.tile(np.arange(n, dtype=np.float64), (3, 1))
    r = oracle.reduce(img)
    np.testing.assert_allclose(r[1, 1:-1], 2.0 * np.arange(1, 15), atol=1e-13)
    assert abs(r[1, 0] - 0.75) < 1e-15
    g = np.tile(np.arange(16, dtype=np.float64), (3, 1))
    e = oracle.expand(g, (5, 32))
    np.testing.assert_allclose(e[2, 2:-2], np.arange(2, 30) / 2.0, atol=1e-13)
    # fine x=0: taps k=-1 (->1) weight 1/8, k=0 weight 6/8, k=1 weight 1/8 -> 2/8
    assert abs(e[2, 0] - 0.25) < 1e-15


# ---------------------------------------------------------------------------------------------
# P7: dense-matrix brute force on tiny sizes


@pytest.mark.parametrize("h,w", [(1, 1), (1, 2), (2, 1), (3, 3), (4, 5), (7, 9), (9, 7), (6, 8), (17, 33)])
def test_reduce_expand_match_dense_matrices(h, w):
    img = RNG.standard_normal((h, w, 4))
    np.testing.assert_allclose(oracle.reduce(img), dense_ref.reduce2d(img), atol=1e-13)
    c = RNG.standard_normal(((h + 1) // 2, (w + 1) // 2, 3))
    np.testing.assert_allclose(oracle.expand(c, (h, w)), dense_ref.expand2d(c, (h, w)), atol=1e-13)


# ---------------------------------------------------------------------------------------------
# P3: collapse of an unblended Laplacian pyramid reconstructs the image (telescoping)


@pytest.mark.parametrize("h,w,L", [(1, 1, 3), (13, 7, 3), (40, 64, 4), (37, 91, 6)])
def test_collapse_of_laplacian_is_identity(h, w, L):
    img = RNG.uniform(0, 1, (h, w, 3))
    np.testing.assert_allclose(oracle.collapse(oracle.laplacian_pyramid(img, L)), img, atol=1e-12)


# ---------------------------------------------------------------------------------------------
# warp (S1) and feather weight (S2)


def test_identity_homography_reproduces_input():
    """P1: one camera, canvas = image, M = I: float output = frame/255, u8 output == frame."""
    for (h, w, L) in [(23, 37, 3), (48, 64, 4), (1, 1, 1), (5, 2, 2)]:
        fr = _rand_frame(h, w, seed=h)
        cam = Camera(w, h, np.eye(3))
        r = oracle.forward([cam], [fr], w, h, L)
        np.testing.assert_allclose(r["out"], fr / 255.0, atol=1e-12)
        assert np.array_equal(r["u8"], fr)


def test_integer_translation_warp_is_exact_shift():
    """P2 (level 0): M = T(tx, ty) samples frame[y-ty, x-tx] exactly; outside the image the value
    is the clamped edge texel and the raw weight is 0."""
    fr = _rand_frame(11, 17, 3)
    tx, ty = 5, -3
    cam = Camera(17, 11, _T(tx, ty))
    img, wr = oracle.warp(cam, fr, 30, 12)
    for y in range(12):
        for x in range(30):
            u, v = x - tx, y - ty
            uc, vc = min(max(u, 0), 16), min(max(v, 0), 10)
            np.testing.assert_array_equal(img[y, x], fr[vc, uc] / 255.0)
            inside = 0 <= u < 17 and 0 <= v < 11
            assert (wr[y, x] > 0) == inside


def test_integer_translation_full_path_exact_when_covered():
    """P2 (whole path): a translated camera covering the whole canvas reproduces the shifted
    frame exactly."""
    fr = _rand_frame(40, 60, 4)
    cam = Camera(60, 40, _T(-7, -5))
    r = oracle.forward([cam], [fr], 45, 29, 4)
    assert np.array_equal(r["u8"], fr[5:34, 7:52])
    np.testing.assert_allclose(r["out"], fr[5:34, 7:52] / 255.0, atol=1e-12)


def test_half_pixel_translation_is_neighbour_average():
    """Bilinear at a half-pixel offset is the mean of the two neighbours (closed form)."""
    fr = _rand_frame(6, 9, 5)
    cam = Camera(9, 6, _T(0.5, 0.0))
    img, _ = oracle.warp(cam, fr, 9, 6)
    np.testing.assert_allclose(img[:, 1:9], (fr[:, 0:8].astype(float) + fr[:, 1:9]) / 2 / 255.0, atol=1e-15)
    np.testing.assert_allclose(img[:, 0], fr[:, 0] / 255.0, atol=1e-15)  # u=-0.5 clamps to texel 0


def test_feather_weight_distance_to_border():
    """Raw weight = distance (source px) to the nearest image border, measured to the outer
    pixel edge: 0.5 on the border pixels, k+0.5 on ring k, 0 outside."""
    W, H = 9, 7
    cam = Camera(W, H, _T(2, 1))
    _, wr = oracle.warp(cam, np.zeros((H, W, 3), np.uint8), 14, 10)
    for y in range(10):
        for x in range(14):
            u, v = x - 2, y - 1
            if 0 <= u < W and 0 <= v < H:
                ring = min(u, v, W - 1 - u, H - 1 - v)
                assert wr[y, x] == ring + 0.5
            else:
                assert wr[y, x] == 0.0


def test_gain_scales_and_output_clamps():
    fr = np.full((8, 8, 3), 200, np.uint8)
    cam = Camera(8, 8, np.eye(3), gain=2.0)
    r = oracle.forward([cam], [fr], 8, 8, 3)
    assert np.all(r["out"] == 1.0) and np.all(r["u8"] == 255)
    cam.gain = 0.5
    r = oracle.forward([cam], [fr], 8, 8, 3)
    np.testing.assert_allclose(r["out"], 100 / 255.0, atol=1e-12)


# ---------------------------------------------------------------------------------------------
# P4 / P5: constants and weights


def test_constant_inputs_blend_to_the_constant():
    """P4: every camera shows the same constant -> output is that constant on every covered pixel
    and 0 where no camera is valid."""
    cfg = synth.config_2cam(scale=0.25)
    frames = [np.full((c.height, c.width, 3), (37, 180, 255), np.uint8) for c in cfg.cameras]
    r = oracle.forward(cfg.cameras, frames, cfg.canvas_w, cfg.canvas_h, 4)
    covered = np.zeros((cfg.canvas_h, cfg.canvas_w), bool)
    for c in cfg.cameras:
        covered |= oracle.warp(c, frames[0], cfg.canvas_w, cfg.canvas_h)[1] > 0
    assert covered.any() and (~covered).any()
    got = r["out"][covered]
    np.testing.assert_allclose(got, np.broadcast_to(np.array([37, 180, 255]) / 255.0, got.shape), atol=1e-12)
    assert np.all(r["out"][~covered] == 0.0)


def test_weights_sum_to_one_at_every_level():
    """P5: S^0 = sum_i What_i is 1 on covered pixels and 0 elsewhere, and S^l equals the l-fold
    REDUCE of the coverage indicator (dense-matrix formulation)."""
    cfg = synth.config_2cam(scale=0.2)
    frames = cfg.frame(0)
    L = 4
    r = oracle.forward(cfg.cameras, frames, cfg.canvas_w, cfg.canvas_h, L, debug=True)
    covered = np.zeros((cfg.canvas_h, cfg.canvas_w))
    for c, f in zip(cfg.cameras, frames):
        covered = np.maximum(covered, (oracle.warp(c, f, cfg.canvas_w, cfg.canvas_h)[1] > 0).astype(float))
    g = dense_ref.gaussian(covered, L)
    for l in range(L):
        x0, x1, y0, y1 = r["regions"][l][:4]
        assert (x0, y0) == (0, 0) and (x1, y1) == (g[l].shape[1], g[l].shape[0])
        np.testing.assert_allclose(r["S"][l], g[l], atol=1e-13)


def test_two_identical_cameras_average_their_frames():
    """Two cameras with the same homography get What = 1/2 each at every level, so two constant
    frames a and b blend to (a+b)/2, and equal frames reproduce the single-camera result."""
    M = synth.rig_planar(32, 24, 30.0, [5.0], 40, 30)[0]
    cams = [Camera(32, 24, M), Camera(32, 24, M)]
    fa = np.full((24, 32, 3), 40, np.uint8)
    fb = np.full((24, 32, 3), 200, np.uint8)
    r = oracle.forward(cams, [fa, fb], 40, 30, 3)
    _, wr = oracle.warp(cams[0], fa, 40, 30)
    cov = wr > 0
    np.testing.assert_allclose(r["out"][cov], 120 / 255.0, atol=1e-12)
    fr = _rand_frame(24, 32, 9)
    r2 = oracle.forward(cams, [fr, fr], 40, 30, 3)
    r1 = oracle.forward(cams[:1], [fr], 40, 30, 3)
    np.testing.assert_allclose(r2["out"], r1["out"], atol=1e-12)


def test_two_constant_cameras_blend_by_coarsest_weight_pyramid():
    """Constant frames a (camera A) and b (camera B) have zero Laplacian bands below the top, so
    the blend is the top-level weight mix expanded back: out = E^{L-1}(G^{L-1}(WA) a + G^{L-1}(WB) b)
    / E^{L-1}(S^{L-1}) reduces, with S = 1 everywhere, to E^{L-1}(G^{L-1}(WA)) (a - b) + b.
    Expected values come from the dense-matrix operators."""
    Wc, Hc, L = 48, 20, 3
    ca = Camera(30, 20, _T(0, 0))   # covers x in [0, 30)
    cb = Camera(30, 20, _T(18, 0))  # covers x in [18, 48)
    fa = np.full((20, 30, 3), 60, np.uint8)
    fb = np.full((20, 30, 3), 220, np.uint8)
    r = oracle.forward([ca, cb], [fa, fb], Wc, Hc, L)
    _, wa = oracle.warp(ca, fa, Wc, Hc)
    _, wb = oracle.warp(cb, fb, Wc, Hc)
    What_a = np.where(wa + wb > 0, wa / np.where(wa + wb > 0, wa + wb, 1), 0)
    g = dense_ref.gaussian(What_a, L)
    top = g[-1]
    e = top
    shapes = [dense_ref.gaussian(np.zeros((Hc, Wc)), L)[l].shape for l in range(L)]
    for l in range(L - 2, -1, -1):
        e = dense_ref.expand2d(e, shapes[l])
    expect = e * (60 / 255.0) + (1 - e) * (220 / 255.0)
    np.testing.assert_allclose(r["out"][:, :, 0], expect, atol=1e-12)


# ---------------------------------------------------------------------------------------------
# regions / windows


def test_window_is_bit_identical_to_full_canvas():
    cfg = synth.config_2cam(scale=0.3)
    frames = cfg.frame(0)
    full = oracle.forward(cfg.cameras, frames, cfg.canvas_w, cfg.canvas_h, 4)
    for win in [(0, 0, 17, 9), (cfg.canvas_w - 23, cfg.canvas_h - 11, 23, 11), (101, 37, 64, 40)]:
        x0, y0, w, h = win
        part = oracle.forward(cfg.cameras, frames, cfg.canvas_w, cfg.canvas_h, 4, window=win)
        assert np.array_equal(part["out"], full["out"][y0:y0 + h, x0:x0 + w])
        assert np.array_equal(part["u8"], full["u8"][y0:y0 + h, x0:x0 + w])


# ---------------------------------------------------------------------------------------------
# S7: loss and gradient


def _params_of(cams, gains=None):
    ps = []
    for i, c in enumerate(cams):
        A = oracle.invert_h(c.H).reshape(9)
        assert A[8] == 1.0
        ps.append(np.r_[A[:8], 1.0 if gains is None else gains[i]])
    return np.array(ps)


def test_loss_closed_form_for_constant_frames():
    """Constant frames c_A, c_B with gains g_A, g_B: loss = K * 3 * (g_A c_A - g_B c_B)^2 / 255^2,
    K = number of canvas pixels valid in both."""
    ca = Camera(20, 10, _T(0, 0))
    cb = Camera(20, 10, _T(12, 3))
    fa = np.full((10, 20, 3), 100, np.uint8)
    fb = np.full((10, 20, 3), 30, np.uint8)
    p = _params_of([ca, cb], [0.9, 1.3])
    loss, g = oracle.loss_grad([20, 20], [10, 10], p, [fa, fb], (0, 0, 32, 13))
    K = 8 * 7
    assert abs(loss - K * 3 * (0.9 * 100 - 1.3 * 30) ** 2 / 255.0 ** 2) < 1e-10
    # the gain gradients have the closed form 2 * sum r * I / g
    dA = 0.9 * 100 / 255.0 - 1.3 * 30 / 255.0
    assert abs(g[0, 8] - K * 3 * 2 * dA * 100 / 255.0) < 1e-9
    assert abs(g[1, 8] + K * 3 * 2 * dA * 30 / 255.0) < 1e-9
    # constant frames: no spatial gradient
    assert np.all(np.abs(g[:, :8]) < 1e-12)


def _fd_check(cfg, frames, window, tol=2e-5):
    n = len(cfg.cameras)
    p0 = _params_of(cfg.cameras, [1.0 + 0.05 * i for i in range(n)])
    # move every camera off the true alignment a little so residuals are not ~0
    p0[:, 2] += 0.37
    p0[:, 5] -= 0.21
    loss, g = oracle.loss_grad([c.width for c in cfg.cameras], [c.height for c in cfg.cameras], p0, frames,
                               window)
    # the spatial parts must be populated, otherwise the check below is vacuous
    assert np.all(np.abs(g[:, :8]).max(axis=1) > 1e-3 * np.abs(g).max())
    Ws = [c.width for c in cfg.cameras]
    Hs = [c.height for c in cfg.cameras]
    # step of each parameter sized so the sample coordinates move by ~1e-6 px over the window
    ext = float(max(window[0] + window[2], window[1] + window[3]))
    steps = [1e-6 / ext, 1e-6 / ext, 1e-6, 1e-6 / ext, 1e-6 / ext, 1e-6, 1e-6 / ext ** 2, 1e-6 / ext ** 2, 1e-6]
    for i in range(n):
        for k in range(9):
            h = steps[k]
            pp = p0.copy(); pp[i, k] += h
            pm = p0.copy(); pm[i, k] -= h
            lp, _ = oracle.loss_grad(Ws, Hs, pp, frames, window, mask_params=p0, grad=False)
            lm, _ = oracle.loss_grad(Ws, Hs, pm, frames, window, mask_params=p0, grad=False)
            fd = (lp - lm) / (2 * h)
            scale = max(abs(g[i, k]), 1e-3 * np.abs(g[i]).max())
            assert abs(fd - g[i, k]) <= tol * scale, (i, k, fd, g[i, k])
    return loss, g


def test_gradient_matches_central_differences():
    """P8: analytic gradient vs central differences with frozen masks (tiny relative steps keep the
    difference inside one bilinear cell almost everywhere)."""
    cfg = synth.config_2cam(scale=0.15)
    frames = cfg.frame(0)
    _fd_check(cfg, frames, (0, 0, cfg.canvas_w, cfg.canvas_h))


def _three_camera_rig():
    th = math.radians(7.0)
    rot = np.array([[math.cos(th), -math.sin(th), 19.4], [math.sin(th), math.cos(th), 1.7], [6e-4, -4e-4, 1.0]])
    cams = [Camera(24, 18, _T(2.3, 3.7)), Camera(22, 17, rot, 1.1),
            Camera(20, 16, np.array([[0.8, 0.0, 9.6], [0.0, 0.8, 11.2], [0.0, 0.0, 1.0]]), 0.9)]
    frames = [_rand_frame(c.height, c.width, seed=k + 11) for k, c in enumerate(cams)]
    return cams, frames


def test_three_camera_loss_and_gradient_are_sums_over_pairs():
    """The loss is a sum over camera pairs of their overlap terms (S7), so on a rig where some
    pixels are covered by two cameras and some by all three, the loss and each camera's gradient
    equal the sums of the two-camera problems that contain it."""
    cams, frames = _three_camera_rig()
    Ws, Hs = [c.width for c in cams], [c.height for c in cams]
    p = _params_of(cams, [1.0, 1.1, 0.9])
    p[:, 2] += 0.37
    win = (0, 0, 44, 27)
    loss, g = oracle.loss_grad(Ws, Hs, p, frames, win)
    want_loss, want_g = 0.0, np.zeros_like(g)
    for i, j in ((0, 1), (0, 2), (1, 2)):
        lij, gij = oracle.loss_grad([Ws[i], Ws[j]], [Hs[i], Hs[j]], p[[i, j]], [frames[i], frames[j]], win)
        assert lij > 0.0  # every pair overlaps
        want_loss += lij
        want_g[i] += gij[0]
        want_g[j] += gij[1]
    assert abs(loss - want_loss) <= 1e-12 * want_loss
    np.testing.assert_allclose(g, want_g, rtol=1e-10, atol=1e-12 * np.abs(want_g).max())
    # the rig has pixels covered by exactly two cameras and pixels covered by all three
    ys, xs = np.mgrid[0:27, 0:44]
    cov = []
    for k, c in enumerate(cams):
        q = np.tensordot(np.linalg.inv(np.asarray(c.H)), np.stack([xs, ys, np.ones_like(xs)]), 1)
        cov.append((q[2] > 0) & (q[0] / q[2] >= -0.5) & (q[0] / q[2] < c.width - 0.5) & (q[1] / q[2] >= -0.5) &
                   (q[1] / q[2] < c.height - 0.5))
    n_cov = sum(c.astype(int) for c in cov)
    assert (n_cov == 2).sum() > 20 and (n_cov == 3).sum() > 20


def test_three_camera_gradient_matches_central_differences():
    """P8 on the three-camera rig (partial triple overlap, a projective camera, gains != 1)."""
    cams, frames = _three_camera_rig()

    class _Rig:
        cameras = cams
    _fd_check(_Rig, frames, (0, 0, 44, 27))


def test_translation_gradient_has_lucas_kanade_form():
    """For a pure translation A = T(-t) the a13 / a23 gradients are 2 sum r dI/du and 2 sum r dI/dv
    (w = 1), i.e. minus the gradient of the loss with respect to the canvas shift of the camera;
    checked by moving the camera instead of its parameters."""
    fr_a = _rand_frame(30, 40, 1)
    fr_b = _rand_frame(30, 40, 2)
    ca = Camera(40, 30, _T(0, 0))
    cb = Camera(40, 30, _T(10.3, 4.6))
    p = _params_of([ca, cb])
    win = (0, 0, 52, 36)
    loss, g = oracle.loss_grad([40, 40], [30, 30], p, [fr_a, fr_b], win)
    h = 1e-6
    # camera B shifted on the canvas by +h in x: a13 of B decreases by h
    cb2 = Camera(40, 30, _T(10.3 + h, 4.6))
    cb3 = Camera(40, 30, _T(10.3 - h, 4.6))
    lp, _ = oracle.loss_grad([40, 40], [30, 30], _params_of([ca, cb2]), [fr_a, fr_b], win, mask_params=p, grad=False)
    lm, _ = oracle.loss_grad([40, 40], [30, 30], _params_of([ca, cb3]), [fr_a, fr_b], win, mask_params=p, grad=False)
    d_shift = (lp - lm) / (2 * h)
    assert abs(d_shift + g[1, 2]) <= 1e-5 * abs(g[1, 2])
    # and a11/a12 gradients equal x- and y-weighted sums of the same integrand (w = 1)
    assert abs(g[1, 6]) > 0  # projective terms are populated


def test_invert_h_roundtrip():
    M = synth.config_2cam().cameras[1].H
    A = oracle.invert_h(M)
    P = M @ A
    np.testing.assert_allclose(P / P[2, 2], np.eye(3), atol=1e-12)
    assert A[2, 2] == 1.0


def test_inverse_keeps_the_in_front_sign():
    """A camera yawed so far that the canvas origin is behind it: the inverse keeps w > 0 on the
    camera's own footprint (a33 = -1 then), so its pixels are valid and the footprint centre maps
    back to the image centre."""
    cfg = synth.config_4x1080p(scale=0.25, frames=1)
    cam = cfg.cameras[3]
    A = oracle.invert_h(cam.H)
    assert A[2, 2] == -1.0
    p = cam.H @ np.array([(cam.width - 1) / 2, (cam.height - 1) / 2, 1.0])
    q = A @ (p / p[2])
    assert q[2] > 0
    np.testing.assert_allclose(q[:2] / q[2], [(cam.width - 1) / 2, (cam.height - 1) / 2], atol=1e-9)
    _, wr = oracle.warp(cam, np.zeros((cam.height, cam.width, 3), np.uint8), cfg.canvas_w, cfg.canvas_h)
    assert (wr > 0).sum() > 0.5 * cam.width * cam.height



# ---------------------------------------------------------------------------------------------
# seam weights (binary masks of the multiresolution spline)


def _owner_map(cams, frames, Wc, Hc):
    """Owner of every canvas pixel from the cameras' raw feather weights (oracle.warp), with the
    tie rule written out in NumPy: lowest index with w > 0 and w >= (1 - 1e-9) max w; -1: none."""
    w = np.stack([oracle.warp(c, f, Wc, Hc)[1] for c, f in zip(cams, frames)])
    wmax = w.max(axis=0)
    ok = (w > 0) & (w >= (1 - 1e-9) * wmax[None])
    own = np.where(ok.any(axis=0), ok.argmax(axis=0), -1)
    return own, w


def test_seam_single_level_is_hard_cut_to_the_owner():
    """With one level there is no pyramid: each covered pixel is its owner camera's warped
    sample, uncovered pixels are 0."""
    cfg = synth.config_2cam(scale=0.2)
    frames = cfg.frame(0)
    r = oracle.forward(cfg.cameras, frames, cfg.canvas_w, cfg.canvas_h, 1, weights="seam")
    own, _ = _owner_map(cfg.cameras, frames, cfg.canvas_w, cfg.canvas_h)
    imgs = [oracle.warp(c, f, cfg.canvas_w, cfg.canvas_h)[0] for c, f in zip(cfg.cameras, frames)]
    expect = np.zeros_like(r["out"])
    for i, img in enumerate(imgs):
        expect[own == i] = np.clip(img[own == i], 0, 1)
    assert (own == 0).any() and (own == 1).any() and (own == -1).any()
    np.testing.assert_allclose(r["out"], expect, atol=1e-15)


def test_seam_ties_go_to_the_lower_camera():
    """Two mirror-symmetric cameras: on the symmetry column both feather weights are equal, and
    the pixel belongs to camera 0 (one level, so the output is the owner's sample)."""
    Wc, Hc = 41, 16
    ca = Camera(30, 16, _T(0, 0))    # covers x in [0, 30)
    cb = Camera(30, 16, _T(11, 0))   # covers x in [11, 41); column 20 is equidistant
    fa = np.full((16, 30, 3), 50, np.uint8)
    fb = np.full((16, 30, 3), 150, np.uint8)
    r = oracle.forward([ca, cb], [fa, fb], Wc, Hc, 1, weights="seam")
    wa = oracle.warp(ca, fa, Wc, Hc)[1]
    wb = oracle.warp(cb, fb, Wc, Hc)[1]
    tie = (wa == wb) & (wa > 0)
    assert tie[:, 20].all()
    np.testing.assert_allclose(r["out"][tie], 50 / 255.0, atol=1e-15)
    np.testing.assert_allclose(r["out"][(wa > wb)], 50 / 255.0, atol=1e-15)
    np.testing.assert_allclose(r["out"][(wb > wa) & (wb > 0)], 150 / 255.0, atol=1e-15)


def test_seam_weights_are_one_hot_and_blend_constants_exactly():
    """S^0 = 1 on covered pixels (exactly one owner), S^l follows the REDUCE of the coverage, and
    constant frames still blend to the constant (P4 holds for binary masks too)."""
    cfg = synth.config_2cam(scale=0.2)
    frames = cfg.frame(0)
    L = 4
    r = oracle.forward(cfg.cameras, frames, cfg.canvas_w, cfg.canvas_h, L, debug=True, weights="seam")
    own, _ = _owner_map(cfg.cameras, frames, cfg.canvas_w, cfg.canvas_h)
    covered = (own >= 0).astype(float)
    g = dense_ref.gaussian(covered, L)
    for l in range(L):
        np.testing.assert_allclose(r["S"][l], g[l], atol=1e-13)
    const = [np.full((c.height, c.width, 3), (90, 12, 240), np.uint8) for c in cfg.cameras]
    rc = oracle.forward(cfg.cameras, const, cfg.canvas_w, cfg.canvas_h, L, weights="seam")
    np.testing.assert_allclose(rc["out"][own >= 0], np.broadcast_to(np.array([90, 12, 240]) / 255.0,
                                                                    rc["out"][own >= 0].shape), atol=1e-12)


def test_seam_blend_of_two_constants_follows_the_mask_pyramid():
    """Camera A constant a, camera B constant b, seam masks: out = E^{L-1}(G^{L-1}(M_A))(a - b) + b
    with M_A the owner mask of A (dense-matrix operators), as for feather weights."""
    Wc, Hc, L = 48, 20, 3
    ca = Camera(30, 20, _T(0, 0))
    cb = Camera(30, 20, _T(18, 0))
    fa = np.full((20, 30, 3), 60, np.uint8)
    fb = np.full((20, 30, 3), 220, np.uint8)
    r = oracle.forward([ca, cb], [fa, fb], Wc, Hc, L, weights="seam")
    own, _ = _owner_map([ca, cb], [fa, fb], Wc, Hc)
    assert (own >= 0).all()
    e = dense_ref.gaussian((own == 0).astype(float), L)[-1]
    shapes = [dense_ref.gaussian(np.zeros((Hc, Wc)), L)[l].shape for l in range(L)]
    for l in range(L - 2, -1, -1):
        e = dense_ref.expand2d(e, shapes[l])
    expect = e * (60 / 255.0) + (1 - e) * (220 / 255.0)
    np.testing.assert_allclose(r["out"][:, :, 0], expect, atol=1e-12)


def test_seam_and_feather_agree_for_one_camera():
    cfg = synth.config_2cam(scale=0.2)
    frames = cfg.frame(0)
    a = oracle.forward(cfg.cameras[:1], frames[:1], cfg.canvas_w, cfg.canvas_h, 4)
    b = oracle.forward(cfg.cameras[:1], frames[:1], cfg.canvas_w, cfg.canvas_h, 4, weights="seam")
    assert np.array_equal(a["out"], b["out"])


# ---------------------------------------------------------------------------------------------
# cylindrical canvas


def test_cylindrical_warp_closed_form():
    """Camera P = K (looking along the canvas centre column) on a cylindrical canvas of focal
    length fc: canvas (x, y) sees source u = f tan(t) + (W-1)/2, v = f (y - cy)/(fc cos t) + (H-1)/2
    with t = (x - cx)/fc.  A frame whose red channel is u and green channel is 2v (a linear ramp,
    reproduced exactly by bilinear interpolation) pins both formulas."""
    W, H, f = 256, 120, 150.0
    Wc, Hc, fc = 300, 140, 180.0
    cx, cy = 149.5, 69.5
    u = np.arange(W)[None, :].repeat(H, 0)
    v = np.arange(H)[:, None].repeat(W, 1)
    frame = np.stack([u, 2 * v, np.full_like(u, 7)], axis=2).astype(np.uint8)
    P = synth._K(f, W, H)
    img, wr = oracle.warp(Camera(W, H, P), frame, Wc, Hc, canvas=(fc, cx, cy))
    x = np.arange(Wc)[None, :]
    y = np.arange(Hc)[:, None]
    t = (x - cx) / fc
    uu = f * np.tan(t) + (W - 1) / 2.0 + 0 * y
    vv = f * (y - cy) / (fc * np.cos(t)) + (H - 1) / 2.0
    inside = (uu > 0.5) & (uu < W - 1.5) & (vv > 0.5) & (vv < H - 1.5)
    assert inside.mean() > 0.5
    np.testing.assert_allclose(img[..., 0][inside], uu[inside] / 255.0, atol=1e-12)
    np.testing.assert_allclose(img[..., 1][inside], 2 * vv[inside] / 255.0, atol=1e-12)
    # feather weight: distance to the nearest pixel-edge border of the source rectangle
    m = np.minimum(np.minimum(uu + 0.5, vv + 0.5), np.minimum(W - 0.5 - uu, H - 0.5 - vv))
    np.testing.assert_allclose(wr[inside], m[inside], atol=1e-9)


def test_cylindrical_panorama_reproduces_the_scene():
    """Views rendered from a scene on a cylindrical canvas (ray -> canvas by atan2/hypot in the
    input generator) and stitched back (canvas -> camera by sin/cos here) reproduce the scene:
    a smooth scene (noise only) within a few LSB; a wrong mapping shows errors everywhere."""
    cfg = synth.config_cyl(scale=0.25)
    cfg.scene.rects = cfg.scene.rects[:0]
    cfg.scene.lattice = 48.0  # smooth at this scale: bilinear resampling stays near 1 LSB
    frames = cfg.frame(0)
    r = oracle.forward(cfg.cameras, frames, cfg.canvas_w, cfg.canvas_h, cfg.levels, canvas=cfg.canvas)
    cov = np.zeros((cfg.canvas_h, cfg.canvas_w), bool)
    for c, f in zip(cfg.cameras, frames):
        cov |= oracle.warp(c, f, cfg.canvas_w, cfg.canvas_h, canvas=cfg.canvas)[1] > 0
    ref = synth.render_scene(cfg.scene, cfg.scene.off_x, cfg.scene.off_y, cfg.canvas_w, cfg.canvas_h)
    d = np.abs(r["u8"].astype(int) - ref.astype(int))[cov]
    assert cov.mean() > 0.8
    assert np.median(d) <= 1 and np.percentile(d, 99) <= 4, (np.median(d), np.percentile(d, 99))


def _numpy_forward(cams, frames, Wc, Hc, L):
    """S1-S6 written out with NumPy from the definitions (vectorised over the canvas, pyramids by
    the dense REDUCE/EXPAND matrices), sharing nothing with the oracle's loops."""
    ys, xs = np.mgrid[0:Hc, 0:Wc].astype(np.float64)
    imgs, wraws = [], []
    for c, f in zip(cams, frames):
        A = np.linalg.inv(np.asarray(c.H, dtype=np.float64))
        A = A / abs(A[2, 2])
        w = A[2, 0] * xs + A[2, 1] * ys + A[2, 2]
        front = w > 0.0
        ws = np.where(front, w, 1.0)
        u = (A[0, 0] * xs + A[0, 1] * ys + A[0, 2]) / ws
        v = (A[1, 0] * xs + A[1, 1] * ys + A[1, 2]) / ws
        H, W = f.shape[:2]
        uc, vc = np.clip(u, 0, W - 1), np.clip(v, 0, H - 1)
        i0, j0 = np.floor(uc).astype(int), np.floor(vc).astype(int)
        fx, fy = (uc - i0)[..., None], (vc - j0)[..., None]
        i1, j1 = np.minimum(i0 + 1, W - 1), np.minimum(j0 + 1, H - 1)
        t = f.astype(np.float64)
        top = (1 - fx) * t[j0, i0] + fx * t[j0, i1]
        bot = (1 - fx) * t[j1, i0] + fx * t[j1, i1]
        img = getattr(c, "gain", 1.0) * ((1 - fy) * top + fy * bot) / 255.0
        img[~front] = 0.0
        valid = front & (u >= -0.5) & (u < W - 0.5) & (v >= -0.5) & (v < H - 0.5)
        m = np.minimum(np.minimum(u + 0.5, v + 0.5), np.minimum(W - 0.5 - u, H - 0.5 - v))
        imgs.append(img)
        wraws.append(np.where(valid, np.maximum(m, 0.0), 0.0))
    wsum = np.sum(wraws, axis=0)
    what = [np.where(wsum > 0, wr / np.where(wsum > 0, wsum, 1.0), 0.0) for wr in wraws]
    shapes = [g.shape for g in dense_ref.gaussian(np.zeros((Hc, Wc)), L)]
    N = [np.zeros(s + (3,)) for s in shapes]
    S = [np.zeros(s) for s in shapes]
    for img, wh in zip(imgs, what):
        gi, gw = dense_ref.gaussian(img, L), dense_ref.gaussian(wh, L)
        for l in range(L):
            lap = gi[l] - dense_ref.expand2d(gi[l + 1], shapes[l]) if l + 1 < L else gi[l]
            N[l] += gw[l][..., None] * lap
            S[l] += gw[l]
    B = [np.where((s > 1e-12)[..., None], n / np.where(s > 1e-12, s, 1.0)[..., None], 0.0) for n, s in zip(N, S)]
    R = B[L - 1]
    for l in range(L - 2, -1, -1):
        R = B[l] + dense_ref.expand2d(R, shapes[l])
    return np.where((wsum > 0)[..., None], np.clip(R, 0.0, 1.0), 0.0)


def test_full_path_matches_an_independent_numpy_formulation():
    """Three textured cameras (a translation, a rotation with perspective, a scaled view) blended on
    a small canvas with 3 levels: the oracle's output equals the NumPy formulation of S1-S6 to
    rounding level, blended overlaps included (pixels within 1e-6 px of a validity edge, where two
    FP64 evaluations of the position may disagree, are left out)."""
    cams, frames = _three_camera_rig()
    Wc, Hc, L = 44, 27, 3
    ref = oracle.forward(cams, frames, Wc, Hc, L)
    got = _numpy_forward(cams, frames, Wc, Hc, L)
    keep = ref["mindist"] >= 1e-6
    assert keep.mean() > 0.95
    np.testing.assert_allclose(ref["out"][keep], got[keep], atol=1e-12)
    # the rig has real overlaps: pixels where two or three cameras blend
    ys, xs = np.mgrid[0:Hc, 0:Wc]
    n_cov = sum(((lambda p: (p[2] > 0) & (p[0] / p[2] >= -0.5) & (p[0] / p[2] < c.width - 0.5) &
                  (p[1] / p[2] >= -0.5) & (p[1] / p[2] < c.height - 0.5))(
        np.tensordot(np.linalg.inv(np.asarray(c.H)), np.stack([xs, ys, np.ones_like(xs)]), 1))).astype(int)
        for c in cams)
    assert (n_cov >= 2).sum() > 50


def test_oracle_rejects_frames_that_do_not_match_the_cameras():
    """The oracle's wrappers refuse frame lists whose count or shapes differ from the cameras (the
    C code would read past them)."""
    cams = [Camera(8, 6, np.eye(3)), Camera(8, 6, _T(3, 0))]
    good = [_rand_frame(6, 8, 1), _rand_frame(6, 8, 2)]
    oracle.forward(cams, good, 12, 6, 2)
    with pytest.raises(ValueError, match="expected 2 frames"):
        oracle.forward(cams, good[:1], 12, 6, 2)
    with pytest.raises(ValueError, match="frame 1"):
        oracle.forward(cams, [good[0], good[1][:5]], 12, 6, 2)
    with pytest.raises(ValueError, match="frame 0"):
        oracle.warp(cams[0], good[0][:, :7], 12, 6)
    p = np.array([np.r_[np.eye(3).reshape(9)[:8], 1.0]] * 2)
    with pytest.raises(ValueError, match="expected 2 frames"):
        oracle.loss_grad([8, 8], [6, 6], p, good[:1], (0, 0, 12, 6))
    with pytest.raises(ValueError, match=r"\(H, W, 3\)"):
        oracle.lorb(good[0][..., 0], [(0, 0, 8, 6)], synth.brief_pattern(0))
