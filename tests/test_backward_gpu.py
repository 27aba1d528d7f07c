"""S7 on the GPU: loss and gradient against the FP64 oracle, finite differences through the
corner parametrisation, and gradient-based refinement of perturbed homographies."""
import numpy as np
import pytest

import oracle
import synth
from tests import gpu_util

pytestmark = pytest.mark.gpu


def _rig_and_params(cfg, rng=None, corner_noise=0.0, gain_range=None):
    import torch
    from paper_1810_03988_gb300 import Rig
    from paper_1810_03988_gb300.autograd import corners_of, params_from_corners
    rig = Rig(cfg.cameras, cfg.canvas_w, cfg.canvas_h, cfg.levels)
    n = len(cfg.cameras)
    signs = [float(rig.camera_map(i)[0][2, 2]) for i in range(n)]
    corners = np.stack([corners_of(c.H, c.width, c.height) for c in cfg.cameras])
    gains = np.ones(n)
    if rng is not None:
        corners[1:] += rng.uniform(-corner_noise, corner_noise, corners[1:].shape)
        if gain_range:
            gains[1:] = rng.uniform(*gain_range, n - 1)
    p = params_from_corners(torch.tensor(corners), torch.tensor(gains),
                            [(c.width, c.height) for c in cfg.cameras], signs).numpy()
    return rig, p, signs, corners, gains


def _px_scale(cfg):
    ext = float(max(cfg.canvas_w, cfg.canvas_h))
    return np.array([1 / ext, 1 / ext, 1, 1 / ext, 1 / ext, 1, 1 / ext ** 2, 1 / ext ** 2, 1.0])


def _compare(cfg, rig, params, signs, frames, tol_grad=1e-3, tol_loss=1e-4):
    import torch
    dev = gpu_util.gpu_frames(frames)
    pt = torch.tensor(params, device="cuda")
    loss, grad = rig.backward(dev, pt)
    torch.cuda.synchronize()
    loss = float(loss.cpu()[0])
    grad = grad.cpu().numpy()
    lo, go = oracle.loss_grad([c.width for c in cfg.cameras], [c.height for c in cfg.cameras], params, frames,
                              (0, 0, cfg.canvas_w, cfg.canvas_h), a33=signs)
    assert abs(loss - lo) <= tol_loss * lo, (loss, lo)
    s = _px_scale(cfg)
    worst = 0.0
    for i in range(len(cfg.cameras)):
        ref = np.abs(go[i] * s).max()
        err = np.abs((grad[i] - go[i]) * s).max() / ref
        worst = max(worst, err)
        assert err <= tol_grad, (i, err, grad[i], go[i])
    return loss, lo, worst


def test_backward_matches_oracle_scaled():
    cfg = synth.config_refine(scale=0.25)
    frames = cfg.frame(0)
    rig, p, signs, _, _ = _rig_and_params(cfg, np.random.default_rng(1), 1.0, (0.8, 1.2))
    with rig:
        _compare(cfg, rig, p, signs, frames)
        # at the true geometry the loss is the resampling floor and the gradient still matches
        _, p0, _, _, _ = _rig_and_params(cfg)
        _compare(cfg, rig, p0, signs, frames)


def test_backward_entrywise_against_oracle():
    """Entry by entry: every gradient entry whose pixel-scaled size is at least 1 % of its camera's
    largest is within 1e-3 of the oracle's value, relative to that entry (scaled rig, perturbed
    corners and gains, and the true geometry)."""
    import torch
    cfg = synth.config_refine(scale=0.25)
    frames = cfg.frame(0)
    dev = gpu_util.gpu_frames(frames)
    rig, p, signs, _, _ = _rig_and_params(cfg, np.random.default_rng(1), 1.0, (0.8, 1.2))
    _, p0, _, _, _ = _rig_and_params(cfg)
    s = _px_scale(cfg)
    with rig:
        for params in (p, p0):
            _, grad = rig.backward(dev, torch.tensor(params, device="cuda"))
            torch.cuda.synchronize()
            grad = grad.cpu().numpy()
            _, go = oracle.loss_grad([c.width for c in cfg.cameras], [c.height for c in cfg.cameras], params, frames,
                                     (0, 0, cfg.canvas_w, cfg.canvas_h), a33=signs)
            for i in range(len(cfg.cameras)):
                big = np.abs(go[i] * s) >= 0.01 * np.abs(go[i] * s).max()
                rel = np.abs(grad[i] - go[i])[big] / np.abs(go[i])[big]
                assert rel.max() <= 1e-3, (i, rel.max(), grad[i], go[i])


def test_backward_matches_oracle_full_size():
    """The 4-camera 1920x1080 refinement rig (canvas 5200x1300), perturbed corners and gains."""
    cfg = synth.config_refine()
    frames = cfg.frame(0)
    rig, p, signs, _, _ = _rig_and_params(cfg, np.random.default_rng(2), 3.0, (0.8, 1.2))
    with rig:
        _compare(cfg, rig, p, signs, frames)


def test_backward_other_geometries():
    """2-camera rig, a tangent-plane rig and the 12-camera grid (more than 4 cameras per tile)."""
    from synth import Camera
    for cfg in (synth.config_2cam(scale=0.5), synth.config_8x4k(scale=0.1, frames=1)):
        frames = cfg.frame(0)
        rig, p, signs, _, _ = _rig_and_params(cfg, np.random.default_rng(3), 0.5, (0.9, 1.1))
        with rig:
            _compare(cfg, rig, p, signs, frames)
    T = lambda tx, ty: np.array([[1.0, 0, tx], [0, 1.0, ty], [0, 0, 1.0]])
    # sub-pixel offsets keep every camera off integer source positions: there bilinear sampling
    # has a kink and the one-sided derivative depends on the last bit of the position
    cams = [Camera(40, 30, T(gx * 25.3 + 0.37, gy * 18.7 + 0.21)) for gy in range(3) for gx in range(4)]
    cfg = synth.RigConfig("grid", cams, 120, 70, 3, 1, None)
    rng = np.random.default_rng(4)
    frames = [rng.integers(0, 256, (30, 40, 3), dtype=np.uint8) for _ in cams]
    rig, p, signs, _, _ = _rig_and_params(cfg, np.random.default_rng(5), 0.3, (0.9, 1.1))
    with rig:
        _compare(cfg, rig, p, signs, frames)


def test_corner_gradient_central_differences():
    """Gradient with respect to the corner offsets (kernel + DLT chain rule) against central
    differences of the kernel's loss with eps = 1e-3 px.  Bilinear sampling has kinks at integer
    source coordinates, so the difference quotient differs from the one-sided derivative at the
    pixels whose coordinates cross one; the tolerance is relative to the gradient norm."""
    import torch
    from paper_1810_03988_gb300.autograd import StitchLoss, params_from_corners
    cfg = synth.config_refine(scale=0.25)
    frames = cfg.frame(0)
    rig, _, signs, corners, gains = _rig_and_params(cfg, np.random.default_rng(6), 2.0, (0.9, 1.1))
    dev = gpu_util.gpu_frames(frames)
    sizes = [(c.width, c.height) for c in cfg.cameras]
    with rig:
        def loss_of(cr):
            p = params_from_corners(torch.tensor(cr, device="cuda"), torch.tensor(gains, device="cuda"), sizes, signs)
            return float(StitchLoss.apply(p, rig, dev))
        c = torch.tensor(corners, device="cuda", requires_grad=True)
        p = params_from_corners(c, torch.tensor(gains, device="cuda"), sizes, signs)
        StitchLoss.apply(p, rig, dev).backward()
        g = c.grad.cpu().numpy()
        eps = 1e-3
        fd = np.zeros_like(g)
        for i in range(1, len(cfg.cameras)):
            for k in range(4):
                for d in range(2):
                    cp = corners.copy(); cp[i, k, d] += eps
                    cm = corners.copy(); cm[i, k, d] -= eps
                    fd[i, k, d] = (loss_of(cp) - loss_of(cm)) / (2 * eps)
    for i in range(1, len(cfg.cameras)):
        rel = np.abs(fd[i] - g[i]).max() / np.abs(g[i]).max()
        assert rel < 5e-2, (i, rel)


def test_refinement_reduces_loss_and_corner_error():
    """50 Adam steps through the hand-written backward from corners perturbed by +-3 px and gains in
    U[0.8, 1.2] (camera 0 fixed) reduce the overlap loss and the corner error."""
    from paper_1810_03988_gb300.autograd import corners_of, refine
    cfg = synth.config_refine()
    frames = cfg.frame(0)
    rng = np.random.default_rng(7)
    true = np.stack([corners_of(c.H, c.width, c.height) for c in cfg.cameras])
    start = true.copy()
    start[1:] += rng.uniform(-3, 3, start[1:].shape)
    gains = np.ones(len(cfg.cameras))
    gains[1:] = rng.uniform(0.8, 1.2, len(cfg.cameras) - 1)
    from paper_1810_03988_gb300 import Rig
    dev = gpu_util.gpu_frames(frames)
    with Rig(cfg.cameras, cfg.canvas_w, cfg.canvas_h, cfg.levels) as rig:
        corners, g, hist = refine(rig, dev, start, gains, steps=50)
    e0 = np.abs(start - true)[1:].mean()
    e1 = np.abs(corners - true)[1:].mean()
    assert hist[-1] < 0.5 * hist[0], (hist[0], hist[-1])
    assert e1 < e0, (e0, e1)
    assert np.abs(g[1:] - 1.0).mean() < np.abs(gains[1:] - 1.0).mean()
