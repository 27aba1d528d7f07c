"""Seam weights (binary owner masks of the multiresolution spline) on the GPU against the oracle:
full canvases on both paths, the 12-camera grid (GENERAL tiles), full-size 8x4K windows around
the seams, FP16 bands, and the batched launch."""
import numpy as np
import pytest

import oracle
import synth
from synth import Camera
from tests import gpu_util

pytestmark = pytest.mark.gpu


def _run(cfg, frames, path="fused", out_float=True, band_fp16=False):
    import torch
    from paper_1810_03988_gb300 import Rig
    with Rig(cfg.cameras, cfg.canvas_w, cfg.canvas_h, cfg.levels, band_fp16=band_fp16, out_float=out_float,
             path=path, weights="seam") as rig:
        out = rig.stitch(gpu_util.gpu_frames(frames))
        torch.cuda.synchronize()
        return out.cpu().numpy()


@pytest.mark.parametrize("path", ["fused", "plain"])
@pytest.mark.parametrize("cfg_name", ["2cam", "4x1080p_scaled"])
def test_seam_full_canvas(path, cfg_name):
    cfg = {"2cam": lambda: synth.config_2cam(),
           "4x1080p_scaled": lambda: synth.config_4x1080p(scale=0.25, frames=1)}[cfg_name]()
    frames = cfg.frame(0)
    ref = oracle.forward(cfg.cameras, frames, cfg.canvas_w, cfg.canvas_h, cfg.levels, weights="seam")
    for out_float in (True, False):
        gpu_util.compare(_run(cfg, frames, path, out_float), ref, out_float)
    # the seam blend differs from the feather blend
    feather = oracle.forward(cfg.cameras, frames, cfg.canvas_w, cfg.canvas_h, cfg.levels)
    assert np.abs(feather["out"] - ref["out"]).max() > 1e-2


def test_seam_general_tiles():
    """12 overlapping cameras: canvas tiles with more than four cameras (GENERAL) on the fused
    path, and the plain path."""
    T = lambda tx, ty: np.array([[1.0, 0, tx], [0, 1.0, ty], [0, 0, 1.0]])
    cams = [Camera(40, 30, T(gx * 25.3, gy * 18.7)) for gy in range(3) for gx in range(4)]
    cfg = synth.RigConfig("grid", cams, 120, 70, 4, 1, None)
    rng = np.random.default_rng(3)
    frames = [rng.integers(0, 256, (30, 40, 3), dtype=np.uint8) for _ in cams]
    ref = oracle.forward(cams, frames, 120, 70, 4, weights="seam")
    for path in ("fused", "plain"):
        gpu_util.compare(_run(cfg, frames, path, True), ref, True)


def test_seam_8x4k_full_size_windows():
    cfg = synth.config_8x4k(frames=1)
    frames = cfg.frame(0)
    got = _run(cfg, frames, "fused", True)
    for (x0, y0, w, h) in gpu_util.sample_windows(cfg, 14, 48):
        ref = oracle.forward(cfg.cameras, frames, cfg.canvas_w, cfg.canvas_h, cfg.levels, window=(x0, y0, w, h),
                             weights="seam")
        gpu_util.compare(got[y0:y0 + h, x0:x0 + w], ref, True)


def test_seam_fp16_bands():
    cfg = synth.config_4x1080p(scale=0.25, frames=1)
    frames = cfg.frame(0)
    ref = oracle.forward(cfg.cameras, frames, cfg.canvas_w, cfg.canvas_h, cfg.levels, weights="seam")
    gpu_util.compare(_run(cfg, frames, "fused", True, band_fp16=True), ref, True, gpu_util.TOL_F16)


def test_seam_batch_equals_per_rig():
    import torch
    from paper_1810_03988_gb300 import Batch, Rig
    cfgs = synth.config_batch(4, seed=3, scale=0.125)
    rigs = [Rig(c.cameras, c.canvas_w, c.canvas_h, c.levels, weights="seam") for c in cfgs]
    frames = [gpu_util.gpu_frames(c.frame(0)) for c in cfgs]
    ref = [r.stitch(f).cpu().numpy() for r, f in zip(rigs, frames)]
    with Batch(rigs) as b:
        got = [o.cpu().numpy() for o in b.stitch(frames)]
    torch.cuda.synchronize()
    for g, r in zip(got, ref):
        assert np.array_equal(g, r)
    for r in rigs:
        r.close()
