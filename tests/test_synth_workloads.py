"""The seeded synthetic workloads that stand in for the paper's videos: their shapes, rig geometry
and determinism (CPU only).  The generator holds no stitching arithmetic; these checks keep the
benchmarked and tested workloads at the sizes they are quoted with."""
import numpy as np
import pytest

import synth


def _footprint_x(cam):
    """Canvas x-range of a planar camera's image rectangle (corners through camera->canvas H)."""
    W, H = cam.width, cam.height
    c = np.array([[-0.5, -0.5, 1], [W - 0.5, -0.5, 1], [W - 0.5, H - 0.5, 1], [-0.5, H - 0.5, 1]]).T
    p = np.asarray(cam.H) @ c
    assert (p[2] > 0).all()
    x = p[0] / p[2]
    return x.min(), x.max()


@pytest.mark.parametrize("make,n,size,canvas,levels,frames", [
    (lambda: synth.config_2cam(), 2, (640, 360), (1100, 400), 4, 1),
    (lambda: synth.config_4x1080p(frames=60), 4, (1920, 1080), (5200, 1300), 5, 60),
    (lambda: synth.config_refine(), 4, (1920, 1080), (5200, 1300), 5, 1),
    (lambda: synth.config_8x4k(frames=30), 8, (3840, 2160), (24000, 2600), 6, 30),
    (lambda: synth.config_cyl(), 4, (1280, 720), (2528, 760), 5, 1),
])
def test_workload_shapes(make, n, size, canvas, levels, frames):
    cfg = make()
    assert len(cfg.cameras) == n
    assert all((c.width, c.height) == size for c in cfg.cameras)
    assert (cfg.canvas_w, cfg.canvas_h) == canvas and cfg.levels == levels and cfg.frames == frames


@pytest.mark.parametrize("make", [synth.config_2cam, synth.config_4x1080p, synth.config_8x4k])
def test_neighbouring_cameras_overlap_and_cover_the_canvas_width(make):
    cfg = make()
    spans = sorted(_footprint_x(c) for c in cfg.cameras)
    for (a0, a1), (b0, b1) in zip(spans, spans[1:]):
        assert b0 < a1, "neighbouring views must overlap"
    lo, hi = spans[0][0], spans[-1][1]
    if cfg.name == "8x4k":
        # 280 degrees of yaw at f = 4125 plus one view: the views tile the ~24000 px canvas
        assert lo <= 50 and hi >= cfg.canvas_w - 50
        # views 40 degrees apart: f * 40 deg between centres on average; the seeded +-2 degree
        # yaw of each tangent plane moves a centre by up to f tan(2 deg) ~ 144 px
        steps = np.diff([0.5 * (a + b) for a, b in spans])
        assert abs(steps.mean() - 4125 * np.radians(40.0)) < 0.02 * 4125 * np.radians(40.0)
        assert np.abs(steps - 4125 * np.radians(40.0)).max() < 2 * 2 * 4125 * np.tan(np.radians(2.0))


def test_batch_rigs_are_uneven_and_within_the_stated_ranges():
    rigs = synth.config_batch(16)
    assert len(rigs) == 16
    ncam = [len(r.cameras) for r in rigs]
    assert min(ncam) >= 2 and max(ncam) <= 6 and len(set(ncam)) > 1
    res = {(r.cameras[0].width, r.cameras[0].height) for r in rigs}
    assert res <= set(synth.RESOLUTIONS) and len(res) > 1
    assert all(len({(c.width, c.height) for c in r.cameras}) == 1 for r in rigs)
    assert all(4 <= r.levels <= 6 for r in rigs) and len({r.levels for r in rigs}) > 1
    assert all(20.0 <= r.extra["spacing"] <= 30.0 for r in rigs)


def test_frames_are_seeded_and_deterministic():
    a = synth.config_2cam(scale=0.2).frame(0)
    b = synth.config_2cam(scale=0.2).frame(0)
    c = synth.config_2cam(scale=0.2, seed=1).frame(0)
    for x, y, z in zip(a, b, c):
        assert x.dtype == np.uint8 and x.shape == y.shape and x.flags.c_contiguous
        assert np.array_equal(x, y) and not np.array_equal(x, z)
    # a sequence differs from frame to frame (the scene moves 3 px per frame)
    cfg = synth.config_4x1080p(scale=0.1, frames=3)
    assert not np.array_equal(cfg.frame(0)[0], cfg.frame(1)[0])


def test_registration_inputs():
    pat = synth.brief_pattern(0)
    assert pat.shape == (256, 4) and pat.dtype == np.int8 and np.abs(pat).max() <= 15
    assert np.array_equal(pat, synth.brief_pattern(0)) and not np.array_equal(pat, synth.brief_pattern(1))
    bits = synth.lsh_bits(0)
    assert bits.shape == (8, 16) and bits.dtype == np.uint8
    assert all(len(set(row)) == 16 for row in bits)
    w = synth.prosac_words(0, 100)
    assert w.shape == (100, 4) and w.dtype == np.uint32 and w.max() > 2 ** 31
