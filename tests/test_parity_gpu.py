"""GPU parity of the forward path (S1-S6) against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

import oracle
import synth
from synth import Camera
from tests import gpu_util

pytestmark = pytest.mark.gpu

PATHS = ["plain", "fused"]


def _T(tx, ty):
    return np.array([[1.0, 0, tx], [0, 1.0, ty], [0, 0, 1.0]])


def _rand(h, w, seed):
    return np.random.default_rng(seed).integers(0, 256, (h, w, 3), dtype=np.uint8)


@pytest.fixture(scope="module")
def cfg2():
    c = synth.config_2cam()
    return c, c.frame(0)


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("out_float", [True, False])
def test_2cam_full_canvas(cfg2, path, out_float):
    """Two 640x360 cameras -> 1100x400, 4 levels: every canvas pixel against the oracle."""
    cfg, frames = cfg2
    st = gpu_util.full_parity(cfg, frames, path, out_float)
    assert st["excluded"] < 1e-3 * cfg.canvas_w * cfg.canvas_h


@pytest.mark.parametrize("path", PATHS)
def test_4x1080p_scaled(path):
    """The 4-camera 25-degree rig at 1/4 scale (480x270 -> 1301x325, 5 levels), two frames."""
    cfg = synth.config_4x1080p(scale=0.25, frames=2)
    for t in (0, 1):
        gpu_util.full_parity(cfg, cfg.frame(t), path, True)
    gpu_util.full_parity(cfg, cfg.frame(1), path, False)


@pytest.mark.parametrize("path", PATHS)
def test_8x4k_scaled(path):
    """The 8-camera 40-degree tangent-plane rig at 1/10 scale (384x216 -> 2401x261, 6 levels)."""
    cfg = synth.config_8x4k(scale=0.1, frames=1)
    gpu_util.full_parity(cfg, cfg.frame(0), path, True)


@pytest.mark.parametrize("path", PATHS)
def test_batch_rigs_scaled(path):
    """A few of the uneven batch rigs (2-6 cameras, 4-6 levels) at 1/8 scale."""
    for cfg in synth.config_batch(n_rigs=4, seed=3, scale=0.125):
        gpu_util.full_parity(cfg, cfg.frame(0), path, True)


# ---------------------------------------------------------------------------------------------
# method invariants on the GPU


@pytest.mark.parametrize("path", PATHS)
def test_identity_reproduces_input(path):
    for (h, w, L) in [(23, 37, 3), (64, 96, 5), (1, 1, 1), (2, 3, 2), (300, 257, 6)]:
        fr = _rand(h, w, h + w)
        cfg = synth.RigConfig("id", [Camera(w, h, np.eye(3))], w, h, L, 1, None)
        got = gpu_util.run_gpu(cfg, [fr], path, out_float=False)
        assert np.array_equal(got, fr), (h, w, L)
        gotf = gpu_util.run_gpu(cfg, [fr], path, out_float=True)
        assert np.abs(gotf - fr / 255.0).max() <= 1e-6


@pytest.mark.parametrize("path", PATHS)
def test_integer_translation_exact(path):
    fr = _rand(80, 120, 7)
    cfg = synth.RigConfig("t", [Camera(120, 80, _T(-9, -4))], 101, 67, 4, 1, None)
    got = gpu_util.run_gpu(cfg, [fr], path, out_float=False)
    assert np.array_equal(got, fr[4:71, 9:110])


@pytest.mark.parametrize("path", PATHS)
def test_constant_frames_blend_to_constant(path):
    cfg = synth.config_2cam(scale=0.3)
    frames = [np.full((c.height, c.width, 3), (11, 128, 250), np.uint8) for c in cfg.cameras]
    ref = oracle.forward(cfg.cameras, frames, cfg.canvas_w, cfg.canvas_h, cfg.levels)
    got = gpu_util.run_gpu(cfg, frames, path, out_float=False)
    cov = ref["out"].sum(axis=2) > 0
    assert np.all(got[cov] == np.array([11, 128, 250], np.uint8))
    assert np.all(got[~cov] == 0)


@pytest.mark.parametrize("path", PATHS)
def test_gain_and_clamp(path):
    cfg = synth.config_2cam(scale=0.2)
    for c, g in zip(cfg.cameras, (1.7, 0.6)):
        c.gain = g
    frames = cfg.frame(0)
    gpu_util.full_parity(cfg, frames, path, True)


# ---------------------------------------------------------------------------------------------
# edge cases


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("Wc,Hc,L", [(1, 1, 1), (1, 1, 4), (2, 3, 3), (5, 7, 4), (33, 17, 6), (130, 9, 5)])
def test_tiny_and_ragged_canvases(path, Wc, Hc, L):
    cams = [Camera(9, 6, _T(-1.25, 0.5)), Camera(7, 8, _T(Wc / 2.0, -0.3))]
    frames = [_rand(6, 9, 1), _rand(8, 7, 2)]
    cfg = synth.RigConfig("tiny", cams, Wc, Hc, L, 1, None)
    gpu_util.full_parity(cfg, frames, path, True)


@pytest.mark.parametrize("path", PATHS)
def test_single_level_is_feather_blend(path):
    cfg = synth.config_2cam(scale=0.25)
    gpu_util.full_parity(cfg, cfg.frame(0), path, True, levels=1)


@pytest.mark.parametrize("path", PATHS)
def test_invisible_camera_is_ignored(path):
    cfg = synth.config_2cam(scale=0.25)
    frames = cfg.frame(0)
    off = Camera(50, 40, _T(10000, 10000))
    cfg.cameras.append(off)
    frames.append(_rand(40, 50, 3))
    gpu_util.full_parity(cfg, frames, path, True)


@pytest.mark.parametrize("path", PATHS)
def test_many_cameras(path):
    """12 small overlapping cameras in a grid (more cameras per pixel than any workload)."""
    cams, frames = [], []
    k = 0
    for gy in range(3):
        for gx in range(4):
            cams.append(Camera(40, 30, _T(gx * 25.3, gy * 18.7)))
            frames.append(_rand(30, 40, 100 + k))
            k += 1
    cfg = synth.RigConfig("grid", cams, 120, 70, 4, 1, None)
    gpu_util.full_parity(cfg, frames, path, True)


def test_bad_geometry_is_rejected():
    from paper_1810_03988_gb300 import Rig, StitchError, stitch
    sing = np.array([[1.0, 2, 3], [2, 4, 6], [0, 0, 1]])
    with pytest.raises(StitchError) as e:
        Rig([Camera(10, 10, sing)], 20, 20, 3)
    assert e.value.status == stitch.STITCH_EINVAL
    behind = np.array([[1.0, 0, 0], [0, 1, 0], [-0.2, 0, 1]])  # w <= 0 inside the image
    with pytest.raises(StitchError) as e:
        Rig([Camera(10, 10, behind)], 20, 20, 3)
    assert e.value.status == stitch.STITCH_EINVAL


def test_profiling_counts_every_launch():
    import torch
    from paper_1810_03988_gb300 import Rig
    cfg = synth.config_2cam(scale=0.25)
    dev = gpu_util.gpu_frames(cfg.frame(0))
    for path in PATHS:
        with Rig(cfg.cameras, cfg.canvas_w, cfg.canvas_h, cfg.levels, path=path) as rig:
            rig.set_profiling(True)
            for _ in range(3):
                rig.stitch(dev)
            t = rig.kernel_times()
            torch.cuda.synchronize()
            assert sum(n for _, n in t.values()) == 3 * rig.info()["num_kernels"]
            assert all(ms > 0 for ms, _ in t.values())


@pytest.mark.parametrize("path", PATHS)
def test_host_buffer_entry_point(path):
    import torch
    from paper_1810_03988_gb300 import Rig
    cfg = synth.config_2cam(scale=0.3)
    frames = cfg.frame(0)
    with Rig(cfg.cameras, cfg.canvas_w, cfg.canvas_h, cfg.levels, path=path) as rig:
        host = rig.stitch_host(frames)
        dev = rig.stitch(gpu_util.gpu_frames(frames)).cpu().numpy()
        torch.cuda.synchronize()
    assert np.array_equal(host, dev)


@pytest.mark.parametrize("path,out_float", [("fused", False), ("fused", True), ("plain", False)])
def test_host_async_pipeline(path, out_float):
    """Six overlapped host-buffer calls on different frames (pinned inputs, distinct pinned
    outputs, one synchronisation at the end) give the same canvases as device-buffer calls."""
    import torch
    from paper_1810_03988_gb300 import Rig
    cfg = synth.config_4x1080p(scale=0.2, frames=6)
    fr = [cfg.frame(t) for t in range(6)]
    pinned = [[torch.from_numpy(f).pin_memory() for f in fs] for fs in fr]
    dt = torch.float32 if out_float else torch.uint8
    outs = [torch.full((cfg.canvas_h, cfg.canvas_w, 3), 7, dtype=dt).pin_memory() for _ in fr]
    with Rig(cfg.cameras, cfg.canvas_w, cfg.canvas_h, cfg.levels, path=path, out_float=out_float) as rig:
        ref = [rig.stitch(gpu_util.gpu_frames(fs)).cpu().numpy() for fs in fr]
        for fs, o in zip(pinned, outs):
            rig.stitch_host_async(fs, o)
        torch.cuda.current_stream().synchronize()
        for o, r in zip(outs, ref):
            assert np.array_equal(o.numpy(), r)
        # a second round on the same rig reuses the staging slots
        for fs, o in zip(pinned[::-1], outs):
            rig.stitch_host_async(fs, o)
        torch.cuda.synchronize()
        for o, r in zip(outs, ref[::-1]):
            assert np.array_equal(o.numpy(), r)


# ---------------------------------------------------------------------------------------------
# full-size configurations, sampled windows (the oracle evaluates each window exactly)


@pytest.mark.parametrize("path", PATHS)
def test_4x1080p_full_size_windows(path):
    cfg = synth.config_4x1080p(frames=1)
    frames = cfg.frame(0)
    got = gpu_util.run_gpu(cfg, frames, path, out_float=True)
    for (x0, y0, w, h) in gpu_util.sample_windows(cfg, 12, 40):
        ref = oracle.forward(cfg.cameras, frames, cfg.canvas_w, cfg.canvas_h, cfg.levels, window=(x0, y0, w, h))
        gpu_util.compare(got[y0:y0 + h, x0:x0 + w], ref, True)


@pytest.mark.parametrize("path", PATHS)
def test_8x4k_full_size_windows(path):
    cfg = synth.config_8x4k(frames=1)
    frames = cfg.frame(0)
    got = gpu_util.run_gpu(cfg, frames, path, out_float=False)
    for (x0, y0, w, h) in gpu_util.sample_windows(cfg, 26, 32):
        ref = oracle.forward(cfg.cameras, frames, cfg.canvas_w, cfg.canvas_h, cfg.levels, window=(x0, y0, w, h))
        gpu_util.compare(got[y0:y0 + h, x0:x0 + w], ref, False)


def test_tile_classes_are_exercised():
    """The full-canvas parity cases above cover every class of canvas tile of the fused path."""
    from paper_1810_03988_gb300 import Rig
    cfg = synth.config_2cam()
    with Rig(cfg.cameras, cfg.canvas_w, cfg.canvas_h, cfg.levels) as rig:
        t = rig.info()["tiles"]
    assert t["zero"] > 0 and t["solo"] > 0 and t["full2"] > 0, t
    cams = [Camera(40, 30, _T(gx * 25.3, gy * 18.7)) for gy in range(3) for gx in range(4)]
    with Rig(cams, 120, 70, 4) as rig:
        t = rig.info()["tiles"]
    assert t["full4"] + t["general"] > 0 and t["general"] > 0, t
    cfg = synth.config_8x4k(frames=1)
    with Rig(cfg.cameras, cfg.canvas_w, cfg.canvas_h, cfg.levels) as rig:
        t = rig.info()["tiles"]
    assert t["solo"] > 0 and t["full2"] > 0, t


def test_down1_staged_and_unstaged_tiles():
    """down1 stages a tile's source footprint in shared memory when it fits; a camera whose source
    pixels are 2.5x denser than the canvas has footprints beyond the capacity and takes the
    unstaged path.  One rig holds both kinds of tile; the canvas matches the oracle."""
    from paper_1810_03988_gb300 import Rig
    S = lambda s, tx, ty: np.array([[s, 0, tx], [0, s, ty], [0, 0, 1.0]])
    cams = [Camera(400, 240, S(0.4, 10.3, 8.7)), Camera(400, 240, S(0.9, 150.2, 5.1))]
    cfg = synth.RigConfig("mixed_density", cams, 520, 230, 4, 1, None)
    rng = np.random.default_rng(11)
    frames = [rng.integers(0, 256, (240, 400, 3), dtype=np.uint8) for _ in cams]
    with Rig(cfg.cameras, cfg.canvas_w, cfg.canvas_h, cfg.levels) as rig:
        t = rig.info()["tiles"]
    assert 0 < t["down1_staged"] < t["down1"], t
    ref = oracle.forward(cfg.cameras, frames, cfg.canvas_w, cfg.canvas_h, cfg.levels)
    for out_float in (True, False):
        gpu_util.compare(gpu_util.run_gpu(cfg, frames, "fused", out_float), ref, out_float)
    # at least 99 % of the 8x4K rig's tiles are staged (it takes the smaller footprint capacity,
    # whose few larger footprints read from the frame)
    cfg = synth.config_8x4k(frames=1)
    with Rig(cfg.cameras, cfg.canvas_w, cfg.canvas_h, cfg.levels) as rig:
        t = rig.info()["tiles"]
    assert t["down1_staged"] >= 0.99 * t["down1"] and t["down1_interior"] > 0, t


@pytest.mark.parametrize("cfg_name", ["2cam", "4x1080p_scaled", "8x4k_scaled"])
def test_fp16_bands(cfg_name):
    """Pyramid data stored in FP16 between kernels (all arithmetic FP32): within 1e-3 of the oracle
    on the float canvas and 1 LSB on uint8."""
    cfg = {"2cam": lambda: synth.config_2cam(),
           "4x1080p_scaled": lambda: synth.config_4x1080p(scale=0.25, frames=1),
           "8x4k_scaled": lambda: synth.config_8x4k(scale=0.1, frames=1)}[cfg_name]()
    frames = cfg.frame(0)
    gpu_util.full_parity(cfg, frames, "fused", True, band_fp16=True, tol=gpu_util.TOL_F16)
    gpu_util.full_parity(cfg, frames, "fused", False, band_fp16=True)


def test_fp16_bands_8x4k_full_size_windows():
    cfg = synth.config_8x4k(frames=1)
    frames = cfg.frame(0)
    got = gpu_util.run_gpu(cfg, frames, "fused", out_float=True, band_fp16=True)
    for (x0, y0, w, h) in gpu_util.sample_windows(cfg, 20, 32):
        ref = oracle.forward(cfg.cameras, frames, cfg.canvas_w, cfg.canvas_h, cfg.levels, window=(x0, y0, w, h))
        gpu_util.compare(got[y0:y0 + h, x0:x0 + w], ref, True, tol=gpu_util.TOL_F16)


def _max_rig():
    """32 cameras (the ABI's maximum) in an 8 x 4 grid of overlapping 160 x 120 views with small
    rotations and a perspective term, on a 1140 x 420 canvas with 12 levels (the maximum: the
    level sizes run 1140, 570, ..., 2, 1)."""
    from paper_1810_03988_gb300 import stitch
    cams, frames = [], []
    rng = np.random.default_rng(11)
    for gy in range(4):
        for gx in range(8):
            a = rng.uniform(-0.05, 0.05)
            H = np.array([[np.cos(a), -np.sin(a), 10.0 + gx * 140.0 + rng.uniform(-3, 3)],
                          [np.sin(a), np.cos(a), 8.0 + gy * 100.0 + rng.uniform(-3, 3)],
                          [rng.uniform(-2e-5, 2e-5), rng.uniform(-2e-5, 2e-5), 1.0]])
            cams.append(Camera(160, 120, H))
            frames.append(_rand(120, 160, 500 + len(frames)))
    assert len(cams) == stitch.STITCH_MAX_CAMERAS
    return synth.RigConfig("max", cams, 1140, 420, stitch.STITCH_MAX_LEVELS, 1, None), frames


@pytest.mark.parametrize("path", PATHS)
def test_abi_maxima_full_canvas(path):
    """32 cameras and 12 pyramid levels: every canvas pixel against the oracle, float and uint8."""
    cfg, frames = _max_rig()
    ref = oracle.forward(cfg.cameras, frames, cfg.canvas_w, cfg.canvas_h, cfg.levels)
    for out_float in (True, False):
        got = gpu_util.run_gpu(cfg, frames, path, out_float=out_float)
        gpu_util.compare(got, ref, out_float)
