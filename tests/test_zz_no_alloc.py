"""stitch_frames_static: stitching with no device allocation (fixed static scratch array).

Some callers of this library cannot allocate device memory at all: real-time loops that cannot
pay for the allocator's implicit synchronisation, hosts that hand the library a fixed memory
budget, or plugins whose host application owns every device allocation.  stitch_frames_static
serves them with the plain-path kernels and a file-scope device array instead of rig buffers.
It runs the same kernels in the same order as a STITCH_PATH_PLAIN rig, so its output must be
identical to that rig's stitch_frames, bit for bit, on every call.
This file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

import synth
from tests import gpu_util

pytestmark = pytest.mark.gpu


def _static_call(lib, stitch, cfg, dev_frames, out, out_float, weights="feather"):
    import torch
    desc, keep = stitch.make_desc(cfg.cameras, cfg.canvas_w, cfg.canvas_h, cfg.levels, out_float=out_float,
                                  path="plain", weights=weights, canvas=cfg.canvas)
    n = len(dev_frames)
    fp = (ctypes.c_void_p * n)(*[f.data_ptr() for f in dev_frames])
    pt = (ctypes.c_int64 * n)(*[f.stride(0) for f in dev_frames])
    st = lib.stitch_frames_static(ctypes.byref(desc), fp, pt, out.data_ptr(), out.stride(0) * out.element_size(),
                                  torch.cuda.current_stream().cuda_stream)
    del keep
    return st


def _check_twice(cfg, other_cfg, out_float, weights="feather"):
    """The rig's stitch_frames result, then the static entry on the same frames, on another frame
    set (so the array holds other contents) and on the same frames again: identical results."""
    import torch
    from paper_1810_03988_gb300 import Rig, stitch
    lib = stitch.load()
    dev = gpu_util.gpu_frames(cfg.frame(0))
    with Rig(cfg.cameras, cfg.canvas_w, cfg.canvas_h, cfg.levels, out_float=out_float, path="plain",
             weights=weights, canvas=cfg.canvas) as rig:
        ref = rig.stitch(dev).cpu().numpy()
    torch.cuda.synchronize()
    second = gpu_util.gpu_frames(other_cfg.frame(0))
    for call, frs in enumerate((dev, second, dev)):
        out = torch.full((cfg.canvas_h, cfg.canvas_w, 3), 7, dtype=torch.float32 if out_float else torch.uint8,
                         device="cuda")
        assert _static_call(lib, stitch, cfg, frs, out, out_float, weights) == stitch.STITCH_OK
        torch.cuda.synchronize()
        if call == 1:
            continue
        got = out.cpu().numpy()
        assert np.array_equal(got, ref), f"call {call}: max difference {np.abs(got.astype(np.float64) - ref).max()}"


@pytest.mark.parametrize("out_float", [False, True])
def test_static_entry_matches_stitch_frames_twice(out_float):
    """Two-camera planar rig with feather weights, uint8 and float output."""
    _check_twice(synth.config_2cam(), synth.config_2cam(seed=5), out_float)


def test_static_entry_seam_weights():
    """The same with the binary seam masks in place of feather weights."""
    _check_twice(synth.config_2cam(), synth.config_2cam(seed=5), True, weights="seam")


def test_static_entry_cylindrical_canvas():
    """The same on a cylindrical canvas (4 cameras at 0.3 scale)."""
    _check_twice(synth.config_cyl(scale=0.3), synth.config_cyl(scale=0.3, seed=5), False)


def test_static_entry_rejects_oversized_rigs():
    import torch
    from paper_1810_03988_gb300 import stitch
    lib = stitch.load()
    cfg = synth.config_4x1080p(frames=1)
    dev = gpu_util.gpu_frames([np.zeros((c.height, c.width, 3), np.uint8) for c in cfg.cameras])
    out = torch.empty((cfg.canvas_h, cfg.canvas_w, 3), dtype=torch.uint8, device="cuda")
    assert _static_call(lib, stitch, cfg, dev, out, False) == stitch.STITCH_ETOOLARGE
