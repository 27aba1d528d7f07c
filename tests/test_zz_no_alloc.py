"""stitch_frames_static: stitching with no device allocation (fixed static scratch array).

Some callers of this library cannot allocate device memory at all, for instance code running
inside a CUDA graph capture, real-time loops that cannot pay for the allocator's implicit
synchronisation, or hosts that hand the library a fixed memory budget.  stitch_frames_static
serves them with the plain-path kernels and a file-scope device array instead of rig buffers.
This file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

import synth
from tests import gpu_util

pytestmark = pytest.mark.gpu


def _static_call(lib, stitch, cfg, dev_frames, out, out_float):
    import torch
    desc, keep = stitch.make_desc(cfg.cameras, cfg.canvas_w, cfg.canvas_h, cfg.levels, out_float=out_float,
                                  path="plain")
    n = len(dev_frames)
    fp = (ctypes.c_void_p * n)(*[f.data_ptr() for f in dev_frames])
    pt = (ctypes.c_int64 * n)(*[f.stride(0) for f in dev_frames])
    st = lib.stitch_frames_static(ctypes.byref(desc), fp, pt, out.data_ptr(), out.stride(0) * out.element_size(),
                                  torch.cuda.current_stream().cuda_stream)
    del keep
    return st


@pytest.mark.parametrize("out_float", [False, True])
def test_static_entry_matches_stitch_frames_twice(out_float):
    """Two calls in a row through the C ABI give the existing entry point's result."""
    import torch
    from paper_1810_03988_gb300 import Rig, stitch
    lib = stitch.load()
    cfg = synth.config_2cam()
    frames = cfg.frame(0)
    dev = gpu_util.gpu_frames(frames)
    with Rig(cfg.cameras, cfg.canvas_w, cfg.canvas_h, cfg.levels, out_float=out_float, path="plain") as rig:
        ref = rig.stitch(dev).cpu().numpy()
    torch.cuda.synchronize()
    second = gpu_util.gpu_frames(synth.config_2cam(seed=5).frame(0))
    for call, frs in enumerate((dev, second, dev)):
        out = torch.full((cfg.canvas_h, cfg.canvas_w, 3), 7, dtype=torch.float32 if out_float else torch.uint8,
                         device="cuda")
        assert _static_call(lib, stitch, cfg, frs, out, out_float) == stitch.STITCH_OK
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        if call == 1:
            continue  # a different frame set in between, so the array holds other contents
        if out_float:
            assert np.abs(got.astype(np.float64) - ref).max() <= gpu_util.TOL_F32
        else:
            assert np.abs(got.astype(np.int32) - ref.astype(np.int32)).max() <= 1


def test_static_entry_rejects_oversized_rigs():
    import torch
    from paper_1810_03988_gb300 import stitch
    lib = stitch.load()
    cfg = synth.config_4x1080p(frames=1)
    dev = gpu_util.gpu_frames([np.zeros((c.height, c.width, 3), np.uint8) for c in cfg.cameras])
    out = torch.empty((cfg.canvas_h, cfg.canvas_w, 3), dtype=torch.uint8, device="cuda")
    assert _static_call(lib, stitch, cfg, dev, out, False) == stitch.STITCH_ETOOLARGE
