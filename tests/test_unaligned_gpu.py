"""Frames whose base address and row pitch are not multiples of 4 bytes (views into padded
buffers): the stitch (fused and plain paths, both weight modes) and L-ORB take their byte-load
paths there and must give exactly what they give on aligned frames."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _views(frames, pad_left=1, pad_right=2):
    """Each frame as a view into a wider buffer: base 3 * pad_left bytes in, pitch
    3 * (W + pad_left + pad_right) bytes."""
    import torch
    out = []
    for f in frames:
        h, w, _ = f.shape
        buf = torch.zeros((h, w + pad_left + pad_right, 3), dtype=torch.uint8, device="cuda")
        buf[:, pad_left:pad_left + w] = torch.from_numpy(f).cuda()
        v = buf[:, pad_left:pad_left + w]
        assert v.data_ptr() % 4 != 0 and v.stride(0) % 4 != 0
        out.append(v)
    return out


@pytest.mark.parametrize("path,weights", [("fused", "feather"), ("fused", "seam"), ("plain", "feather")])
def test_stitch_on_unaligned_frames_equals_aligned(path, weights):
    import torch
    from paper_1810_03988_gb300 import Rig
    cfg = synth.config_4x1080p(scale=0.5, frames=1)
    frames = cfg.frame(0)
    aligned = [torch.from_numpy(f).cuda() for f in frames]
    with Rig(cfg.cameras, cfg.canvas_w, cfg.canvas_h, cfg.levels, path=path, weights=weights, out_float=True) as rig:
        a = rig.stitch(aligned).cpu().numpy()
        b = rig.stitch(_views(frames)).cpu().numpy()
    np.testing.assert_array_equal(a, b)


def test_lorb_on_unaligned_frame_matches_oracle():
    import torch
    from paper_1810_03988_gb300 import LORB
    cfg = synth.config_4x1080p(scale=0.5, frames=1)
    f = cfg.frame(0)[1]
    H, W = f.shape[:2]
    pat = synth.brief_pattern(4)
    areas = [(0, 0, W, H)]
    ref = oracle.lorb(f, areas, pat, 20, 0, 700)
    with LORB(W, H, 700) as ctx:
        xy, resp, desc, cnt = ctx.detect(_views([f])[0], areas, pat, 20, 0, 700)
        torch.cuda.synchronize()
        n = int(cnt.cpu()[0])
        np.testing.assert_array_equal(xy[:n].cpu().numpy(), ref["xy"])
        np.testing.assert_array_equal(resp[:n].cpu().numpy(), ref["resp"])
        np.testing.assert_array_equal(desc[:n].cpu().numpy(), ref["desc"])
