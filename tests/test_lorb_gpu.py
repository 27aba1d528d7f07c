"""L-ORB on the GPU against the integer oracle: keypoints, responses and descriptors bit-exact on
synthetic views (several detection areas, thresholds and point counts), the full 4K view, the
corner image, empty areas and an out-of-range pattern."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _gpu(frame, areas, pattern, fast_t, harris_t, max_points, ctx=None):
    import torch
    from paper_1810_03988_gb300 import LORB
    H, W = frame.shape[:2]
    own = ctx is None
    ctx = ctx or LORB(W, H, max(max_points, 1))
    xy, resp, desc, cnt = ctx.detect(torch.from_numpy(frame).cuda(), areas, pattern, fast_t, harris_t, max_points)
    torch.cuda.synchronize()
    n = int(cnt.cpu()[0])
    out = xy[:n].cpu().numpy(), resp[:n].cpu().numpy(), desc[:n].cpu().numpy()
    if own:
        ctx.close()
    return out


def _check(frame, areas, pattern, fast_t=20, harris_t=0, max_points=500, ctx=None):
    ref = oracle.lorb(frame, areas, pattern, fast_t, harris_t, max_points)
    xy, resp, desc = _gpu(frame, areas, pattern, fast_t, harris_t, max_points, ctx)
    np.testing.assert_array_equal(xy, ref["xy"])
    np.testing.assert_array_equal(resp, ref["resp"])
    np.testing.assert_array_equal(desc, ref["desc"])
    return len(xy)


@pytest.mark.parametrize("fast_t,harris_t,max_points", [(20, 0, 500), (10, 10 ** 12, 2048), (40, 0, 37), (20, 0, 0)])
def test_lorb_matches_oracle(fast_t, harris_t, max_points):
    cfg = synth.config_4x1080p(scale=0.5, frames=1)
    frames = cfg.frame(0)
    pat = synth.brief_pattern(1)
    H, W = frames[0].shape[:2]
    areas = [(0, 0, W // 3, H), (2 * W // 3, 0, W, H), (W // 4, H // 3, W // 2, H // 2)]
    n = sum(_check(f, areas, pat, fast_t, harris_t, max_points) for f in frames[:2])
    assert max_points == 0 or n > 0


def test_lorb_full_4k_view_and_reuse():
    from paper_1810_03988_gb300 import LORB
    cfg = synth.config_8x4k(frames=1)
    frames = cfg.frame(0)
    pat = synth.brief_pattern(2)
    H, W = frames[0].shape[:2]
    with LORB(W, H, 1000) as ctx:
        for f in frames[:2]:
            assert _check(f, [(0, 0, W, H)], pat, 20, 0, 1000, ctx) == 1000
        # overlap strips only (the detection areas of Algorithm 2)
        _check(frames[2], [(0, 0, 600, H), (W - 600, 0, W, H)], pat, 25, 0, 800, ctx)


def test_lorb_corner_image_and_empty_areas():
    img = np.full((96, 120, 3), 30, np.uint8)
    img[35:60, 40:75] = 220
    pat = synth.brief_pattern(0)
    assert _check(img, [(0, 0, 120, 96)], pat, 20, 0, 10) == 4
    assert _check(img, [], pat, 20, 0, 10) == 0
    assert _check(img, [(0, 0, 10, 10)], pat, 20, 0, 10) == 0


def test_lorb_rejects_bad_arguments():
    import torch
    from paper_1810_03988_gb300 import LORB, StitchError, stitch
    img = torch.zeros((64, 64, 3), dtype=torch.uint8, device="cuda")
    pat = synth.brief_pattern(0).copy()
    with LORB(64, 64, 16) as ctx:
        pat[0, 0] = 16
        with pytest.raises(StitchError) as e:
            ctx.detect(img, [(0, 0, 64, 64)], pat)
        assert e.value.status == stitch.STITCH_EINVAL
        with pytest.raises(StitchError):
            ctx.detect(img, [(0, 0, 64, 64)], synth.brief_pattern(0), max_points=17)
    with pytest.raises(StitchError):
        LORB(20, 64, 16)
