"""Host-side logic of the package that runs without a GPU."""
import numpy as np
import pytest

import oracle
import synth


def test_dlt_corner_parametrisation_roundtrip():
    """The refinement's corner parametrisation reproduces a camera's homography and its inverse."""
    torch = pytest.importorskip("torch")
    from paper_1810_03988_gb300.autograd import corners_of, homography_from_corners, image_corners, params_from_corners
    cfg = synth.config_refine(scale=0.25)
    for c in cfg.cameras:
        cr = torch.tensor(corners_of(c.H, c.width, c.height))
        H = homography_from_corners(image_corners(c.width, c.height), cr).numpy()
        np.testing.assert_allclose(H, c.H / c.H[2, 2], rtol=1e-9, atol=1e-9)
        A = oracle.invert_h(c.H)
        p = params_from_corners(cr[None], torch.ones(1, dtype=torch.float64), [(c.width, c.height)],
                                [A[2, 2]]).numpy()[0]
        np.testing.assert_allclose(p[:8], A.reshape(9)[:8], rtol=1e-8, atol=1e-10)


def test_binding_checks_host_images_before_the_library_sees_them():
    """The binding hands the library only images whose shape, element size and pixel packing match
    the buffer it will read or write: anything else raises ValueError on the host."""
    torch = pytest.importorskip("torch")
    from paper_1810_03988_gb300.stitch import _frame_args, _image_args
    cams = synth.config_2cam(scale=0.1).cameras
    frames = [np.zeros((c.height, c.width, 3), np.uint8) for c in cams]
    ptrs, pitches = _frame_args(frames, cams, None)
    assert pitches == [3 * c.width for c in cams] and ptrs == [f.ctypes.data for f in frames]
    # a padded view: the row pitch is the parent's, the pointer the view's first pixel
    c = cams[0]
    big = torch.zeros((c.height, c.width + 3, 3), dtype=torch.uint8)
    view = big[:, 1:1 + c.width]
    assert _image_args(view, c.height, c.width, 1, None, "v") == (view.data_ptr(), 3 * (c.width + 3))
    # a float canvas: pitch in bytes
    canvas = np.zeros((7, 11, 3), np.float32)
    assert _image_args(canvas, 7, 11, 4, None, "c") == (canvas.ctypes.data, 11 * 12)
    bad = [
        (frames[:1], "expected 2 frames"),                                            # a frame missing
        (frames + frames[:1], "expected 2 frames"),                                   # one too many
        ([frames[0][:-1], frames[1]], "expected shape"),                              # a row short
        ([frames[0].astype(np.uint16), frames[1]], "expected shape"),                 # 2-byte elements
        ([np.ascontiguousarray(frames[0].transpose(1, 0, 2)).transpose(1, 0, 2), frames[1]], "packed"),
        ([frames[0][::-1], frames[1]], "packed"),                                     # negative pitch
        ([torch.zeros((c.height, c.width, 3), dtype=torch.uint8).expand(c.height, c.width, 3)[:, :, :], frames[1]],
         None),                                                                       # a plain tensor is fine
        ([list(frames[0]), frames[1]], "expected a host tensor"),                     # not an array
    ]
    for fs, msg in bad:
        if msg is None:
            _frame_args(fs, cams, None)
            continue
        with pytest.raises(ValueError, match=msg):
            _frame_args(fs, cams, None)
    # a host frame where device frames are required
    with pytest.raises(ValueError, match="expected a tensor on cuda:0"):
        _frame_args([torch.from_numpy(f) for f in frames], cams, 0)
    with pytest.raises(ValueError, match="expected a CUDA tensor"):
        _frame_args(frames, cams, 0)
    # broadcast rows (stride 0) would make every row alias the first
    row = torch.zeros((1, c.width, 3), dtype=torch.uint8).expand(c.height, c.width, 3)
    with pytest.raises(ValueError, match="packed"):
        _image_args(row, c.height, c.width, 1, None, "r")


def test_bench_frame_percentiles():
    """Nearest-rank percentiles of the bench's per-frame times."""
    from bench import frame_percentiles
    assert frame_percentiles([]) == {}
    r = frame_percentiles([float(v) for v in range(1, 11)])  # 1 .. 10 ms
    assert (r["p10"], r["median"], r["p90"], r["frames"]) == (1.0, 5.5, 9.0, 10)
    r = frame_percentiles([3.0])
    assert r["p10"] == r["median"] == r["p90"] == 3.0
    r = frame_percentiles([5.0, 1.0, 4.0, 2.0, 3.0])
    assert (r["p10"], r["median"], r["p90"]) == (1.0, 3.0, 5.0)


def test_bench_code_digest_ignores_comments_only(tmp_path):
    """The kernel-source digest that keys the committed DRAM traffic figure changes with the code,
    not with comments, layout or comment markers inside string literals."""
    from bench import code_digest, profiled_traffic
    base = 'int f(int x) {\n    return x + 1;  // one\n}\nconst char* s = "a // b /* c */";\n'
    variants = {
        "same": 'int f(int x) {\n    /* block\n comment */ return x + 1;\n}\n// trailing\nconst char* s = "a // b /* c */";\n',
        "layout": 'int f(int x) { return x + 1; }\n\n\nconst char* s = "a // b /* c */";',
        "code": 'int f(int x) {\n    return x + 2;  // one\n}\nconst char* s = "a // b /* c */";\n',
        "string": 'int f(int x) {\n    return x + 1;  // one\n}\nconst char* s = "a // b /* d */";\n',
    }
    p = tmp_path / "k.cu"
    p.write_text(base)
    d0 = code_digest(str(p))
    for name, text in variants.items():
        p.write_text(text)
        assert (code_digest(str(p)) == d0) == (name in ("same", "layout")), name
    # the committed traffic line parses: a figure while the code matches, a stale marker after
    n, src = profiled_traffic("fused_down1", "8x4k")
    assert src.startswith("profiles/down1_8x4k.md") and (n == 1362720304 or "stale" in src), src
