"""C-ABI checks that need no GPU: the library loads, exports every declared symbol, and rejects
bad descriptors before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "stitch.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(stitch_[a-z_0-9]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1810_03988_gb300 import _build, stitch
    _build.build()
    return stitch.load()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for n in ["stitch_rig_create", "stitch_frames", "stitch_backward", "stitch_rig_destroy", "stitch_batch_create",
              "stitch_batch_frames", "stitch_batch_destroy", "stitch_status_string"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1810_03988_gb300 import stitch
    for n in _declared_functions():
        assert hasattr(lib, n), f"{n} declared in include/stitch.h but not exported"
        assert n in stitch.SIGNATURES, f"{n} has no binding signature"


def test_status_strings(lib):
    from paper_1810_03988_gb300 import stitch
    for s in range(7):
        assert stitch.status_string(s).startswith("STITCH_")


def test_create_rejects_bad_descriptors_without_a_device(lib):
    from paper_1810_03988_gb300 import stitch
    import synth
    cfg = synth.config_2cam(scale=0.1)
    out = ctypes.c_void_p()

    def create(**kw):
        desc, keep = stitch.make_desc(cfg.cameras, cfg.canvas_w, cfg.canvas_h, cfg.levels)
        for k, v in kw.items():
            setattr(desc, k, v)
        return lib.stitch_rig_create(ctypes.byref(desc), 0, ctypes.byref(out))

    assert create(num_cameras=0) == stitch.STITCH_EINVAL
    assert create(num_cameras=stitch.STITCH_MAX_CAMERAS + 1) == stitch.STITCH_EINVAL
    assert create(levels=0) == stitch.STITCH_EINVAL
    assert create(levels=stitch.STITCH_MAX_LEVELS + 1) == stitch.STITCH_EINVAL
    assert create(canvas_w=0) == stitch.STITCH_EINVAL
    assert create(out_float=2) == stitch.STITCH_EINVAL
    assert create(path=7) == stitch.STITCH_EINVAL
    assert create(weights=2) == stitch.STITCH_EINVAL
    assert lib.stitch_rig_create(None, 0, ctypes.byref(out)) == stitch.STITCH_EINVAL
    assert out.value is None
    # destroy is NULL-safe
    lib.stitch_rig_destroy(None)


def test_null_rig_calls_are_rejected(lib):
    from paper_1810_03988_gb300 import stitch
    assert lib.stitch_frames(None, None, None, None, 0, None) == stitch.STITCH_EINVAL
    assert lib.stitch_backward(None, None, None, None, None, None, None) == stitch.STITCH_EINVAL
    assert lib.stitch_rig_get_info(None, None) == stitch.STITCH_EINVAL
    assert lib.stitch_batch_frames(None, None, None, None, None, None) != stitch.STITCH_OK


def test_matcher_rejects_bad_arguments_without_a_device(lib):
    from paper_1810_03988_gb300 import stitch
    out = ctypes.c_void_p()
    assert lib.stitch_matcher_create(0, 16, 0, ctypes.byref(out)) == stitch.STITCH_EINVAL
    assert lib.stitch_matcher_create(4096, 16, 0, ctypes.byref(out)) == stitch.STITCH_EINVAL
    assert lib.stitch_matcher_create(100, -1, 0, ctypes.byref(out)) == stitch.STITCH_EINVAL
    assert lib.stitch_matcher_create(100, 16, 0, None) == stitch.STITCH_EINVAL
    prm = stitch.stitch_match_params(8, 16, 80, 4, 5, 0, 3.0)
    assert lib.stitch_match_homography(None, None, None, None, None, None, None, ctypes.byref(prm), None, None, None,
                                       None, None, None, None, None) == stitch.STITCH_EINVAL
    lib.stitch_matcher_destroy(None)


def test_remaining_entry_points_reject_bad_arguments_without_a_device(lib):
    """Every other entry point validates its handles and sizes before it touches the device."""
    from paper_1810_03988_gb300 import stitch
    import synth
    E = stitch.STITCH_EINVAL
    out = ctypes.c_void_p()
    buf = (ctypes.c_uint8 * 64)()
    pit = (ctypes.c_int64 * 4)(3, 3, 3, 3)
    # frames through host buffers
    assert lib.stitch_frames_host(None, buf, pit, buf, 64, None) == E
    assert lib.stitch_frames_host_async(None, buf, pit, buf, 64, None) == E
    # per-call scratch path: the descriptor is checked first
    cfg = synth.config_2cam(scale=0.1)
    for field, bad in (("num_cameras", 0), ("levels", 0), ("canvas_h", 0), ("out_float", 3), ("band_fp16", 1)):
        desc, keep = stitch.make_desc(cfg.cameras, cfg.canvas_w, cfg.canvas_h, cfg.levels)
        setattr(desc, field, bad)
        assert lib.stitch_frames_static(ctypes.byref(desc), buf, pit, buf, 64, None) == E, field
    assert lib.stitch_frames_static(None, buf, pit, buf, 64, None) == E
    # cylindrical canvas: focal length, centre must be finite (and the focal length positive)
    for k, bad in ((0, float("inf")), (0, float("nan")), (0, -1.0), (1, float("nan")), (2, float("-inf"))):
        cyl = [1000.0, 50.0, 20.0]
        cyl[k] = bad
        desc, keep = stitch.make_desc(cfg.cameras, cfg.canvas_w, cfg.canvas_h, cfg.levels, canvas=cyl)
        assert lib.stitch_frames_static(ctypes.byref(desc), buf, pit, buf, 64, None) == E, (k, bad)
        assert lib.stitch_rig_create(ctypes.byref(desc), 0, ctypes.byref(out)) == E and out.value is None, (k, bad)
    # rig queries and profiling
    a = (ctypes.c_double * 9)()
    vis = ctypes.c_int32()
    cnt = ctypes.c_int32()
    assert lib.stitch_rig_get_camera(None, 0, a, ctypes.byref(vis)) == E
    assert lib.stitch_rig_set_profiling(None, 1) == E
    assert lib.stitch_rig_kernel_times(None, None, None, None, 0, ctypes.byref(cnt)) == E
    # batches
    assert lib.stitch_batch_create(None, 1, ctypes.byref(out)) == E
    assert lib.stitch_batch_create(None, 1, None) == E
    rigs = (ctypes.c_void_p * 2)(None, None)
    assert lib.stitch_batch_create(rigs, 2, ctypes.byref(out)) == E and out.value is None
    assert lib.stitch_batch_get_schedule(None, None, None, None) == E
    assert lib.stitch_batch_wait_test(None, 10, 0) == E
    assert lib.stitch_batch_sync(None) == E
    assert lib.stitch_rig_debug_check(None, None, None) == E
    lib.stitch_batch_destroy(None)
    # L-ORB: sizes below the 37-pixel minimum, point limits, missing outputs
    assert lib.stitch_lorb_create(36, 100, 100, 0, ctypes.byref(out)) == E
    assert lib.stitch_lorb_create(100, 36, 100, 0, ctypes.byref(out)) == E
    assert lib.stitch_lorb_create(100, 100, 0, 0, ctypes.byref(out)) == E
    assert lib.stitch_lorb_create(100, 100, 2049, 0, ctypes.byref(out)) == E
    assert lib.stitch_lorb_create(100, 100, 100, 0, None) == E
    prm = stitch.stitch_lorb_params(20, 0, 100)
    assert lib.stitch_lorb_detect(None, buf, 8, 8, 24, None, 0, ctypes.byref(prm), buf, buf, buf, buf, buf,
                                  None) == E
    lib.stitch_lorb_destroy(None)
