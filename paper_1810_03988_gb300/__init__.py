"""GB300 (sm_103a) per-frame panoramic stitching path behind a C ABI (libstitch).

The compute runs in hand-written CUDA kernels (``csrc/``); ``stitch`` is the ctypes binding of
``include/stitch.h`` (argument marshalling only).
"""
from .stitch import (STITCH_PATH_FUSED, STITCH_PATH_PLAIN, LORB, Batch, Matcher, Rig, StitchError, library_path, load,  # noqa: F401
                     status_string, stitch_backward, stitch_batch_create, stitch_batch_destroy,
                     stitch_batch_frames, stitch_frames, stitch_frames_host, stitch_frames_host_async, stitch_frames_static, stitch_rig_create, stitch_rig_destroy,
                     stitch_rig_get_camera, stitch_rig_get_info, stitch_rig_kernel_times, stitch_rig_set_profiling,
                     stitch_lorb_create, stitch_lorb_destroy, stitch_lorb_detect,
                     stitch_match_homography, stitch_matcher_create, stitch_matcher_destroy)

stitch_status_string = status_string
