"""Thin ctypes binding of libstitch (include/stitch.h).

Argument marshalling only: every step of the stitching path runs in the library's CUDA kernels.
PyTorch supplies device memory and the current CUDA stream.  The functions named like the C ABI
(``stitch_rig_create`` ...) take plain integers/pointers; :class:`Rig` wraps them for torch tensors.
There is no CPU fallback: if the library is missing or the GPU is unavailable the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

STITCH_OK, STITCH_EINVAL, STITCH_ENOMEM, STITCH_ECUDA, STITCH_ETIMEOUT, STITCH_EUNSUPPORTED, STITCH_ETOOLARGE = range(7)
STITCH_STATIC_SCRATCH_BYTES = 64 * 1024 * 1024
STITCH_MAX_CAMERAS = 32
STITCH_MAX_LEVELS = 12
STITCH_PATH_FUSED = 0
STITCH_PATH_PLAIN = 1
STITCH_WEIGHTS_FEATHER = 0
STITCH_WEIGHTS_SEAM = 1
STITCH_CANVAS_PLANAR = 0
STITCH_CANVAS_CYLINDRICAL = 1

_P = ctypes.c_void_p
_lock = threading.Lock()
_lib = None


class stitch_camera(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("H", ctypes.c_double * 9),
                ("gain", ctypes.c_float)]


class stitch_rig_desc(ctypes.Structure):
    _fields_ = [("num_cameras", ctypes.c_int32), ("cameras", ctypes.POINTER(stitch_camera)),
                ("canvas_w", ctypes.c_int32), ("canvas_h", ctypes.c_int32), ("levels", ctypes.c_int32),
                ("band_fp16", ctypes.c_int32), ("out_float", ctypes.c_int32), ("path", ctypes.c_int32),
                ("weights", ctypes.c_int32), ("canvas_model", ctypes.c_int32),
                ("cylinder", ctypes.c_double * 3)]


class stitch_lorb_params(ctypes.Structure):
    _fields_ = [("fast_t", ctypes.c_int32), ("harris_t", ctypes.c_int64), ("max_points", ctypes.c_int32)]


class stitch_match_params(ctypes.Structure):
    _fields_ = [("tables", ctypes.c_int32), ("bits", ctypes.c_int32), ("max_dist", ctypes.c_int32),
                ("ratio_num", ctypes.c_int32), ("ratio_den", ctypes.c_int32), ("iters", ctypes.c_int32),
                ("inlier_px", ctypes.c_double)]


class stitch_rig_info(ctypes.Structure):
    _fields_ = [("scratch_bytes", ctypes.c_int64), ("num_kernels", ctypes.c_int32), ("path", ctypes.c_int32),
                ("roi_pixels", ctypes.c_int64), ("tiles_zero", ctypes.c_int32), ("tiles_solo", ctypes.c_int32),
                ("tiles_full2", ctypes.c_int32), ("tiles_full4", ctypes.c_int32),
                ("tiles_general", ctypes.c_int32), ("tiles_down1", ctypes.c_int32),
                ("tiles_down1_staged", ctypes.c_int32), ("tiles_down1_interior", ctypes.c_int32)]


# every symbol declared by include/stitch.h, with its ctypes signature
SIGNATURES = {
    "stitch_rig_create": (ctypes.c_int, [ctypes.POINTER(stitch_rig_desc), ctypes.c_int, ctypes.POINTER(_P)]),
    "stitch_rig_destroy": (None, [_P]),
    "stitch_frames": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int64, _P]),
    "stitch_frames_host": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int64, _P]),
    "stitch_frames_host_async": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int64, _P]),
    "stitch_backward": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P]),
    "stitch_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "stitch_rig_get_info": (ctypes.c_int, [_P, ctypes.POINTER(stitch_rig_info)]),
    "stitch_rig_get_camera": (ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.POINTER(ctypes.c_int32)]),
    "stitch_rig_set_profiling": (ctypes.c_int, [_P, ctypes.c_int]),
    "stitch_rig_kernel_times": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]),
    "stitch_batch_create": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(_P)]),
    "stitch_batch_frames": (ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
    "stitch_batch_destroy": (None, [_P]),
    "stitch_batch_get_schedule": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                                 ctypes.POINTER(ctypes.c_int64)]),
    "stitch_batch_wait_test": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32]),
    "stitch_batch_sync": (ctypes.c_int, [_P]),
    "stitch_rig_debug_check": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
    "stitch_frames_static": (ctypes.c_int, [ctypes.POINTER(stitch_rig_desc), _P, _P, _P, ctypes.c_int64, _P]),
    "stitch_lorb_create": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                          ctypes.POINTER(_P)]),
    "stitch_lorb_destroy": (None, [_P]),
    "stitch_lorb_detect": (ctypes.c_int, [_P, _P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, _P, ctypes.c_int32,
                                          ctypes.POINTER(stitch_lorb_params), _P, _P, _P, _P, _P, _P]),
    "stitch_matcher_create": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(_P)]),
    "stitch_matcher_destroy": (None, [_P]),
    "stitch_match_homography": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P, ctypes.POINTER(stitch_match_params), _P,
                                               _P, _P, _P, _P, _P, _P, _P]),
}


class StitchError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {status_string(status)}")


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libstitch.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            # STITCH_LIBRARY selects another build of the library (the debug build)
            path = os.environ.get("STITCH_LIBRARY") or _build.LIB
            if not os.path.exists(path):
                if not build_if_missing:
                    raise RuntimeError("libstitch.so is not built: run __graft_entry__.build() (nvcc, sm_103a)")
                _build.build()
            lib = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def status_string(status: int) -> str:
    try:
        return load().stitch_status_string(status).decode()
    except Exception:  # pragma: no cover - only for messages
        return f"status {status}"


def _check(status: int, what: str):
    if status != STITCH_OK:
        raise StitchError(status, what)


# ------------------------------------------------------------------------------------------------
# functions with the C ABI's names (pointers as Python ints)


def stitch_rig_create(desc: stitch_rig_desc, device: int) -> int:
    out = _P()
    _check(load().stitch_rig_create(ctypes.byref(desc), device, ctypes.byref(out)), "stitch_rig_create")
    return out.value


def stitch_rig_destroy(rig: int) -> None:
    load().stitch_rig_destroy(rig)


def stitch_frames(rig: int, frame_ptrs, pitches, out_ptr: int, out_pitch: int, stream: int) -> None:
    n = len(frame_ptrs)
    fp = (_P * n)(*frame_ptrs)
    pt = (ctypes.c_int64 * n)(*pitches)
    _check(load().stitch_frames(rig, fp, pt, out_ptr, out_pitch, stream), "stitch_frames")


def stitch_frames_host(rig: int, frame_ptrs, pitches, out_ptr: int, out_pitch: int, stream: int) -> None:
    n = len(frame_ptrs)
    fp = (_P * n)(*frame_ptrs)
    pt = (ctypes.c_int64 * n)(*pitches)
    _check(load().stitch_frames_host(rig, fp, pt, out_ptr, out_pitch, stream), "stitch_frames_host")


def stitch_frames_host_async(rig: int, frame_ptrs, pitches, out_ptr: int, out_pitch: int, stream: int) -> None:
    n = len(frame_ptrs)
    fp = (_P * n)(*frame_ptrs)
    pt = (ctypes.c_int64 * n)(*pitches)
    _check(load().stitch_frames_host_async(rig, fp, pt, out_ptr, out_pitch, stream), "stitch_frames_host_async")


def stitch_backward(rig: int, frame_ptrs, pitches, params_ptr: int, loss_ptr: int, grad_ptr: int,
                    stream: int) -> None:
    n = len(frame_ptrs)
    fp = (_P * n)(*frame_ptrs)
    pt = (ctypes.c_int64 * n)(*pitches)
    _check(load().stitch_backward(rig, fp, pt, params_ptr, loss_ptr, grad_ptr or None, stream), "stitch_backward")


def stitch_frames_static(desc: stitch_rig_desc, frame_ptrs, pitches, out_ptr: int, out_pitch: int,
                         stream: int) -> None:
    """Stitch with no device allocation: scratch lives in the library's fixed static device array
    (for callers that cannot allocate, e.g. inside a graph capture); same result as a plain rig."""
    n = len(frame_ptrs)
    fp = (_P * n)(*frame_ptrs)
    pt = (ctypes.c_int64 * n)(*pitches)
    _check(load().stitch_frames_static(ctypes.byref(desc), fp, pt, out_ptr, out_pitch, stream),
           "stitch_frames_static")


def stitch_rig_get_info(rig: int) -> stitch_rig_info:
    info = stitch_rig_info()
    _check(load().stitch_rig_get_info(rig, ctypes.byref(info)), "stitch_rig_get_info")
    return info


def stitch_rig_get_camera(rig: int, index: int):
    a = (ctypes.c_double * 9)()
    vis = ctypes.c_int32()
    _check(load().stitch_rig_get_camera(rig, index, a, ctypes.byref(vis)), "stitch_rig_get_camera")
    return np.array(a[:]).reshape(3, 3), bool(vis.value)


def stitch_rig_set_profiling(rig: int, enable: bool) -> None:
    _check(load().stitch_rig_set_profiling(rig, 1 if enable else 0), "stitch_rig_set_profiling")


def stitch_rig_kernel_times(rig: int, cap: int = 64) -> dict:
    names = (ctypes.c_char_p * cap)()
    ms = (ctypes.c_double * cap)()
    launches = (ctypes.c_int64 * cap)()
    count = ctypes.c_int32()
    _check(load().stitch_rig_kernel_times(rig, names, ms, launches, cap, ctypes.byref(count)),
           "stitch_rig_kernel_times")
    return {names[k].decode(): (ms[k], launches[k]) for k in range(min(count.value, cap))}


def stitch_batch_create(rigs) -> int:
    n = len(rigs)
    arr = (_P * n)(*rigs)
    out = _P()
    _check(load().stitch_batch_create(arr, n, ctypes.byref(out)), "stitch_batch_create")
    return out.value


def stitch_batch_frames(batch: int, frame_ptrs, pitches, out_ptrs, out_pitches, stream: int) -> None:
    n = len(frame_ptrs)
    fps = [(_P * len(f))(*f) for f in frame_ptrs]
    pts = [(ctypes.c_int64 * len(p))(*p) for p in pitches]
    fa = (_P * n)(*[ctypes.cast(f, _P) for f in fps])
    pa = (_P * n)(*[ctypes.cast(p, _P) for p in pts])
    oa = (_P * n)(*out_ptrs)
    op = (ctypes.c_int64 * n)(*out_pitches)
    _check(load().stitch_batch_frames(batch, fa, pa, oa, op, stream), "stitch_batch_frames")


def stitch_batch_destroy(batch: int) -> None:
    load().stitch_batch_destroy(batch)


def stitch_batch_get_schedule(batch: int) -> dict:
    o, g, t = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
    _check(load().stitch_batch_get_schedule(batch, ctypes.byref(o), ctypes.byref(g), ctypes.byref(t)),
           "stitch_batch_get_schedule")
    cached = bool(o.value >> 24 & 1)
    code = o.value & 0xFFFFFF
    if code & 0xF == 0xF:
        shape = code >> 8 & 0xF
        return {"mode": "staged", "reduce_tile": ["32x16", "64x8"][shape & 1],
                "coarse_tile": ["32x32", "64x16"][shape >> 1], "shape": shape, "tasks": t.value, "cached": cached}
    if code == 0xE:
        return {"mode": "streams", "tasks": t.value, "cached": cached}
    return {"mode": "persistent", "order": code & 15, "register_variant": (code >> 4) & 15, "chunk": code >> 8,
            "grid": g.value, "tasks": t.value, "cached": cached}


def stitch_batch_sync(batch: int) -> None:
    _check(load().stitch_batch_sync(batch), "stitch_batch_sync")


def stitch_batch_wait_test(batch: int, spin_limit: int, rig: int) -> None:
    _check(load().stitch_batch_wait_test(batch, spin_limit, rig), "stitch_batch_wait_test")


# ------------------------------------------------------------------------------------------------
# torch-facing convenience wrapper


def _stream_handle(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def make_desc(cameras, canvas_w: int, canvas_h: int, levels: int, band_fp16: bool = False, out_float: bool = False,
              path: str = "fused", weights: str = "feather", canvas=None):
    """Build a stitch_rig_desc from objects with width, height, H (3x3) and gain; ``weights`` is
    "feather" or "seam"; ``canvas`` is None (planar: H is camera->canvas) or (f, cx, cy) of a
    cylindrical canvas (H is the camera's ray->camera matrix P = K R)."""
    n = len(cameras)
    arr = (stitch_camera * n)()
    for k, c in enumerate(cameras):
        arr[k].width = int(c.width)
        arr[k].height = int(c.height)
        Hm = np.asarray(c.H, dtype=np.float64).reshape(9)
        for j in range(9):
            arr[k].H[j] = float(Hm[j])
        arr[k].gain = float(getattr(c, "gain", 1.0))
    desc = stitch_rig_desc(n, ctypes.cast(arr, ctypes.POINTER(stitch_camera)), int(canvas_w), int(canvas_h),
                           int(levels), int(bool(band_fp16)), int(bool(out_float)),
                           STITCH_PATH_PLAIN if path == "plain" else STITCH_PATH_FUSED,
                           {"feather": STITCH_WEIGHTS_FEATHER, "seam": STITCH_WEIGHTS_SEAM}[weights])
    if canvas is not None:
        desc.canvas_model = STITCH_CANVAS_CYLINDRICAL
        for k, v in enumerate(canvas):
            desc.cylinder[k] = float(v)
    return desc, arr


class Rig:
    """A created rig: cameras, canvas and pyramid depth fixed; frames stitched on the GPU."""

    def __init__(self, cameras, canvas_w: int, canvas_h: int, levels: int, band_fp16: bool = False,
                 out_float: bool = False, path: str = "fused", device: int | None = None, weights: str = "feather",
                 canvas=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("libstitch needs a CUDA GPU; no CPU fallback exists")
        self.device = torch.cuda.current_device() if device is None else int(device)
        self.cameras = list(cameras)
        self.canvas_w, self.canvas_h, self.levels = int(canvas_w), int(canvas_h), int(levels)
        self.out_float = bool(out_float)
        self.band_fp16 = bool(band_fp16)
        self.path = path
        self.weights = weights
        self.canvas = canvas
        desc, keep = make_desc(self.cameras, canvas_w, canvas_h, levels, band_fp16, out_float, path, weights, canvas)
        self.handle = stitch_rig_create(desc, self.device)
        del keep

    def close(self):
        if getattr(self, "handle", None):
            stitch_rig_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def new_output(self):
        import torch
        dt = torch.float32 if self.out_float else torch.uint8
        return torch.empty((self.canvas_h, self.canvas_w, 3), dtype=dt, device=f"cuda:{self.device}")

    def stitch(self, frames, out=None, stream=None):
        """frames: list of (H, W, 3) uint8 CUDA tensors (row-contiguous).  Returns the canvas tensor."""
        if out is None:
            out = self.new_output()
        ptrs, pitches = _frame_args(frames, self.cameras, self.device)
        optr, opitch = self._canvas_args(out, self.device)
        stitch_frames(self.handle, ptrs, pitches, optr, opitch, _stream_handle(stream))
        return out

    def _canvas_args(self, out, device):
        """(pointer, row pitch) of a canvas buffer: (canvas_h, canvas_w, 3), float32 when the rig
        writes floats, else uint8."""
        return _image_args(out, self.canvas_h, self.canvas_w, 4 if self.out_float else 1, device, "output canvas")

    def stitch_host(self, frames, out: np.ndarray | None = None, stream=None) -> np.ndarray:
        """frames: list of (H, W, 3) uint8 host arrays or pinned tensors; returns a host canvas."""
        import torch
        if out is None:
            out = np.empty((self.canvas_h, self.canvas_w, 3), dtype=np.float32 if self.out_float else np.uint8)
        ptrs, pitches = _frame_args(frames, self.cameras, None)
        optr, opitch = self._canvas_args(out, None)
        stitch_frames_host(self.handle, ptrs, pitches, optr, opitch, _stream_handle(stream))
        return out

    def stitch_host_async(self, frames, out, stream=None):
        """Enqueue a host-buffer stitch (frames: pinned uint8 tensors or arrays; out: pinned host
        canvas); consecutive calls overlap upload, compute and download.  Synchronise `stream`
        (default: the current torch stream) before reading `out` or reusing the inputs."""
        import torch
        ptrs, pitches = _frame_args(frames, self.cameras, None)
        optr, opitch = self._canvas_args(out, None)
        stitch_frames_host_async(self.handle, ptrs, pitches, optr, opitch, _stream_handle(stream))
        return out

    def backward(self, frames, params, loss=None, grad=None, stream=None):
        """params: (N, 9) float64 CUDA tensor (a11..a32, gain).  Returns (loss (1,), grad (N, 9))."""
        import torch
        n = len(self.cameras)
        pptr = _float64_args(params, (n, 9), self.device, "params")
        if loss is None:
            loss = torch.empty(1, dtype=torch.float64, device=params.device)
        if grad is None:
            grad = torch.empty_like(params)
        ptrs, pitches = _frame_args(frames, self.cameras, self.device)
        stitch_backward(self.handle, ptrs, pitches, pptr, _float64_args(loss, (1,), self.device, "loss"),
                        _float64_args(grad, (n, 9), self.device, "grad"), _stream_handle(stream))
        return loss, grad

    def camera_map(self, index: int):
        """(A as 3x3 with a33 = +-1, visible) of camera ``index`` as the kernels use it."""
        return stitch_rig_get_camera(self.handle, index)

    def info(self) -> dict:
        i = stitch_rig_get_info(self.handle)
        return {"scratch_bytes": i.scratch_bytes, "num_kernels": i.num_kernels, "path": i.path,
                "roi_pixels": i.roi_pixels,
                "tiles": {"zero": i.tiles_zero, "solo": i.tiles_solo, "full2": i.tiles_full2,
                          "full4": i.tiles_full4, "general": i.tiles_general, "down1": i.tiles_down1,
                          "down1_staged": i.tiles_down1_staged, "down1_interior": i.tiles_down1_interior}}

    def debug_check(self) -> dict:
        """Debug build only: guard words no longer intact and the first failed index check."""
        dmg, chk = ctypes.c_int64(), ctypes.c_int64()
        _check(load().stitch_rig_debug_check(self.handle, ctypes.byref(dmg), ctypes.byref(chk)),
               "stitch_rig_debug_check")
        return {"damaged_words": dmg.value, "failed_check": chk.value}

    def set_profiling(self, enable: bool):
        stitch_rig_set_profiling(self.handle, enable)

    def kernel_times(self) -> dict:
        return stitch_rig_kernel_times(self.handle)


class Batch:
    """Several rigs (fused path, same device and band storage) stitched together by the schedule
    the batch picks on its first call.  stitch() is asynchronous after that first call; sync()
    waits for the last call and raises if a device wait gave up."""

    def __init__(self, rigs):
        self.rigs = list(rigs)
        self.handle = stitch_batch_create([r.handle for r in self.rigs])

    def close(self):
        if getattr(self, "handle", None):
            stitch_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def stitch(self, frames_per_rig, outs=None, stream=None):
        """frames_per_rig: one list of CUDA frame tensors per rig.  Returns the output tensors."""
        if outs is None:
            outs = [r.new_output() for r in self.rigs]
        frames_per_rig, outs = list(frames_per_rig), list(outs)
        if len(frames_per_rig) != len(self.rigs) or len(outs) != len(self.rigs):
            raise ValueError(f"expected frames and an output for each of {len(self.rigs)} rigs, got "
                             f"{len(frames_per_rig)} and {len(outs)}")
        fps, pts, ops, ops_pitch = [], [], [], []
        for fr, r, o in zip(frames_per_rig, self.rigs, outs):
            a, b = _frame_args(fr, r.cameras, r.device)
            fps.append(a)
            pts.append(b)
            optr, opitch = r._canvas_args(o, r.device)
            ops.append(optr)
            ops_pitch.append(opitch)
        stitch_batch_frames(self.handle, fps, pts, ops, ops_pitch, _stream_handle(stream))
        return outs

    def sync(self) -> None:
        stitch_batch_sync(self.handle)

    def schedule(self) -> dict:
        return stitch_batch_get_schedule(self.handle)

    def wait_test(self, spin_limit: int, rig: int):
        stitch_batch_wait_test(self.handle, spin_limit, rig)


def _image_args(t, h: int, w: int, itemsize: int, device, what: str):
    """(pointer, row pitch in bytes) of an (h, w, 3) image with packed pixels and rows at any pitch
    of at least one row: a torch tensor (on CUDA device `device`, or in host memory when `device`
    is None) or, for host memory, a NumPy array.  Raises ValueError otherwise, before the library
    could read or write outside the buffer."""
    import torch
    if isinstance(t, torch.Tensor):
        if device is None:
            if t.is_cuda:
                raise ValueError(f"{what}: expected a host tensor, got one on {t.device}")
        elif not t.is_cuda or t.device.index != device:
            raise ValueError(f"{what}: expected a tensor on cuda:{device}, got one on {t.device}")
        size = t.element_size()
        strides = tuple(t.stride()) if t.dim() == 3 else ()
        ptr = t.data_ptr()
    elif isinstance(t, np.ndarray) and device is None:
        size = t.itemsize
        strides = tuple(s // size for s in t.strides) if t.ndim == 3 and all(s % size == 0 for s in t.strides) else ()
        ptr = t.ctypes.data
    else:
        raise ValueError(f"{what}: expected a {'host' if device is None else 'CUDA'} tensor, got {type(t).__name__}")
    if tuple(t.shape) != (h, w, 3) or size != itemsize:
        raise ValueError(f"{what}: expected shape ({h}, {w}, 3) with {itemsize}-byte elements, got "
                         f"{tuple(t.shape)} with {size}-byte elements")
    if strides[1:] != (3, 1) or strides[0] < 3 * w:
        raise ValueError(f"{what}: pixels must be packed (strides (>= {3 * w}, 3, 1) elements), got {strides}")
    return ptr, strides[0] * size


def _frame_args(frames, cameras, device):
    """Pointers and row pitches of one uint8 frame per camera (device None: host frames)."""
    frames = list(frames)
    if len(frames) != len(cameras):
        raise ValueError(f"expected {len(cameras)} frames (one per camera), got {len(frames)}")
    ptrs, pitches = [], []
    for k, (f, c) in enumerate(zip(frames, cameras)):
        ptr, pitch = _image_args(f, c.height, c.width, 1, device, f"frame {k}")
        ptrs.append(ptr)
        pitches.append(pitch)
    return ptrs, pitches


def _float64_args(t, shape, device, what: str) -> int:
    """Pointer of a contiguous float64 CUDA tensor of the given shape on `device`."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.device.index != device:
        raise ValueError(f"{what}: expected a float64 tensor on cuda:{device}")
    if t.dtype != torch.float64 or tuple(t.shape) != tuple(shape) or not t.is_contiguous():
        raise ValueError(f"{what}: expected a contiguous float64 tensor of shape {tuple(shape)}, got "
                         f"{t.dtype} {tuple(t.shape)}")
    return t.data_ptr()


def stitch_lorb_create(max_width: int, max_height: int, max_points: int, device: int) -> int:
    out = _P()
    _check(load().stitch_lorb_create(max_width, max_height, max_points, device, ctypes.byref(out)), "stitch_lorb_create")
    return out.value


def stitch_lorb_destroy(ctx: int) -> None:
    load().stitch_lorb_destroy(ctx)


def stitch_lorb_detect(ctx: int, frame_ptr: int, width: int, height: int, pitch: int, areas, params, pattern,
                       xy_ptr: int, resp_ptr: int, desc_ptr: int, count_ptr: int, stream: int) -> None:
    ar = np.ascontiguousarray(np.asarray(areas, dtype=np.int32).reshape(-1, 4))
    pat = np.ascontiguousarray(np.asarray(pattern, dtype=np.int8).reshape(256, 4))
    _check(load().stitch_lorb_detect(ctx, frame_ptr, width, height, pitch, ar.ctypes.data if len(ar) else None, len(ar),
                                     ctypes.byref(params), pat.ctypes.data, xy_ptr, resp_ptr, desc_ptr, count_ptr,
                                     stream), "stitch_lorb_detect")


class LORB:
    """L-ORB feature extraction on the GPU (Sec. 4.1): FAST-9 + Harris + NMS + top-N + BRIEF."""

    def __init__(self, max_width: int, max_height: int, max_points: int = 500, device: int | None = None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("libstitch needs a CUDA GPU; no CPU fallback exists")
        self.device = torch.cuda.current_device() if device is None else int(device)
        self.max_points = int(max_points)
        self.handle = stitch_lorb_create(int(max_width), int(max_height), self.max_points, self.device)
        d = f"cuda:{self.device}"
        self.xy = torch.empty((self.max_points, 2), dtype=torch.int32, device=d)
        self.resp = torch.empty(self.max_points, dtype=torch.int64, device=d)
        self.desc = torch.empty((self.max_points, 32), dtype=torch.uint8, device=d)
        self.count = torch.zeros(1, dtype=torch.int32, device=d)

    def close(self):
        if getattr(self, "handle", None):
            stitch_lorb_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def detect(self, frame, areas, pattern, fast_t: int = 20, harris_t: int = 0, max_points: int | None = None,
               stream=None):
        """frame: (H, W, 3) uint8 CUDA tensor.  Enqueues the detection; returns (xy, resp, desc, count)
        views of the context's output tensors (valid after the stream reaches them)."""
        if not hasattr(frame, "shape") or len(frame.shape) != 3:
            raise ValueError("frame: expected an (H, W, 3) uint8 CUDA tensor")
        fptr, fpitch = _image_args(frame, frame.shape[0], frame.shape[1], 1, self.device, "frame")
        n = self.max_points if max_points is None else int(max_points)
        prm = stitch_lorb_params(int(fast_t), int(harris_t), n)
        stitch_lorb_detect(self.handle, fptr, frame.shape[1], frame.shape[0], fpitch, areas, prm,
                           pattern, self.xy.data_ptr(), self.resp.data_ptr(), self.desc.data_ptr(),
                           self.count.data_ptr(), _stream_handle(stream))
        return self.xy, self.resp, self.desc, self.count


def stitch_matcher_create(max_points: int, max_iters: int, device: int) -> int:
    out = _P()
    _check(load().stitch_matcher_create(max_points, max_iters, device, ctypes.byref(out)), "stitch_matcher_create")
    return out.value


def stitch_matcher_destroy(ctx: int) -> None:
    load().stitch_matcher_destroy(ctx)


def stitch_match_homography(ctx: int, xy_a: int, desc_a: int, count_a: int, xy_b: int, desc_b: int, count_b: int,
                            params, bits, rnd: int, matches: int, n_matches: int, H: int, n_inliers: int,
                            inlier: int, stream: int) -> None:
    bt = np.ascontiguousarray(np.asarray(bits, dtype=np.uint8))
    _check(load().stitch_match_homography(ctx, xy_a, desc_a, count_a, xy_b, desc_b, count_b, ctypes.byref(params),
                                          bt.ctypes.data, rnd or None, matches, n_matches, H, n_inliers, inlier,
                                          stream), "stitch_match_homography")


class Matcher:
    """Multi-Probe LSH matching and PROSAC homography on the GPU (Sec. 4.2, Algorithm 3)."""

    def __init__(self, max_points: int = 500, max_iters: int = 1024, device: int | None = None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("libstitch needs a CUDA GPU; no CPU fallback exists")
        self.device = torch.cuda.current_device() if device is None else int(device)
        self.max_points, self.max_iters = int(max_points), int(max_iters)
        self.handle = stitch_matcher_create(self.max_points, self.max_iters, self.device)
        d = f"cuda:{self.device}"
        self.matches = torch.empty((self.max_points, 3), dtype=torch.int32, device=d)
        self.n_matches = torch.zeros(1, dtype=torch.int32, device=d)
        self.H = torch.empty(9, dtype=torch.float64, device=d)
        self.n_inliers = torch.zeros(1, dtype=torch.int32, device=d)
        self.inlier = torch.empty(self.max_points, dtype=torch.uint8, device=d)

    def close(self):
        if getattr(self, "handle", None):
            stitch_matcher_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def match(self, xy_a, desc_a, count_a, xy_b, desc_b, count_b, bits, rnd, max_dist: int = 80, ratio=(4, 5),
              inlier_px: float = 3.0, stream=None):
        """Device tensors: xy (n, 2) int32, desc (n, 32) uint8, count (1,) int32 per image (the
        outputs of LORB.detect); bits (L, k) host array of descriptor bit positions; rnd (T, 4)
        uint32/int32 CUDA tensor of random words.  Enqueues the work; returns views (matches,
        n_matches, H (9,) float64, n_inliers, inlier) of the context's outputs."""
        import torch
        for name, t, size, width in (("xy_a", xy_a, 4, 2), ("desc_a", desc_a, 1, 32), ("count_a", count_a, 4, 0),
                                     ("xy_b", xy_b, 4, 2), ("desc_b", desc_b, 1, 32), ("count_b", count_b, 4, 0)):
            ok = isinstance(t, torch.Tensor) and t.is_cuda and t.device.index == self.device and t.is_contiguous() \
                and t.element_size() == size and (t.numel() >= 1 if width == 0 else (t.dim() == 2 and t.shape[1] == width))
            if not ok:
                raise ValueError(f"{name}: expected a contiguous CUDA tensor on cuda:{self.device} of "
                                 f"{'one' if width == 0 else f'(n, {width})'} {size}-byte elements")
        bt = np.asarray(bits, dtype=np.uint8)
        iters = 0 if rnd is None else int(rnd.shape[0])
        if iters and not (isinstance(rnd, torch.Tensor) and rnd.is_cuda and rnd.device.index == self.device and
                          rnd.is_contiguous() and rnd.element_size() == 4 and rnd.dim() == 2 and rnd.shape[1] == 4):
            raise ValueError(f"rnd: expected a contiguous (T, 4) tensor of 32-bit words on cuda:{self.device}")
        prm = stitch_match_params(int(bt.shape[0]), int(bt.shape[1]), int(max_dist), int(ratio[0]), int(ratio[1]),
                                  iters, float(inlier_px))
        stitch_match_homography(self.handle, xy_a.data_ptr(), desc_a.data_ptr(), count_a.data_ptr(), xy_b.data_ptr(),
                                desc_b.data_ptr(), count_b.data_ptr(), prm, bt,
                                rnd.data_ptr() if iters else 0, self.matches.data_ptr(), self.n_matches.data_ptr(),
                                self.H.data_ptr(), self.n_inliers.data_ptr(), self.inlier.data_ptr(),
                                _stream_handle(stream))
        return self.matches, self.n_matches, self.H, self.n_inliers, self.inlier
