"""FP64 CPU oracle of the panoramic stitching path (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
this package.  The product (``paper_1810_03988_gb300``) never imports it and shares no code with
it: the oracle is a separate C library (``oracle.c``) compiled with gcc, evaluated in double
precision, loaded through ctypes.

Paper anchors: Sec. 4.3 / Alg. 4 step 1 (frames "cut and transformed" on the GPU) and step 6
("transform the video and blend it into a panoramic video"), Sec. 1 contribution 3 ("multi band
fusion").  The paper states no formulas; ``oracle.c`` lists the readings it evaluates.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None
_threads_used = None

_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double


def compile_library(src: str, out: str) -> None:
    """gcc -O2, IEEE double without contractions, OpenMP when available: ``src`` -> shared ``out``."""
    base = ["gcc", "-O2", "-fPIC", "-shared", "-std=c99", "-fno-fast-math", "-ffp-contract=off", src, "-o", out,
            "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` (see compile_library).  ORACLE_LIBRARY names a prebuilt library to load
    instead (the pin tests run against deliberately broken copies that way)."""
    override = os.environ.get("ORACLE_LIBRARY")
    if override:
        return override
    src = os.path.join(_HERE, "oracle.c")
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(src):
        return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = f"{_LIB_PATH}.{os.getpid()}.tmp"
    compile_library(src, tmp)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.oracle_invert_h.argtypes = [_P, _P]
            lib.oracle_reduce.argtypes = [_P, _I, _I, _I, _P]
            lib.oracle_expand.argtypes = [_P, _I, _I, _I, _I, _I, _P]
            lib.oracle_regions.argtypes = [_I, _I, _I, _I, _I, _I, _I, _P]
            lib.oracle_forward.argtypes = [_I, _P, _P, _P, _P, _P, _P, _I, _I, _I, _I, _I, _I, _I, _P, _P, _P,
                                           _P, _P, _I, _P]
            lib.oracle_warp.argtypes = [_I, _I, _P, _D, _P, ctypes.c_int64, _I, _I, _P, _P, _P]
            lib.oracle_lorb.argtypes = [_I, _I, _P, ctypes.c_int64, _P, _I, _I, ctypes.c_int64, _I, _P, _P, _P, _P,
                                        _P, _P]
            lib.oracle_lorb.restype = _I
            lib.oracle_match_prosac.argtypes = [_I, _P, _P, _I, _P, _P, _I, _I, _P, _I, _I, _I, _D, _I, _P, _P, _P,
                                                _P, _P, _P]
            lib.oracle_match_prosac.restype = _I
            lib.oracle_prosac_schedule.argtypes = [_I, _I, _P, _P]
            lib.oracle_prosac_schedule.restype = _I
            lib.oracle_prosac_sample.argtypes = [_I, _I, _P, _P]
            lib.oracle_prosac_sample.restype = _I
            lib.oracle_loss_grad.argtypes = [_I, _P, _P, _P, _P, _P, _P, _P, _I, _I, _I, _I, _P, _P]
            for f in ("oracle_invert_h", "oracle_reduce", "oracle_expand", "oracle_regions", "oracle_forward",
                      "oracle_warp", "oracle_loss_grad"):
                getattr(lib, f).restype = _I
            _lib = lib
    return _lib


def threads() -> int:
    """Number of OpenMP threads the oracle runs with (OMP_NUM_THREADS, else the affinity mask)."""
    env = os.environ.get("OMP_NUM_THREADS")
    if env:
        return int(env)
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def _check(rc: int, what: str):
    if rc != 0:
        raise ValueError(f"oracle {what} failed with status {rc}")


def invert_h(M) -> np.ndarray:
    """Canvas->camera map A = M^-1 / |(M^-1)_33| (a33 = +1 or -1, the sign of w is kept)."""
    M = np.ascontiguousarray(M, dtype=np.float64).reshape(9)
    A = np.empty(9)
    _check(_load().oracle_invert_h(M.ctypes.data, A.ctypes.data), "invert_h")
    return A.reshape(3, 3)


def reduce(img: np.ndarray) -> np.ndarray:
    """One REDUCE step (separable [1,4,6,4,1]/16, even-index decimation, reflect-101) of HxWxC."""
    img = np.ascontiguousarray(img, dtype=np.float64)
    if img.ndim == 2:
        return reduce(img[:, :, None])[:, :, 0]
    h, w, c = img.shape
    out = np.empty(((h + 1) // 2, (w + 1) // 2, c))
    _check(_load().oracle_reduce(img.ctypes.data, w, h, c, out.ctypes.data), "reduce")
    return out


def expand(img: np.ndarray, shape) -> np.ndarray:
    """One EXPAND step of a coarse HcxWcxC image to the finer size ``shape`` = (h, w)."""
    img = np.ascontiguousarray(img, dtype=np.float64)
    if img.ndim == 2:
        return expand(img[:, :, None], shape)[:, :, 0]
    hc, wc, c = img.shape
    h, w = shape
    out = np.empty((h, w, c))
    _check(_load().oracle_expand(img.ctypes.data, wc, hc, c, w, h, out.ctypes.data), "expand")
    return out


def gaussian_pyramid(img: np.ndarray, levels: int) -> list:
    out = [np.asarray(img, dtype=np.float64)]
    for _ in range(levels - 1):
        out.append(reduce(out[-1]))
    return out


def laplacian_pyramid(img: np.ndarray, levels: int) -> list:
    g = gaussian_pyramid(img, levels)
    return [g[l] - expand(g[l + 1], g[l].shape[:2]) for l in range(levels - 1)] + [g[-1]]


def collapse(lap: list) -> np.ndarray:
    r = lap[-1]
    for l in range(len(lap) - 2, -1, -1):
        r = lap[l] + expand(r, lap[l].shape[:2])
    return r


def _cam_arrays(cams, frames):
    n = len(cams)
    Ws = np.array([c.width for c in cams], dtype=np.int32)
    Hs = np.array([c.height for c in cams], dtype=np.int32)
    Ms = np.ascontiguousarray(np.stack([np.asarray(c.H, dtype=np.float64).reshape(9) for c in cams]))
    gains = np.array([float(getattr(c, "gain", 1.0)) for c in cams], dtype=np.float64)
    frames = _frames(frames, Ws, Hs)
    fp = (ctypes.c_void_p * n)(*[f.ctypes.data for f in frames])
    pitches = np.array([f.strides[0] for f in frames], dtype=np.int64)
    return Ws, Hs, Ms, gains, fp, pitches, frames


def _frames(frames, widths, heights):
    """Contiguous uint8 copies of one (H, W, 3) frame per camera; ValueError on a count or shape
    that does not match the cameras (the C code reads H rows of 3 W bytes from each)."""
    frames = [np.ascontiguousarray(f, dtype=np.uint8) for f in frames]
    if len(frames) != len(widths):
        raise ValueError(f"expected {len(widths)} frames, got {len(frames)}")
    for k, (f, w, h) in enumerate(zip(frames, widths, heights)):
        if f.shape != (int(h), int(w), 3):
            raise ValueError(f"frame {k}: expected shape ({int(h)}, {int(w)}, 3), got {f.shape}")
    return frames


def regions(canvas_w: int, canvas_h: int, levels: int, window=None) -> np.ndarray:
    """Per-level rectangles [X_l | Y_l] as an (L, 8) array of (x0, x1, y0, y1) pairs."""
    x0, y0, w, h = window if window is not None else (0, 0, canvas_w, canvas_h)
    out = np.empty((levels, 8), dtype=np.int32)
    _check(_load().oracle_regions(canvas_w, canvas_h, levels, x0, y0, w, h, out.ctypes.data), "regions")
    return out


def _cyl_arg(canvas):
    """None for the planar canvas, else a (f, cx, cy) double array for a cylindrical one."""
    if canvas is None:
        return None, None
    arr = np.ascontiguousarray(np.asarray(canvas, dtype=np.float64).reshape(3))
    return arr.ctypes.data, arr


def forward(cams, frames, canvas_w: int, canvas_h: int, levels: int, window=None, debug: bool = False,
            weights: str = "feather", canvas=None):
    """Stitch one frame set (S1-S6) in double precision.

    ``weights``: "feather" (normalised distance-to-border weights) or "seam" (binary masks: each
    pixel owned by the camera with the largest feather weight, ties to the lower index).
    ``canvas``: None (planar canvas; ``cam.H`` is camera->canvas) or (f, cx, cy) of a cylindrical
    canvas (``cam.H`` is the camera's P = K R, applied to the canvas ray).

    ``cams``: objects with ``width``, ``height``, ``H`` (camera->canvas 3x3) and ``gain``.
    ``window``: (x0, y0, w, h) output rectangle, default the whole canvas.
    Returns dict with ``out`` (h x w x 3 float64 in [0,1]), ``u8`` (h x w x 3 uint8), ``mindist``
    (h x w distance in source px to the nearest validity border over all cameras) and, when
    ``debug``, ``S``/``B`` per level on the X_l rectangles with ``regions``.
    """
    lib = _load()
    n = len(cams)
    Ws, Hs, Ms, gains, fp, pitches, keep = _cam_arrays(cams, frames)
    x0, y0, w, h = window if window is not None else (0, 0, canvas_w, canvas_h)
    out = np.empty((h, w, 3))
    u8 = np.empty((h, w, 3), dtype=np.uint8)
    md = np.empty((h, w))
    S = B = None
    dS = dB = None
    reg = regions(canvas_w, canvas_h, levels, (x0, y0, w, h))
    if debug:
        S = [np.empty((r[3] - r[2], r[1] - r[0])) for r in reg]
        B = [np.empty((r[3] - r[2], r[1] - r[0], 3)) for r in reg]
        dS = (ctypes.c_void_p * levels)(*[a.ctypes.data for a in S])
        dB = (ctypes.c_void_p * levels)(*[a.ctypes.data for a in B])
    cyl_ptr, cyl_keep = _cyl_arg(canvas)
    rc = lib.oracle_forward(n, Ws.ctypes.data, Hs.ctypes.data, Ms.ctypes.data, gains.ctypes.data, fp,
                            pitches.ctypes.data, canvas_w, canvas_h, levels, x0, y0, w, h, out.ctypes.data,
                            u8.ctypes.data, md.ctypes.data, dS, dB, {"feather": 0, "seam": 1}[weights],
                            cyl_ptr)
    del cyl_keep
    _check(rc, "forward")
    del keep
    res = {"out": out, "u8": u8, "mindist": md, "regions": reg}
    if debug:
        res["S"] = S
        res["B"] = B
    return res


def warp(cam, frame, canvas_w: int, canvas_h: int, canvas=None):
    """Level 0 of one camera on the whole canvas: (I_i as HcxWcx3, raw feather weight HcxWc);
    ``canvas`` as for forward."""
    lib = _load()
    frame = _frames([frame], [cam.width], [cam.height])[0]
    M = np.ascontiguousarray(np.asarray(cam.H, dtype=np.float64).reshape(9))
    img = np.empty((canvas_h, canvas_w, 3))
    wr = np.empty((canvas_h, canvas_w))
    cyl_ptr, cyl_keep = _cyl_arg(canvas)
    rc = lib.oracle_warp(cam.width, cam.height, M.ctypes.data, float(getattr(cam, "gain", 1.0)),
                         frame.ctypes.data, frame.strides[0], canvas_w, canvas_h, img.ctypes.data, wr.ctypes.data,
                         cyl_ptr)
    del cyl_keep
    _check(rc, "warp")
    return img, wr


def loss_grad(widths, heights, params, frames, window, mask_params=None, grad: bool = True, a33=None):
    """Overlap SSD loss (S7) and its gradient with respect to (a11..a32, gain) per camera.

    ``params``/``mask_params``: (n, 9) arrays; ``a33``: per-camera +-1 (default +1);
    ``window``: canvas (x0, y0, w, h).  Returns (loss, grad (n, 9) or None)."""
    lib = _load()
    n = len(widths)
    Ws = np.asarray(widths, dtype=np.int32)
    Hs = np.asarray(heights, dtype=np.int32)
    p = np.ascontiguousarray(params, dtype=np.float64).reshape(n, 9)
    mp = None if mask_params is None else np.ascontiguousarray(mask_params, dtype=np.float64).reshape(n, 9)
    frames = _frames(frames, Ws, Hs)
    fp = (ctypes.c_void_p * n)(*[f.ctypes.data for f in frames])
    pitches = np.array([f.strides[0] for f in frames], dtype=np.int64)
    loss = np.zeros(1)
    g = np.zeros((n, 9)) if grad else None
    x0, y0, w, h = window
    s33 = None if a33 is None else np.ascontiguousarray(a33, dtype=np.float64).reshape(n)
    rc = lib.oracle_loss_grad(n, Ws.ctypes.data, Hs.ctypes.data, p.ctypes.data,
                              None if mp is None else mp.ctypes.data, None if s33 is None else s33.ctypes.data,
                              fp, pitches.ctypes.data, x0, y0, w, h, loss.ctypes.data,
                              None if g is None else g.ctypes.data)
    _check(rc, "loss_grad")
    return float(loss[0]), g


def lorb(frame, areas, pattern, fast_t: int = 20, harris_t: int = 0, max_points: int = 500, debug: bool = False):
    """L-ORB features (FAST-9 + Harris + NMS + top-N + BRIEF, integer arithmetic) of one RGB8 frame.

    ``areas``: (m, 4) int rectangles (x0, y0, x1, y1); ``pattern``: (256, 4) int8 BRIEF point
    pairs.  Returns dict(xy (n, 2) int32, resp (n,) int64, desc (n, 32) uint8[, resp_map])."""
    lib = _load()
    frame = np.ascontiguousarray(frame, dtype=np.uint8)
    if frame.ndim != 3 or frame.shape[2] != 3:
        raise ValueError(f"expected an (H, W, 3) frame, got shape {frame.shape}")
    H, W = frame.shape[:2]
    ar = np.ascontiguousarray(np.asarray(areas, dtype=np.int32).reshape(-1, 4))
    pat = np.ascontiguousarray(np.asarray(pattern, dtype=np.int8).reshape(256, 4))
    xy = np.zeros((max_points, 2), np.int32)
    resp = np.zeros(max_points, np.int64)
    desc = np.zeros((max_points, 32), np.uint8)
    cnt = np.zeros(1, np.int32)
    rmap = np.empty((H, W), np.int64) if debug else None
    rc = lib.oracle_lorb(W, H, frame.ctypes.data, frame.strides[0], ar.ctypes.data if len(ar) else None, len(ar),
                         int(fast_t), int(harris_t), int(max_points), pat.ctypes.data, xy.ctypes.data,
                         resp.ctypes.data, desc.ctypes.data, cnt.ctypes.data,
                         rmap.ctypes.data if debug else None)
    _check(rc, "lorb")
    n = int(cnt[0])
    res = {"xy": xy[:n], "resp": resp[:n], "desc": desc[:n]}
    if debug:
        res["resp_map"] = rmap
    return res


def prosac_schedule(N: int, T: int):
    """PROSAC growth schedule for N matches over iterations t = 1..T: (n(t) int32, uniform(t) bool)."""
    nt = np.zeros(max(T, 1), np.int32)
    uni = np.zeros(max(T, 1), np.uint8)
    _check(_load().oracle_prosac_schedule(int(N), int(T), nt.ctypes.data, uni.ctypes.data), "prosac_schedule")
    return nt[:T], uni[:T].astype(bool)


def prosac_sample(n: int, uniform: bool, words) -> np.ndarray:
    """The 4 match indices (into the quality order) that PROSAC draws from the top n for one
    iteration's 4 random words: (4,) int32."""
    w = np.ascontiguousarray(np.asarray(words, dtype=np.uint32).reshape(4))
    idx = np.zeros(4, np.int32)
    _check(_load().oracle_prosac_sample(int(n), int(bool(uniform)), w.ctypes.data, idx.ctypes.data), "prosac_sample")
    return idx


def match_prosac(xy_a, desc_a, xy_b, desc_b, bits, rnd, max_dist: int = 80, ratio=(4, 5), inlier_px: float = 3.0):
    """Multi-Probe LSH matching (bits: (L, k) positions) and PROSAC homography (rnd: (iters, 4)
    uint32 words).  Returns dict(matches (n, 3): a, b, distance in quality order; H (3, 3) mapping
    image-A points to image B; inliers (count); inlier (n,) bool)."""
    lib = _load()
    xa = np.ascontiguousarray(np.asarray(xy_a, dtype=np.int32).reshape(-1, 2))
    xb = np.ascontiguousarray(np.asarray(xy_b, dtype=np.int32).reshape(-1, 2))
    da = np.ascontiguousarray(np.asarray(desc_a, dtype=np.uint8).reshape(-1, 32))
    db = np.ascontiguousarray(np.asarray(desc_b, dtype=np.uint8).reshape(-1, 32))
    bt = np.ascontiguousarray(np.asarray(bits, dtype=np.uint8))
    L, k = bt.shape
    rw = np.ascontiguousarray(np.asarray(rnd, dtype=np.uint32).reshape(-1, 4))
    na, nb = len(xa), len(xb)
    matches = np.zeros((max(na, 1), 3), np.int32)
    nm = np.zeros(1, np.int32)
    H = np.zeros(9)
    ni = np.zeros(1, np.int32)
    inl = np.zeros(max(na, 1), np.uint8)
    rc = lib.oracle_match_prosac(na, xa.ctypes.data, da.ctypes.data, nb, xb.ctypes.data, db.ctypes.data, L, k,
                                 bt.ctypes.data, int(max_dist), int(ratio[0]), int(ratio[1]), float(inlier_px),
                                 len(rw), rw.ctypes.data if len(rw) else None, matches.ctypes.data, nm.ctypes.data,
                                 H.ctypes.data, ni.ctypes.data, inl.ctypes.data)
    _check(rc, "match_prosac")
    n = int(nm[0])
    return {"matches": matches[:n], "H": H.reshape(3, 3), "inliers": int(ni[0]), "inlier": inl[:n].astype(bool)}
