"""Seeded synthetic rigs, scenes and camera frames (input data for both sides).

This module produces inputs only.  It contains no stitching arithmetic: camera
frames are rendered by point-evaluating a procedural scene (value noise plus
textured rectangles, see ``synth.c``) at the canvas point that each camera
pixel maps to.  The oracle and the CUDA path both consume its output as plain
arrays; neither imports the other.

Rig geometry (the paper fixes none; Alg. 4 step 5 only says a "transformation
matrix" per camera exists):

* planar rig: camera i maps to the canvas by ``M_i = T_c K_c R_y(theta_i) K_i^-1``
  with ``K_i = [[f,0,(W-1)/2],[0,f,(H-1)/2],[0,0,1]]``, ``K_c = diag(f,f,1)`` and
  ``T_c`` moving the plane origin to the canvas centre;
* tangent-plane rig (for spans too wide for one plane): camera i maps by
  ``T(f*theta_i + c_x, c_y) K_c R_y(psi_i) K_i^-1`` with a small seeded yaw
  ``psi_i`` so that each map stays projective.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libsynth.so")
_lock = threading.Lock()
_lib = None

RECT_DTYPE = np.dtype(
    [("x0", "f8"), ("y0", "f8"), ("x1", "f8"), ("y1", "f8"), ("kind", "i4"), ("period", "i4"),
     ("ca", "f8", 3), ("cb", "f8", 3)], align=True)


def build(force: bool = False) -> str:
    """Compile ``synth.c`` into ``_build/libsynth.so`` (gcc, OpenMP when available)."""
    src = os.path.join(_HERE, "synth.c")
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(src):
        return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = f"{_LIB_PATH}.{os.getpid()}.tmp"
    base = ["gcc", "-O2", "-fPIC", "-shared", "-std=c99", src, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.synth_render_view.restype = ctypes.c_int
            lib.synth_render_view.argtypes = [
                ctypes.c_uint64, ctypes.c_double, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_void_p, ctypes.c_int64]
            lib.synth_render_view_cyl.restype = ctypes.c_int
            lib.synth_render_view_cyl.argtypes = [
                ctypes.c_uint64, ctypes.c_double, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                ctypes.c_double, ctypes.c_void_p, ctypes.c_int64]
            lib.synth_render_scene.restype = ctypes.c_int
            lib.synth_render_scene.argtypes = [
                ctypes.c_uint64, ctypes.c_double, ctypes.c_void_p, ctypes.c_int, ctypes.c_double,
                ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
            _lib = lib
    return _lib


@dataclass
class Scene:
    """A procedural scene: noise seed, lattice spacing, rectangles, scene offset of canvas (0,0)."""
    seed: int
    rects: np.ndarray
    off_x: float = 0.0
    off_y: float = 0.0
    lattice: float = 32.0
    shift_per_frame: float = 3.0


def make_scene(seed: int, x0: float, y0: float, width: float, height: float, n_rects: int,
               off_x: float = 0.0, off_y: float = 0.0, size_scale: float = 1.0) -> Scene:
    """Scene whose rectangles lie in [x0, x0+width) x [y0, y0+height) (scene px); rectangle sides
    are uniform in [16, 160] * size_scale px (at least 4 px)."""
    rng = np.random.default_rng(seed)
    r = np.zeros(max(n_rects, 0), dtype=RECT_DTYPE)
    if n_rects > 0:
        lo, hi = max(4.0, 16.0 * size_scale), max(8.0, 160.0 * size_scale)
        w = rng.uniform(lo, hi, n_rects)
        h = rng.uniform(lo, hi, n_rects)
        r["x0"] = x0 + rng.uniform(0.0, 1.0, n_rects) * (width - w)
        r["y0"] = y0 + rng.uniform(0.0, 1.0, n_rects) * (height - h)
        r["x1"] = r["x0"] + w
        r["y1"] = r["y0"] + h
        r["kind"] = rng.integers(0, 4, n_rects)
        r["period"] = rng.integers(3, 13, n_rects)
        r["ca"] = rng.uniform(0.0, 1.0, (n_rects, 3))
        r["cb"] = rng.uniform(0.0, 1.0, (n_rects, 3))
    return Scene(seed=int(seed), rects=r, off_x=off_x, off_y=off_y)


def render_view(scene: Scene, M: np.ndarray, W: int, H: int, t: int = 0,
                out: np.ndarray | None = None) -> np.ndarray:
    """Render frame ``t`` of a camera with camera->canvas homography ``M`` as HxWx3 uint8."""
    lib = _load()
    M = np.ascontiguousarray(M, dtype=np.float64).reshape(9)
    if out is None:
        out = np.empty((H, W, 3), dtype=np.uint8)
    assert out.shape == (H, W, 3) and out.dtype == np.uint8 and out.flags.c_contiguous
    rc = lib.synth_render_view(
        ctypes.c_uint64(scene.seed & 0xFFFFFFFFFFFFFFFF), scene.lattice,
        scene.rects.ctypes.data if len(scene.rects) else None, len(scene.rects), M.ctypes.data, W, H,
        scene.off_x - scene.shift_per_frame * t, scene.off_y, out.ctypes.data, W * 3)
    if rc != 0:
        raise ValueError(f"synth_render_view failed ({rc}): a pixel maps behind the camera")
    return out


def render_scene(scene: Scene, x0: float, y0: float, W: int, H: int) -> np.ndarray:
    lib = _load()
    out = np.empty((H, W, 3), dtype=np.uint8)
    lib.synth_render_scene(ctypes.c_uint64(scene.seed), scene.lattice,
                           scene.rects.ctypes.data if len(scene.rects) else None, len(scene.rects),
                           x0, y0, W, H, out.ctypes.data)
    return out


# ----------------------------------------------------------------------------------------------
# rig geometry


def _K(f: float, W: int, H: int) -> np.ndarray:
    return np.array([[f, 0.0, (W - 1) / 2.0], [0.0, f, (H - 1) / 2.0], [0.0, 0.0, 1.0]])


def _Ry(theta: float) -> np.ndarray:
    c, s = math.cos(theta), math.sin(theta)
    return np.array([[c, 0.0, s], [0.0, 1.0, 0.0], [-s, 0.0, c]])


def _T(tx: float, ty: float) -> np.ndarray:
    return np.array([[1.0, 0.0, tx], [0.0, 1.0, ty], [0.0, 0.0, 1.0]])


def _norm(M: np.ndarray) -> np.ndarray:
    return M / M[2, 2]


def render_view_cyl(scene: Scene, P: np.ndarray, W: int, H: int, canvas, t: int = 0) -> np.ndarray:
    """Render frame ``t`` of a camera with ray->camera matrix ``P`` (= K R) looking at a scene laid
    on the cylindrical canvas ``canvas`` = (f, cx, cy), as HxWx3 uint8."""
    lib = _load()
    Pinv = np.ascontiguousarray(np.linalg.inv(np.asarray(P, dtype=np.float64)), dtype=np.float64).reshape(9)
    out = np.empty((H, W, 3), dtype=np.uint8)
    f, cx, cy = (float(v) for v in canvas)
    rc = lib.synth_render_view_cyl(
        ctypes.c_uint64(scene.seed & 0xFFFFFFFFFFFFFFFF), scene.lattice,
        scene.rects.ctypes.data if len(scene.rects) else None, len(scene.rects), Pinv.ctypes.data, W, H, f, cx, cy,
        scene.off_x - scene.shift_per_frame * t, scene.off_y, out.ctypes.data, W * 3)
    if rc != 0:
        raise RuntimeError(f"synth_render_view_cyl failed ({rc})")
    return out


def rig_cylindrical(W: int, H: int, f: float, yaws_deg) -> list[np.ndarray]:
    """Ray->camera matrices P_i = K R_y(-yaw_i) of pinhole cameras rotating about the vertical axis
    (for a cylindrical canvas, whose column angle increases with x)."""
    K = _K(f, W, H)
    return [K @ _Ry(-math.radians(a)) for a in yaws_deg]


def rig_planar(W: int, H: int, f: float, yaws_deg, Wc: int, Hc: int) -> list[np.ndarray]:
    """Camera->canvas homographies of a rig of pinhole cameras rotating about the vertical axis,
    all projected onto one plane at focal length f, plane origin at the canvas centre."""
    Kc = np.diag([f, f, 1.0])
    Tc = _T((Wc - 1) / 2.0, (Hc - 1) / 2.0)
    Ki = np.linalg.inv(_K(f, W, H))
    return [_norm(Tc @ Kc @ _Ry(math.radians(a)) @ Ki) for a in yaws_deg]


def rig_tangent(W: int, H: int, f: float, spacing_deg: float, n: int, Hc: int, seed: int,
                psi_deg: float = 2.0, x_margin: float = 0.0) -> list[np.ndarray]:
    """Translated tangent planes: camera i is placed at canvas x = f*theta_i + (W-1)/2 + x_margin
    with a small seeded yaw psi_i in [-psi_deg, psi_deg] so that the map stays projective."""
    rng = np.random.default_rng(seed)
    psis = rng.uniform(-psi_deg, psi_deg, n)
    Kc = np.diag([f, f, 1.0])
    Ki = np.linalg.inv(_K(f, W, H))
    out = []
    for i in range(n):
        th = math.radians(spacing_deg * i)
        out.append(_norm(_T(f * th + (W - 1) / 2.0 + x_margin, (Hc - 1) / 2.0) @ Kc @ _Ry(math.radians(psis[i])) @ Ki))
    return out


# ----------------------------------------------------------------------------------------------
# workloads


@dataclass
class Camera:
    width: int
    height: int
    H: np.ndarray  # camera->canvas 3x3, H[2,2] == 1
    gain: float = 1.0


@dataclass
class RigConfig:
    name: str
    cameras: list
    canvas_w: int
    canvas_h: int
    levels: int
    frames: int
    scene: Scene
    extra: dict = field(default_factory=dict)

    @property
    def canvas(self):
        """None for a planar canvas, else (f, cx, cy) of the cylindrical canvas."""
        return self.extra.get("cylinder")

    def frame(self, t: int = 0) -> list[np.ndarray]:
        if self.canvas is not None:
            return [render_view_cyl(self.scene, c.H, c.width, c.height, self.canvas, t) for c in self.cameras]
        return [render_view(self.scene, c.H, c.width, c.height, t) for c in self.cameras]

    @property
    def canvas_mpix(self) -> float:
        return self.canvas_w * self.canvas_h / 1e6


def _scene_for(seed: int, Wc: int, Hc: int, frames: int, scale: float = 1.0, base_area: float = 1400.0 * 500.0,
               base_rects: int = 200, margin: int = 150) -> Scene:
    """Scene covering the canvas plus a margin and the sequence's total shift, with the density of
    200 rectangles per 1400x500 px; at a reduced ``scale`` rectangle sizes and the noise lattice
    shrink with it so that small test rigs keep texture in every overlap."""
    shift = 3.0 * max(frames - 1, 0)
    margin = int(round(margin * min(scale, 1.0)))
    width = Wc + 2 * margin + shift
    height = Hc + 2 * margin
    s2 = min(scale, 1.0)
    n = int(round(base_rects * width * height / (base_area * s2 * s2)))
    # scene coordinate of canvas (0,0) is (margin + shift, margin): frame t shows scene x - 3t
    sc = make_scene(seed, 0.0, 0.0, width, height, n, off_x=margin + shift, off_y=margin, size_scale=s2)
    sc.lattice = max(4.0, 32.0 * s2)
    return sc


def _scaled(v: float, s: float, odd: bool = False) -> int:
    r = max(1, int(round(v * s)))
    if odd and r % 2 == 0:
        r += 1
    return r


def config_cyl(scale: float = 1.0, seed: int = 0, frames: int = 1) -> RigConfig:
    """Four 1280x720 cameras (f = 900) at yaws -45, -15, 15, 45 deg on a cylindrical canvas of focal
    length 900: 2528x760, 5 levels; the scene translates 3 px per frame along the canvas."""
    W, H = _scaled(1280, scale), _scaled(720, scale)
    f = 900.0 * scale
    Wc, Hc = _scaled(2528, scale, odd=scale != 1.0), _scaled(760, scale, odd=scale != 1.0)
    canvas = (f, (Wc - 1) / 2.0, (Hc - 1) / 2.0)
    Ps = rig_cylindrical(W, H, f, [-45.0, -15.0, 15.0, 45.0])
    return RigConfig("cyl_4x720p", [Camera(W, H, P) for P in Ps], Wc, Hc, 5, frames,
                     _scene_for(seed, Wc, Hc, frames, scale), {"cylinder": canvas})


def config_2cam(scale: float = 1.0, seed: int = 0) -> RigConfig:
    """Two 640x360 cameras, f=500, yaw -12/+12 deg, canvas 1100x400, 4 levels, one frame.
    Scene 1400x500 with 200 textured rectangles; canvas (0,0) sits at scene (150, 50)."""
    W, H = _scaled(640, scale), _scaled(360, scale)
    Wc, Hc = _scaled(1100, scale, odd=scale != 1.0), _scaled(400, scale, odd=scale != 1.0)
    f = 500.0 * scale
    Ms = rig_planar(W, H, f, [-12.0, 12.0], Wc, Hc)
    if scale == 1.0:
        scene = make_scene(seed, 0.0, 0.0, 1400.0, 500.0, 200, off_x=150.0, off_y=50.0)
    else:
        scene = _scene_for(seed, Wc, Hc, 1, scale)
    return RigConfig("2cam_640x360", [Camera(W, H, M) for M in Ms], Wc, Hc, 4, 1, scene)


def config_4x1080p(scale: float = 1.0, seed: int = 0, frames: int = 60) -> RigConfig:
    """Four 1920x1080 cameras, f=1400, yaw spacing 25 deg, canvas 5200x1300, 5 levels, a sequence
    in which the scene translates 3 px per frame."""
    W, H = _scaled(1920, scale), _scaled(1080, scale)
    Wc, Hc = _scaled(5200, scale, odd=scale != 1.0), _scaled(1300, scale, odd=scale != 1.0)
    f = 1400.0 * scale
    Ms = rig_planar(W, H, f, [-37.5, -12.5, 12.5, 37.5], Wc, Hc)
    return RigConfig("4x1080p", [Camera(W, H, M) for M in Ms], Wc, Hc, 5, frames,
                     _scene_for(seed, Wc, Hc, frames, scale))


def config_8x4k(scale: float = 1.0, seed: int = 0, frames: int = 30) -> RigConfig:
    """Eight 3840x2160 cameras, 40 deg spacing, f=4125 (span 280 deg -> ~24000 px), canvas
    24000x2600, 6 levels, translated tangent planes with seeded +-2 deg yaw."""
    W, H = _scaled(3840, scale), _scaled(2160, scale)
    Wc, Hc = _scaled(24000, scale, odd=scale != 1.0), _scaled(2600, scale, odd=scale != 1.0)
    f = 4125.0 * scale
    Ms = rig_tangent(W, H, f, 40.0, 8, Hc, seed)
    return RigConfig("8x4k", [Camera(W, H, M) for M in Ms], Wc, Hc, 6, frames,
                     _scene_for(seed, Wc, Hc, frames, scale))


def config_refine(scale: float = 1.0, seed: int = 0) -> RigConfig:
    """Four 1920x1080 cameras at 25 deg spacing (f=1400, canvas 5200x1300): true homographies for
    the alignment-refinement workload."""
    cfg = config_4x1080p(scale, seed, frames=1)
    cfg.name = "refine_4x1080p"
    return cfg


RESOLUTIONS = [(1280, 720), (1920, 1080), (3840, 2160)]


def config_batch(n_rigs: int = 16, seed: int = 0, scale: float = 1.0) -> list[RigConfig]:
    """Independent rigs with uneven sizes drawn from a seed: 2-6 cameras, one resolution per rig
    from {1280x720, 1920x1080, 3840x2160}, yaw spacing 20-30 deg, 4-6 pyramid levels.
    Each view covers 1.4x the yaw spacing, so neighbours overlap by ~30% of a view."""
    rng = np.random.default_rng(1000 + seed)
    rigs = []
    for k in range(n_rigs):
        n = int(rng.integers(2, 7))
        W0, H0 = RESOLUTIONS[int(rng.integers(0, 3))]
        W, H = _scaled(W0, scale), _scaled(H0, scale)
        spacing = float(rng.uniform(20.0, 30.0))
        L = int(rng.integers(4, 7))
        fov = math.radians(1.4 * spacing)
        f = (W / 2.0) / math.tan(fov / 2.0)
        margin_y = int(round(0.1 * H))
        Hc = H + 2 * margin_y
        Wc = int(math.ceil(f * math.radians(spacing) * (n - 1) + W + 2 * 16))
        Ms = rig_tangent(W, H, f, spacing, n, Hc, seed * 7919 + k, x_margin=16.0)
        rigs.append(RigConfig(f"batch{k}", [Camera(W, H, M) for M in Ms], Wc, Hc, L, 1,
                              _scene_for(seed * 7919 + k, Wc, Hc, 1, scale), {"spacing": spacing, "f": f}))
    return rigs


CONFIGS = {
    "2cam_640x360": config_2cam,
    "4x1080p": config_4x1080p,
    "refine_4x1080p": config_refine,
    "8x4k": config_8x4k,
}


def brief_pattern(seed: int = 0, n: int = 256) -> np.ndarray:
    """BRIEF point pairs (n, 4) int8 (px, py, qx, qy): isotropic Gaussian offsets with sigma =
    31/5 px, rounded and clipped to the 31 x 31 patch [-15, 15]^2, seeded."""
    rng = np.random.default_rng(seed)
    return np.clip(np.rint(rng.normal(0.0, 31.0 / 5.0, (n, 4))), -15, 15).astype(np.int8)


def lsh_bits(seed: int = 0, tables: int = 8, bits: int = 16) -> np.ndarray:
    """Bit positions of the LSH tables: (tables, bits) distinct positions of 256 per table, seeded."""
    rng = np.random.default_rng(seed)
    return np.stack([rng.choice(256, bits, replace=False) for _ in range(tables)]).astype(np.uint8)


def prosac_words(seed: int = 0, iters: int = 1024) -> np.ndarray:
    """Random words of the PROSAC samples: (iters, 4) uint32, seeded."""
    return np.random.default_rng(seed).integers(0, 2 ** 32, (iters, 4), dtype=np.uint64).astype(np.uint32)
