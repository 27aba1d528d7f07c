"""Helpers for GPU-vs-oracle parity tests.

Tolerances (from the accuracy targets of the path): uint8 output within 1 LSB of the oracle's
round-half-even result; float output within 2e-4 absolute (1e-3 with FP16 pyramid storage).
Pixels whose oracle source coordinate lies within 1e-2 px of a camera's validity border are
excluded (reading C9: coverage flips between FP32 and FP64 there); their count is returned.
"""
from __future__ import annotations

import numpy as np

import oracle

TOL_F32 = 2e-4
TOL_F16 = 1e-3
BORDER_EXCLUDE = 1e-2


def gpu_frames(frames):
    import torch
    return [torch.from_numpy(np.ascontiguousarray(f)).cuda() for f in frames]


def run_gpu(cfg, frames, path="plain", out_float=True, band_fp16=False, levels=None):
    import torch
    from paper_1810_03988_gb300 import Rig
    L = cfg.levels if levels is None else levels
    with Rig(cfg.cameras, cfg.canvas_w, cfg.canvas_h, L, band_fp16=band_fp16, out_float=out_float,
             path=path) as rig:
        out = rig.stitch(gpu_frames(frames))
        torch.cuda.synchronize()
        return out.cpu().numpy()


def compare(got: np.ndarray, ref: dict, out_float: bool, tol: float | None = None):
    """Compare a GPU canvas (window) with an oracle result dict; returns a stats dict, raises on failure."""
    keep = ref["mindist"] >= BORDER_EXCLUDE
    excluded = int((~keep).sum())
    if out_float:
        tol = TOL_F32 if tol is None else tol
        err = np.abs(got.astype(np.float64) - ref["out"])
        worst = float(err[keep].max()) if keep.any() else 0.0
        assert worst <= tol, f"max abs error {worst:.3e} > {tol:.1e} (excluded {excluded} border pixels)"
        return {"max_abs": worst, "excluded": excluded, "pixels": int(keep.sum())}
    d = np.abs(got.astype(np.int32) - ref["u8"].astype(np.int32))
    worst = int(d[keep].max()) if keep.any() else 0
    assert worst <= 1, f"max LSB difference {worst} (excluded {excluded} border pixels)"
    return {"max_lsb": worst, "lsb1": int((d[keep] == 1).sum()), "excluded": excluded, "pixels": int(keep.sum())}


def full_parity(cfg, frames, path="plain", out_float=True, band_fp16=False, levels=None, tol=None):
    L = cfg.levels if levels is None else levels
    ref = oracle.forward(cfg.cameras, frames, cfg.canvas_w, cfg.canvas_h, L)
    got = run_gpu(cfg, frames, path, out_float, band_fp16, L)
    return compare(got, ref, out_float, tol)


def sample_windows(cfg, n: int, size: int, seed: int = 0):
    """Windows of the canvas chosen to cover overlaps, coverage borders and canvas corners."""
    rng = np.random.default_rng(seed)
    Wc, Hc = cfg.canvas_w, cfg.canvas_h
    s = min(size, Wc, Hc)
    wins = [(0, 0, s, s), (Wc - s, Hc - s, s, s), (0, Hc - s, s, s), (Wc - s, 0, s, s)]
    # seams: midpoint between neighbouring camera centres, at the top border, middle and bottom
    centres = []
    for c in cfg.cameras:
        p = np.asarray(c.H) @ np.array([(c.width - 1) / 2, (c.height - 1) / 2, 1.0])
        centres.append(p[:2] / p[2])
    centres.sort(key=lambda q: q[0])
    for a, b in zip(centres[:-1], centres[1:]):
        mx = int((a[0] + b[0]) / 2)
        for fy in (0.12, 0.5, 0.88):
            wins.append((int(np.clip(mx - s // 2, 0, Wc - s)), int(np.clip(fy * Hc - s // 2, 0, Hc - s)), s, s))
    while len(wins) < n:
        wins.append((int(rng.integers(0, Wc - s + 1)), int(rng.integers(0, Hc - s + 1)), s, s))
    return wins[:max(n, len(wins))]
