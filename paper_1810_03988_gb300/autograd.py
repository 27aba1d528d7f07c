"""torch.autograd wrapper of the hand-written backward kernel, and alignment refinement.

``StitchLoss.apply(params, rig, frames)`` returns the overlap photometric loss (S7) for per-camera
canvas->camera parameters ``params`` (N x 9 float64 tensor: a11..a32, gain; a33 is the rig's ±1;
on any device, moved to the frames' GPU for the kernel); its backward is the gradient computed by
``stitch_backward`` in the same call, on the parameters' device.

Refinement (the "gradient-refined homographies" use of S7): each camera's homography is
parametrised by the canvas positions of its four image corners (8 numbers, px) and a gain; the
camera->canvas homography follows by the direct linear transform, its inverse gives the kernel's
parameters, and torch applies the chain rule from the kernel's gradient to the corners.  Camera 0
is held fixed (gauge: otherwise all gains can shrink to 0 and a common motion of every camera
leaves the loss unchanged).
"""
from __future__ import annotations

import numpy as np
import torch

from .stitch import Rig


class StitchLoss(torch.autograd.Function):
    """loss = sum over canvas pixels and camera pairs i<j valid at the pixel of |I_i - I_j|^2."""

    @staticmethod
    def forward(ctx, params: torch.Tensor, rig: Rig, frames):
        # the kernel runs on the frames' device; loss and gradient return to the parameters' device
        p = params.detach().to(frames[0].device).contiguous()
        loss, grad = rig.backward(frames, p)
        ctx.save_for_backward(grad.to(params.device))
        return loss[0].to(params.device)

    @staticmethod
    def backward(ctx, gout):
        (grad,) = ctx.saved_tensors
        return gout * grad, None, None


def image_corners(width: int, height: int, dtype=torch.float64, device=None) -> torch.Tensor:
    """Source corners (u, v) of an image, centres of the corner pixels: (4, 2)."""
    return torch.tensor([[0.0, 0.0], [width - 1.0, 0.0], [width - 1.0, height - 1.0], [0.0, height - 1.0]],
                        dtype=dtype, device=device)


def corners_of(H: np.ndarray, width: int, height: int) -> np.ndarray:
    """Canvas positions of the image corners under camera->canvas H: (4, 2)."""
    src = image_corners(width, height).numpy()
    p = np.c_[src, np.ones(4)] @ np.asarray(H, dtype=np.float64).T
    return p[:, :2] / p[:, 2:3]


def homography_from_corners(src: torch.Tensor, dst: torch.Tensor) -> torch.Tensor:
    """Direct linear transform: the 3x3 H (h33 = 1) with H (u, v, 1) ~ (x, y, 1) for 4 pairs."""
    rows, rhs = [], []
    for k in range(4):
        u, v = src[k, 0], src[k, 1]
        x, y = dst[k, 0], dst[k, 1]
        one, zero = torch.ones_like(u), torch.zeros_like(u)
        rows.append(torch.stack([u, v, one, zero, zero, zero, -u * x, -v * x]))
        rows.append(torch.stack([zero, zero, zero, u, v, one, -u * y, -v * y]))
        rhs += [x, y]
    h = torch.linalg.solve(torch.stack(rows), torch.stack(rhs))
    return torch.cat([h, torch.ones_like(h[:1])]).reshape(3, 3)


def params_from_corners(corners: torch.Tensor, gains: torch.Tensor, sizes, a33_signs) -> torch.Tensor:
    """(N, 4, 2) canvas corner positions + (N,) gains -> (N, 9) kernel parameters."""
    out = []
    for i, (w, h) in enumerate(sizes):
        H = homography_from_corners(image_corners(w, h, corners.dtype, corners.device), corners[i])
        A = torch.linalg.inv(H)
        A = A / A[2, 2].abs()
        if float(A[2, 2].detach()) * a33_signs[i] < 0:
            raise ValueError("camera moved so far that the canvas origin changed sides of its horizon")
        out.append(torch.cat([A.reshape(9)[:8], gains[i:i + 1]]))
    return torch.stack(out)


def refine(rig: Rig, frames, corners0: np.ndarray, gains0: np.ndarray, steps: int = 50, lr_px: float = 0.25,
           lr_gain: float = 0.01, fixed=(0,), callback=None):
    """Adam on corner offsets (px) and gains, gradient from the hand-written backward kernel.

    The corner -> parameter chain (4-point DLT and inverse per camera, a few hundred scalar
    operations) and the optimiser run on the host; each step moves the (N, 9) parameters to the
    GPU, runs the loss/gradient kernel there and brings the gradient back.

    Returns (corners, gains, history) with history a list of loss values (one per step, before the
    update of that step)."""
    dev = torch.device("cpu")
    n = len(rig.cameras)
    sizes = [(c.width, c.height) for c in rig.cameras]
    signs = [float(rig.camera_map(i)[0][2, 2]) for i in range(n)]
    base = torch.tensor(np.asarray(corners0, dtype=np.float64), device=dev)
    offs = torch.zeros_like(base, requires_grad=True)
    g = torch.tensor(np.asarray(gains0, dtype=np.float64), device=dev, requires_grad=True)
    free = torch.ones(n, dtype=torch.float64, device=dev)
    for i in fixed:
        free[i] = 0.0
    opt = torch.optim.Adam([{"params": [offs], "lr": lr_px}, {"params": [g], "lr": lr_gain}])
    history = []
    for it in range(steps):
        opt.zero_grad()
        corners = base + offs * free[:, None, None]
        gains = g * free + (1 - free) * g.detach()
        params = params_from_corners(corners, gains, sizes, signs)
        loss = StitchLoss.apply(params, rig, frames)
        loss.backward()
        history.append(float(loss.detach()))
        if callback:
            callback(it, history[-1])
        opt.step()
    with torch.no_grad():
        corners = (base + offs * free[:, None, None]).cpu().numpy()
        gains = g.detach().cpu().numpy()
    return corners, gains, history
