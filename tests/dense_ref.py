"""Independent dense-matrix formulation of the pyramid operators, used to pin the oracle.

The oracle evaluates REDUCE/EXPAND as per-pixel index loops.  Here the same operators are built
as explicit 1-D matrices (one row per output sample) and applied as ``R_y @ G @ R_x.T``: a
different formulation whose only shared ingredients are the operator definitions themselves
(5-tap [1,4,6,4,1]/16 kernel, decimation at even indices, reflect-101 borders, EXPAND weights
2w(x-2k)).  Agreement of the two to rounding level pins the loop code (index arithmetic, phase,
border folding, transposed axes).
"""
from __future__ import annotations

import numpy as np

W5 = np.array([1.0, 4.0, 6.0, 4.0, 1.0]) / 16.0


def reflect101(i: int, n: int) -> int:
    # written as explicit repeated mirroring (not the modular form the oracle uses)
    if n == 1:
        return 0
    while i < 0 or i >= n:
        if i < 0:
            i = -i
        if i >= n:
            i = 2 * (n - 1) - i
    return i


def reduce_matrix(n: int) -> np.ndarray:
    nc = (n + 1) // 2
    R = np.zeros((nc, n))
    for k in range(nc):
        for m in range(-2, 3):
            R[k, reflect101(2 * k + m, n)] += W5[m + 2]
    return R


def expand_matrix(n: int) -> np.ndarray:
    nc = (n + 1) // 2
    E = np.zeros((n, nc))
    for x in range(n):
        for k in range(-2, nc + 2):
            d = x - 2 * k
            if -2 <= d <= 2:
                E[x, reflect101(k, nc)] += 2.0 * W5[d + 2]
    return E


def reduce2d(img: np.ndarray) -> np.ndarray:
    h, w = img.shape[:2]
    Ry, Rx = reduce_matrix(h), reduce_matrix(w)
    if img.ndim == 2:
        return Ry @ img @ Rx.T
    return np.einsum("ky,yxc,jx->kjc", Ry, img, Rx)


def expand2d(img: np.ndarray, shape) -> np.ndarray:
    h, w = shape
    Ey, Ex = expand_matrix(h), expand_matrix(w)
    assert Ey.shape[1] == img.shape[0] and Ex.shape[1] == img.shape[1]
    if img.ndim == 2:
        return Ey @ img @ Ex.T
    return np.einsum("yk,kjc,xj->yxc", Ey, img, Ex)


def gaussian(img: np.ndarray, levels: int) -> list:
    g = [np.asarray(img, dtype=np.float64)]
    for _ in range(levels - 1):
        g.append(reduce2d(g[-1]))
    return g
