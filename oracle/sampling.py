"""Primitive sampling (Sec. 4.3) and depth-reinitialization seeds (Sec. 4.2)
(test infrastructure; used only by the tests, the smoke check and the
benchmark's CPU-baseline leg).

weighted_sample(I, E, k)
    k Gaussians drawn without replacement with probability proportional to
    their importance, P_i = I_i / sum_j I_j (Sec. 4.3).  Method: exponential
    clocks (Efraimidis and Spirakis, weighted random sampling): Gaussian i
    rings at E_i / I_i with E_i ~ Exp(1), and the first k to ring are the
    sample -- the same law as k successive proportional draws.  The draws E
    are inputs.  Equivalently the k largest keys I_i / E_i; the key is formed
    in single precision (the precision the selection is decided in), ties go
    to the lower index, Gaussians with I_i = 0 never ring, and the indices are
    returned ascending.

depth_points(depth, imax, target, u, cam, k)
    Sec. 4.2: the rendered depth map (d^mid) is reprojected to world space and
    a random subset of the points, coloured from the ground-truth image, seeds
    the reinitialization.  Reading: the candidates are the pixels with a
    maximum contributor and d^mid > 0; k of them are drawn uniformly without
    replacement, as the k largest of the uniform draws u (inputs); a pixel
    (x, y) at depth d is the camera point d ((x + 0.5 - cx) / fx,
    (y + 0.5 - cy) / fy, 1) (the ray the renderer sampled), mapped to world
    space by the inverse of p_c = R p + t.
"""
from __future__ import annotations

import numpy as np


def _top_k_positive(key: np.ndarray, k: int) -> np.ndarray:
    pos = np.nonzero(key > 0)[0]
    order = pos[np.lexsort((pos, -key[pos]))]          # descending key, then index
    return np.sort(order[:min(k, len(pos))])


def weighted_sample(I, E, k: int) -> np.ndarray:
    key = (np.asarray(I, np.float32) / np.asarray(E, np.float32)).astype(np.float64)
    return _top_k_positive(key, k)


def reproject(depth, pix, cam) -> np.ndarray:
    """World points of view-local pixels pix (y W + x) at depths depth[pix].
    The reprojection of the depth map to world space (Sec. 4.2)."""
    pix = np.asarray(pix, np.int64)
    x, y = pix % cam.width, pix // cam.width
    d = np.asarray(depth, np.float64)[pix]
    pc = np.stack([d * (x + 0.5 - cam.cx) / cam.fx, d * (y + 0.5 - cam.cy) / cam.fy, d], 1)
    R, t = np.asarray(cam.R, np.float64), np.asarray(cam.t, np.float64)
    return (pc - t) @ R                                  # R^T (p_c - t), row-wise


def depth_points(depth, imax, target, u, cam, k: int) -> dict:
    depth = np.asarray(depth, np.float64)
    valid = (np.asarray(imax) >= 0) & (depth > 0)
    pix = _top_k_positive(np.where(valid, np.asarray(u, np.float64), 0.0), k)
    img = np.asarray(target, np.float64).reshape(3, -1)
    return {"pixel_idx": pix, "points": reproject(depth, pix, cam), "colours": img[:, pix].T}
