"""Step B of the oracle: tile lists, their depth order and tile ranges (test infrastructure).

The paper's rasterizer (Sec. 3.1; Sec. 5.2 recalls that the 3DGS
preprocessing culls every Gaussian that reaches no tile) splits the image into
16x16 tiles and gives every tile the depth-ordered list of the Gaussians that
touch it.  The reading adopted here:

  * Gaussian i touches pixel x iff o_i G_i(x) >= alpha_min, i.e.
    q(x) = d^T conic d <= tau_i = 2 ln(o_i / alpha_min), d = x - mean2d;
  * tile T (pixel centres [16 tx + 0.5, 16 tx + 15.5] x [16 ty + 0.5,
    16 ty + 15.5], whether or not they fall inside the image) is kept iff the
    minimum of q over that rectangle is <= tau_i;
  * the candidate tiles are limited to the image's tile grid;
  * keys are (view_tile_base + ty * tiles_x + tx, float32 bits of z); the sort
    is stable with input order (view, Gaussian index, tiles row-major), so
    ties in z fall back to ascending Gaussian index.

The alternative "3sigma" extent (the tile extent of the 3DGS rasterizer the
paper builds on, Sec. 3.1) lists Gaussian i in every tile whose pixel-centre
rectangle meets the square [mx - r, mx + r] x [my - r, my + r] with
r = ceil(3 sqrt(lambda_max)), lambda_max the larger eigenvalue of the 2-D
covariance; no ellipse test.  Rendering keeps the per-pixel alpha rule, so the
support is truncated to those tiles.

These functions take the FP32 projected state as numbers (for the parity check
they are handed the CUDA path's own stage-P outputs) and decide in float64.
"""
from __future__ import annotations

import math

import numpy as np


def rect_min_q(A, B, C, mx, my, x0, x1, y0, y1):
    """Exact minimum of q(x, y) = A dx^2 + 2B dx dy + C dy^2, d = (x - mx, y - my),
    over the rectangle [x0, x1] x [y0, y1], for a positive-definite [[A,B],[B,C]].

    0 if the centre is inside; otherwise the minimum lies on an edge, and on
    each edge q is a 1-D convex quadratic minimised by clamping its vertex.
    The tile test of Sec. 3.1 under the exact-support reading."""
    A, B, C, mx, my, x0, x1, y0, y1 = np.broadcast_arrays(
        *(np.asarray(a, np.float64) for a in (A, B, C, mx, my, x0, x1, y0, y1)))
    inside = (mx >= x0) & (mx <= x1) & (my >= y0) & (my <= y1)
    best = np.full(A.shape, np.inf)
    for X in (x0, x1):                   # vertical edges: dx fixed
        dx = X - mx
        dy = np.clip(-B * dx / C, y0 - my, y1 - my)
        best = np.minimum(best, A * dx * dx + 2 * B * dx * dy + C * dy * dy)
    for Y in (y0, y1):                   # horizontal edges: dy fixed
        dy = Y - my
        dx = np.clip(-B * dy / A, x0 - mx, x1 - mx)
        best = np.minimum(best, A * dx * dx + 2 * B * dx * dy + C * dy * dy)
    return np.where(inside, 0.0, best)


def lambda_max(sxx, syy, sxy):
    """Larger eigenvalue of the symmetric 2x2 matrix [[sxx, sxy], [sxy, syy]]:
    the mean of the diagonal plus the half-difference's hypotenuse with sxy.
    Used by the 3-sigma extent of the 3DGS rasterizer recalled in Sec. 3.1."""
    sxx, syy, sxy = (np.asarray(a, np.float64) for a in (sxx, syy, sxy))
    return 0.5 * (sxx + syy) + np.hypot(0.5 * (sxx - syy), sxy)


def three_sigma_radius(sxx, syy, sxy):
    """r = ceil(3 sqrt(lambda_max)) of a 2-D covariance (the 3-sigma extent).
    The 3-sigma extent of the 3DGS rasterizer recalled in Sec. 3.1."""
    return np.ceil(3.0 * np.sqrt(lambda_max(sxx, syy, sxy)))


def square_tile_range(m, r, n_tiles, tile=16):
    """First and last tile index t (clipped to [0, n_tiles - 1]) whose pixel
    centres [tile t + 0.5, tile t + tile - 0.5] meet [m - r, m + r]; last <
    first when none does.  Tile range of the 3-sigma square (Sec. 3.1, 3-sigma extent)."""
    m, r = np.asarray(m, np.float64), np.asarray(r, np.float64)
    lo = np.ceil((m - r - (tile - 0.5)) / tile)
    hi = np.floor((m + r - 0.5) / tile)
    return np.maximum(lo, 0).astype(np.int64), np.minimum(hi, n_tiles - 1).astype(np.int64)


def _square_lists(mean2d, conic, ok, tx_n, ty_n, tile, eps):
    """Tile lists of the 3-sigma extent; `near` / rejected entries are those
    whose membership changes when r (through 3 sqrt(lambda_max)) or the centre
    moves by eps relative."""
    A, B, C = conic[:, 0], conic[:, 1], conic[:, 2]
    with np.errstate(divide="ignore", invalid="ignore"):
        det = A * C - B * B
        sxx = np.where(ok, C / det, 1.0)            # the covariance is the inverse conic
        syy = np.where(ok, A / det, 1.0)
        sxy = np.where(ok, -B / det, 0.0)
    s3 = 3.0 * np.sqrt(lambda_max(sxx, syy, sxy))
    mx = np.where(ok, mean2d[:, 0], 0.0)
    my = np.where(ok, mean2d[:, 1], 0.0)

    def tiles_of(r, dx, dy):
        x0, x1 = square_tile_range(mx + dx, r, tx_n, tile)
        y0, y1 = square_tile_range(my + dy, r, ty_n, tile)
        out = []
        for i in np.nonzero(ok)[0]:
            out.extend((int(i), int(ty) * tx_n + int(tx))
                       for ty in range(y0[i], y1[i] + 1) for tx in range(x0[i], x1[i] + 1))
        return set(out)

    nominal = tiles_of(np.ceil(s3), 0.0, 0.0)
    shift = eps * np.maximum(1.0, np.abs(mx) + np.abs(my))
    variants = [tiles_of(np.ceil(s3 * f), sx * shift, sy * shift)
                for f in (1.0 - eps, 1.0 + eps) for sx in (-1, 1) for sy in (-1, 1)]
    sure = set.intersection(nominal, *variants)
    either = set.union(nominal, *variants)
    kept = sorted(nominal)
    g_all = np.asarray([g for g, _ in kept], np.int64)
    t_all = np.asarray([t for _, t in kept], np.int64)
    near = np.asarray([e not in sure for e in kept], bool)
    rej = sorted(either - nominal)
    return (g_all, t_all, near, np.asarray([g for g, _ in rej], np.int64),
            np.asarray([t for _, t in rej], np.int64))


def tile_lists(mean2d, conic, opacity, valid, width, height, alpha_min=1.0 / 255.0,
               tile=16, eps=1e-4, extent="exact"):
    """Per-Gaussian touched tiles for one view.

    mean2d [N,2], conic [N,3], opacity [N] (numbers; converted to float64),
    valid [N] bool.  Returns (gauss [E], tiles [E], near [E]) in the order
    (Gaussian index, tiles row-major), where `near` marks entries whose
    decision is within eps (relative to tau) of the boundary, and a second
    array of near-boundary *rejected* candidates (gauss, tiles) for the
    same tolerance.  extent="3sigma" gives the lists of the 3-sigma square
    instead (see the module docstring).  The per-tile binning of Sec. 3.1."""
    mean2d = np.asarray(mean2d, np.float64)
    conic = np.asarray(conic, np.float64)
    opacity = np.asarray(opacity, np.float64)
    valid = np.asarray(valid, bool)
    tx_n = (width + tile - 1) // tile
    ty_n = (height + tile - 1) // tile
    with np.errstate(divide="ignore", invalid="ignore"):
        tau = 2.0 * np.log(opacity / alpha_min)
    ok = valid & (tau > 0)
    A, B, C = conic[:, 0], conic[:, 1], conic[:, 2]
    det = A * C - B * B
    ok &= det > 0
    if extent == "3sigma":
        return _square_lists(np.asarray(mean2d, np.float64), np.asarray(conic, np.float64), ok,
                             tx_n, ty_n, tile, 0.1 * eps)
    with np.errstate(divide="ignore", invalid="ignore"):
        sxx = np.where(ok, C / det, 0.0)       # inverse conic = 2-D covariance
        syy = np.where(ok, A / det, 0.0)
    tau_ok = np.where(ok, tau, 0.0)
    rx = np.sqrt(tau_ok * sxx)
    ry = np.sqrt(tau_ok * syy)
    # generous candidate range (one extra tile each side), clipped to the grid;
    # items that are not kept (their centre may be undefined) get an empty one
    mx = np.where(ok, mean2d[:, 0], 0.0)
    my = np.where(ok, mean2d[:, 1], 0.0)
    tx0 = np.clip(np.floor((mx - rx - 15.5) / tile) - 1, 0, tx_n - 1)
    tx1 = np.clip(np.floor((mx + rx - 0.5) / tile) + 1, 0, tx_n - 1)
    ty0 = np.clip(np.floor((my - ry - 15.5) / tile) - 1, 0, ty_n - 1)
    ty1 = np.clip(np.floor((my + ry - 0.5) / tile) + 1, 0, ty_n - 1)
    g_all, t_all, near_all, rej_g, rej_t = [], [], [], [], []
    idx = np.nonzero(ok)[0]
    nx = (tx1 - tx0 + 1).astype(np.int64)
    ny = (ty1 - ty0 + 1).astype(np.int64)
    cnt = (nx * ny)[idx]
    if len(idx):
        g = np.repeat(idx, cnt)
        start = np.repeat(np.cumsum(cnt) - cnt, cnt)
        k = np.arange(len(g)) - start
        tyy = ty0[g].astype(np.int64) + k // nx[g]
        txx = tx0[g].astype(np.int64) + k % nx[g]
        m = rect_min_q(A[g], B[g], C[g], mean2d[g, 0], mean2d[g, 1],
                       txx * tile + 0.5, txx * tile + tile - 0.5,
                       tyy * tile + 0.5, tyy * tile + tile - 0.5)
        keep = m <= tau[g]
        near = np.abs(m - tau[g]) <= eps * np.maximum(tau[g], 1.0)
        g_all, t_all, near_all = g[keep], tyy[keep] * tx_n + txx[keep], near[keep]
        rej_g, rej_t = g[~keep & near], (tyy * tx_n + txx)[~keep & near]
    return (np.asarray(g_all, np.int64), np.asarray(t_all, np.int64),
            np.asarray(near_all, bool), np.asarray(rej_g, np.int64),
            np.asarray(rej_t, np.int64))


def sort_entries(tile_id, z32, gauss):
    """Stable order of (tile, z) keys: ascending global tile id, then
    ascending float32 bit pattern of z (equal to ascending z for z > 0), then
    input order.  Inputs are listed in (view, Gaussian, tile row-major) order.
    Returns the permutation.  Sec. 3.1: every tile lists its Gaussians in depth order."""
    zb = np.asarray(z32, np.float32).view(np.uint32).astype(np.uint64)
    key = (np.asarray(tile_id, np.uint64) << np.uint64(32)) | zb
    return np.argsort(key, kind="stable")


def tile_ranges(sorted_tile_ids, total_tiles):
    """[start, end) of every global tile in the sorted entry list.
    Sec. 3.1: each tile reads its own run of the sorted list."""
    t = np.asarray(sorted_tile_ids, np.int64)
    ids = np.arange(total_tiles)
    return np.stack([np.searchsorted(t, ids, "left"), np.searchsorted(t, ids, "right")], 1)


def tile_grid(width, height, tile=16):
    """Tiles across and down one view (16x16-pixel tiles, Sec. 3.1)."""
    return (width + tile - 1) // tile, (height + tile - 1) // tile


def view_tile_bases(sizes, tile=16):
    """Global tile-id base of every view when views are concatenated.
    Batching of several views into one list: no counterpart in the paper."""
    bases, acc = [], 0
    for (w, h) in sizes:
        bases.append(acc)
        tx, ty = tile_grid(w, h, tile)
        acc += tx * ty
    return bases, acc


def exclusive_scan(counts):
    """Offsets of a concatenation: out[k] = sum_{j<k} counts[j].
    The entry offsets of the binning of Sec. 3.1."""
    c = np.asarray(counts, np.int64)
    return np.concatenate([[0], np.cumsum(c)[:-1]]) if len(c) else c


def ceil_log2(n: int) -> int:
    """Bits of the global tile id, the sort key of Sec. 3.1."""
    return max(0, math.ceil(math.log2(max(n, 1))))
