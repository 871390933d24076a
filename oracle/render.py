"""Step R of the oracle: per-pixel alpha blending and its side outputs (test infrastructure).

Written from the paper:
  * Eq. 1 (Sec. 3.1): c(x) = sum_i w_i c_i, w_i = T_i alpha_i G2D_i(x),
    T_i = prod_{j<i} (1 - alpha_j G2D_j(x)), Gaussians taken in the depth order
    of their centres;
  * Sec. 3.2: I_i = sum over rays of w_i (importance / accumulated weight);
  * Eq. 2 (Sec. 3.3) and Sec. 4.1: i_max(x) = argmax_i w_i, the midpoint depth
    d^mid_{i_max}(x), the blended depth d^blend = sum_i w_i d_i and the
    maximum-contribution area S_i = #{x : i_max(x) = i}.

Here "alpha_i G2D_i(x)" is evaluated as alpha = min(alpha_max, o_i G_i(x)) and
an entry with alpha < alpha_min is skipped; compositing stops before the
first entry whose blend would bring the transmittance below t_min (that entry
is not blended).  The depth order is ascending float32(z) with ties broken
by ascending Gaussian index.  Pixels with no blended entry get i_max = -1,
w_max = 0 and depth 0.

This is a brute-force renderer: every pixel considers every Gaussian.  It is
dense over [pixels x Gaussians] in chunks, float64, and differentiable by
torch.autograd with respect to the Gaussian parameters.
"""
from __future__ import annotations

import numpy as np
import torch

from .config import OracleConfig
from .project import project, midpoint_depth, f64


def depth_order(z: torch.Tensor, valid: torch.Tensor) -> np.ndarray:
    """Indices of the valid Gaussians in compositing order: ascending
    float32(z), ties by ascending index (Sec. 3.1 depth ordering)."""
    zf = z.detach().numpy().astype(np.float32)
    idx = np.nonzero(valid.numpy())[0]
    order = np.lexsort((idx, zf[idx]))
    return idx[order]


def composite(alpha_raw: torch.Tensor, cfg: OracleConfig):
    """Blend one chunk of pixels.

    alpha_raw [P, M] holds o*G for the M candidate Gaussians of every pixel,
    already in compositing order.  Returns (w [P, M], T_final [P],
    blended [P, M] bool).  Eq. 1 with the side outputs of Sec. 3.2 and 4.1."""
    alpha = torch.clamp(alpha_raw, max=cfg.alpha_max)
    keep = alpha >= cfg.alpha_min
    a = torch.where(keep, alpha, torch.zeros_like(alpha))
    # transmittance after each entry if every kept entry were blended; it is
    # non-increasing, so entries with T_after >= t_min are exactly the ones
    # before the stopping entry.
    t_after = torch.cumprod(1.0 - a, dim=1)
    blended = keep & (t_after.detach() >= cfg.t_min)
    ab = torch.where(blended, a, torch.zeros_like(a))
    one_minus = 1.0 - ab
    t_incl = torch.cumprod(one_minus, dim=1)
    t_excl = torch.cat([torch.ones_like(t_incl[:, :1]), t_incl[:, :-1]], dim=1)
    w = ab * t_excl
    t_final = t_incl[:, -1] if t_incl.shape[1] > 0 else torch.ones(alpha_raw.shape[0], dtype=f64)
    return w, t_final, blended


def _pixel_grid(cam, pix=None):
    if pix is None:
        vv, uu = np.meshgrid(np.arange(cam.height), np.arange(cam.width), indexing="ij")
        return uu.reshape(-1), vv.reshape(-1)
    pix = np.asarray(pix)
    return pix[:, 0], pix[:, 1]


def render_view(proj: dict, cam, cfg: OracleConfig | None = None, pix=None,
                chunk_elems: int = 1 << 22, flag_eps=None, want_depth=True) -> dict:
    """Render one view from the projected state `proj` (oracle.project.project).

    pix: optional [P, 2] integer (u, v) pixel coordinates; default the full
    image in row-major order.  Returns per-pixel tensors of length P:
      colour [P,3], t_final, imax (Gaussian index or -1), wmax, depth (d^mid
      of i_max, 0 if none), depth_center (z of i_max's centre, the
      alternative of Sec. 4.1, 0 if none), depth_blend, last (index of the last blended
      Gaussian or -1), n_blended, flags (near-threshold events, see
      _flags); and per-Gaussian: weight_sum [N] (I_i) and max_area [N] (S_i).
    """
    cfg = cfg or OracleConfig()
    uu, vv = _pixel_grid(cam, pix)
    P = len(uu)
    order = depth_order(proj["z"], proj["valid"])
    M = len(order)
    N = proj["z"].shape[0]
    oi = torch.as_tensor(order, dtype=torch.long)
    mean2d = proj["mean2d"][oi]
    conic = proj["conic"][oi]
    opac = proj["opacity"][oi]
    rgb = proj["rgb"][oi]
    zs = proj["z"][oi]
    bg = torch.tensor(cfg.bg, dtype=f64)
    sq = _square_rects(proj, oi, cam, cfg) if cfg.extent == "3sigma" else None

    colours, tfin, imax, wmax, depth, dblend, last, nbl, flags, dcen = ([] for _ in range(10))
    wsum = torch.zeros(N, dtype=f64)
    area = torch.zeros(N, dtype=torch.long)
    step = max(1, chunk_elems // max(M, 1))
    for s in range(0, P, step):
        u = torch.as_tensor(uu[s:s + step], dtype=f64)
        v = torch.as_tensor(vv[s:s + step], dtype=f64)
        dx = (u + 0.5)[:, None] - mean2d[None, :, 0]
        dy = (v + 0.5)[:, None] - mean2d[None, :, 1]
        q = conic[None, :, 0] * dx * dx + 2.0 * conic[None, :, 1] * dx * dy \
            + conic[None, :, 2] * dy * dy
        alpha_raw = opac[None, :] * torch.exp(-0.5 * q)
        amb = None
        if cfg.extent == "3sigma":
            # only the pixels of the tiles the 3-sigma square meets; amb marks
            # (pixel, Gaussian) pairs whose tile membership a relative change of
            # 1e-5 in the radius or the centre would flip
            inside, amb = _square_membership(sq, uu[s:s + step], vv[s:s + step], cfg.tile)
            alpha_raw = torch.where(torch.as_tensor(inside), alpha_raw, torch.zeros_like(alpha_raw))
        w, tf, blended = composite(alpha_raw, cfg)
        colours.append(w @ rgb + tf[:, None] * bg[None, :])
        tfin.append(tf)
        dblend.append(w @ zs)
        wd = w.detach()
        has = blended.any(dim=1)
        am = torch.argmax(wd, dim=1) if M > 0 else torch.zeros(len(u), dtype=torch.long)
        gi = torch.where(has, oi[am] if M > 0 else am, torch.full_like(am, -1))
        imax.append(gi)
        dcen.append(torch.where(has, proj["z"].detach()[gi.clamp(min=0)], torch.zeros(len(u), dtype=f64)))
        wmax.append(torch.where(has, wd.gather(1, am[:, None])[:, 0] if M > 0 else wd.sum(1),
                                torch.zeros(len(u), dtype=f64)))
        pos = torch.arange(M).expand(len(u), M)
        lastpos = torch.where(blended, pos, torch.full_like(pos, -1)).max(dim=1).values \
            if M > 0 else torch.full((len(u),), -1)
        last.append(torch.where(lastpos >= 0, oi[lastpos.clamp(min=0)] if M > 0 else lastpos,
                                torch.full_like(lastpos, -1)))
        nbl.append(blended.sum(dim=1))
        wsum.index_add_(0, oi, w.sum(dim=0)) if M > 0 else None
        if M > 0:
            area.index_add_(0, gi[has], torch.ones(int(has.sum()), dtype=torch.long))
        if want_depth:
            gsel = gi.clamp(min=0)
            d = midpoint_depth(proj["p_c"].detach()[gsel], proj["ell"][gsel], u, v, cam)
            depth.append(torch.where(has, d, torch.zeros_like(d)))
        fl = _flags(alpha_raw.detach(), wd, blended, zs.detach(), cfg, flag_eps)
        if amb is not None:
            # bit 5: a Gaussian that reaches alpha_min at the pixel (up to 0.1 %)
            # has an ambiguous tile membership there
            reach = (opac[None, :] * torch.exp(-0.5 * q)).detach() >= (1.0 - 1e-3) * cfg.alpha_min
            fl |= (torch.as_tensor(amb) & reach).any(1).long() << 5
        flags.append(fl)
    cat = lambda xs: torch.cat(xs) if xs else torch.zeros(0)
    out = dict(colour=cat(colours), t_final=cat(tfin), imax=cat(imax), wmax=cat(wmax),
               depth_blend=cat(dblend), depth_center=cat(dcen), last=cat(last), n_blended=cat(nbl),
               flags=cat(flags), weight_sum=wsum, max_area=area,
               u=torch.as_tensor(uu), v=torch.as_tensor(vv))
    if want_depth:
        out["depth"] = cat(depth)
    return out


def _square_rects(proj, oi, cam, cfg):
    """Tile rectangles of the 3-sigma squares of the ordered Gaussians, nominal
    and for the radius and centre moved by 1e-5 relative (for the ambiguity
    flag): a list of (tx0, tx1, ty0, ty1) integer arrays."""
    from .binning import lambda_max, square_tile_range
    cov = proj["cov2d"].detach().numpy()[oi.numpy()]
    m = proj["mean2d"].detach().numpy()[oi.numpy()]
    s3 = 3.0 * np.sqrt(lambda_max(cov[:, 0, 0], cov[:, 1, 1], cov[:, 0, 1]))
    tx_n = (cam.width + cfg.tile - 1) // cfg.tile
    ty_n = (cam.height + cfg.tile - 1) // cfg.tile
    shift = 1e-5 * np.maximum(1.0, np.abs(m[:, 0]) + np.abs(m[:, 1]))
    rects = []
    for f, sx, sy in [(1.0, 0, 0)] + [(f, sx, sy) for f in (1 - 1e-5, 1 + 1e-5) for sx in (-1, 1) for sy in (-1, 1)]:
        r = np.ceil(s3 * f)
        x0, x1 = square_tile_range(m[:, 0] + sx * shift, r, tx_n, cfg.tile)
        y0, y1 = square_tile_range(m[:, 1] + sy * shift, r, ty_n, cfg.tile)
        rects.append((x0, x1, y0, y1))
    return rects


def _square_membership(rects, u, v, tile):
    """[P, M] bool: the pixel's tile lies in the nominal rectangle; and whether
    any perturbed rectangle disagrees."""
    tx = (np.asarray(u) // tile)[:, None]
    ty = (np.asarray(v) // tile)[:, None]
    ins = [(tx >= x0[None]) & (tx <= x1[None]) & (ty >= y0[None]) & (ty <= y1[None]) for x0, x1, y0, y1 in rects]
    amb = np.zeros_like(ins[0])
    for other in ins[1:]:
        amb |= other != ins[0]
    return ins[0], amb


# z: the CUDA path's FP32 z (three rounded operations) and float32 of the
# float64 z differ by at most ~2 ulp (2^-23 relative each), so only depths
# within 3e-7 relative can swap order.
DEFAULT_FLAG_EPS = dict(alpha=1e-4, t=1e-4, w=1e-5, z=3e-7, clamp=1e-5)


def _flags(alpha_raw, w, blended, zs, cfg, eps=None):
    """Per-pixel bitmask of events that FP32 rounding can flip.

    bit 0: some entry up to the stopping one has alpha within eps.alpha
           (relative) of alpha_min (skip decision)
    bit 1: the transmittance after some entry up to the stopping one is
           within eps.t (relative) of t_min (stop decision)
    bit 2: the two largest weights are within eps.w (relative) (argmax tie)
    bit 3: two contributing entries have depths within eps.z (relative)
           (depth-order tie)
    bit 4: some blended entry has o*G within eps.clamp of alpha_max (the
           clamp switches the derivative off)
    (bit 5, set by render_view in the 3sigma extent: a Gaussian reaching the
    pixel has an ambiguous tile membership there)"""
    eps = dict(DEFAULT_FLAG_EPS, **(eps or {}))
    P, M = alpha_raw.shape
    out = torch.zeros(P, dtype=torch.long)
    if M == 0:
        return out
    alpha = torch.clamp(alpha_raw, max=cfg.alpha_max)
    keep = alpha >= cfg.alpha_min
    a = torch.where(keep, alpha, torch.zeros_like(alpha))
    t_after = torch.cumprod(1.0 - a, dim=1)
    # entries up to and including the stopping one
    stop_or_before = torch.cumsum((t_after < cfg.t_min).long(), dim=1) <= 1
    near_a = (torch.abs(alpha - cfg.alpha_min) <= eps["alpha"] * cfg.alpha_min) & stop_or_before
    out |= near_a.any(1).long() << 0
    near_t = (torch.abs(t_after - cfg.t_min) <= eps["t"] * cfg.t_min) & keep & stop_or_before
    out |= near_t.any(1).long() << 1
    if M >= 2:
        top2 = torch.topk(w, 2, dim=1).values
        tie = (top2[:, 0] > 0) & (top2[:, 0] - top2[:, 1] <= eps["w"] * top2[:, 0])
        out |= tie.long() << 2
    contrib = (keep & stop_or_before)
    zz = torch.where(contrib, zs[None, :].expand(P, M), torch.full((P, M), float("inf"), dtype=f64))
    zz_sorted = torch.sort(zz, dim=1).values
    gap = zz_sorted[:, 1:] - zz_sorted[:, :-1]
    close = torch.isfinite(zz_sorted[:, 1:]) & (gap <= eps["z"] * zz_sorted[:, 1:].abs())
    out |= close.any(1).long() << 3
    near_c = (torch.abs(alpha_raw - cfg.alpha_max) <= eps["clamp"]) & blended
    out |= near_c.any(1).long() << 4
    return out


def render(scene, cams, cfg: OracleConfig | None = None, masks=None, pix=None,
           want_depth=True) -> list[dict]:
    """Render every camera in `cams` from a Scene (float64, no grad).
    Eq. 1 and 2 with the side outputs of Sec. 3.2 and 4.1."""
    cfg = cfg or OracleConfig()
    outs = []
    with torch.no_grad():
        for k, cam in enumerate(cams):
            proj = project(scene.means, scene.scales, scene.rotations, scene.opacities,
                           scene.sh, scene.sh_degree, cam, cfg,
                           None if masks is None else masks[k])
            outs.append(render_view(proj, cam, cfg, None if pix is None else pix[k],
                                    want_depth=want_depth))
    return outs


def planar(colour: torch.Tensor, cam) -> torch.Tensor:
    """[H*W, 3] row-major pixel colours -> planar [3, H, W].
    Output layout only: no counterpart in the paper."""
    return colour.reshape(cam.height, cam.width, 3).permute(2, 0, 1)


def contributors(proj: dict, pix, alpha_min: float, slack: float = 1e-3) -> np.ndarray:
    """Indices of the Gaussians whose o*G reaches (1 - slack) * alpha_min at
    any of the given (u, v) pixels (no depth order, no termination): a
    superset of the Gaussians that can influence those pixels.
    Test helper for the alpha_min skip rule of Eq. 1."""
    pix = np.asarray(pix).reshape(-1, 2)
    if len(pix) == 0:
        return np.zeros(0, np.int64)
    valid = proj["valid"].numpy()
    m = proj["mean2d"].detach().numpy()
    c = proj["conic"].detach().numpy()
    o = proj["opacity"].detach().numpy()
    hit = np.zeros(len(m), bool)
    for u, v in pix:
        dx, dy = u + 0.5 - m[:, 0], v + 0.5 - m[:, 1]
        q = c[:, 0] * dx * dx + 2 * c[:, 1] * dx * dy + c[:, 2] * dy * dy
        hit |= valid & (o * np.exp(-0.5 * q) >= (1.0 - slack) * alpha_min)
    return np.nonzero(hit)[0]
