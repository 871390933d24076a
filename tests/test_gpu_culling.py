"""Per-block culling of the backward pass.

The backward kernel walks, per 8x4 pixel block, only the entries whose packed
support box meets the block; the forward pass decides membership pixel by
pixel.  The two agree only if every pixel the forward pass blended an entry at
lies inside that entry's box.  Every pixel's i_max is such a (pixel, entry)
pair, so on a scene where most blended pairs are an argmax (sparse needles)
this checks the boxes directly, on the inputs where the FP32 exponent's
rounding is largest next to the support: axis ratios up to 1e3 and opacities
just above the alpha threshold.
"""
import numpy as np
import pytest
import torch

from paper_2411_12788_gb300 import raster, scenes

pytestmark = pytest.mark.gpu


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _unpack_extents(packed: np.ndarray):
    u = packed.astype(np.float32).view(np.uint32)
    ex = (u & 0xFFFF).astype(np.uint16).view(np.float16).astype(np.float32)
    ey = (u >> 16).astype(np.uint16).view(np.float16).astype(np.float32)
    return ex, ey


@pytest.mark.parametrize("seed", [7, 8])
def test_support_boxes_hold_every_blended_pixel(seed):
    _need_gpu()
    W = H = 512
    sc = scenes.needle_scene(4000, seed=seed)
    cam = scenes.origin_camera(W, H, 512.0)
    g = raster.GaussianTensors.from_scene(sc)
    fr = raster.forward(g, [cam])
    st = raster.inspect_preprocess(fr)
    imax = fr.outs["imax"][: W * H].cpu().numpy()
    pix = np.nonzero(imax >= 0)[0]
    assert pix.size > 10000
    i = imax[pix]
    xyz = st["xy_tau_z"].numpy()
    mx, my = xyz[i, 0], xyz[i, 1]
    ex, ey = _unpack_extents(st["rgb"].numpy()[i, 3])
    px = (pix % W).astype(np.float32) + np.float32(0.5)
    py = (pix // W).astype(np.float32) + np.float32(0.5)
    inside = (mx - ex <= px) & (mx + ex >= px) & (my - ey <= py) & (my + ey >= py)
    assert inside.all(), f"{(~inside).sum()} blended pixels outside their entry's box"

    # the scene does reach thin, faint supports
    co = st["conic_o"].numpy()
    vis = st["tiles"].numpy() > 0
    A, B, C = co[vis, 0].astype(np.float64), co[vis, 1].astype(np.float64), co[vis, 2].astype(np.float64)
    disc = np.sqrt(((A - C) / 2) ** 2 + B ** 2)
    kappa = ((A + C) / 2 + disc) / ((A + C) / 2 - disc)
    assert kappa.max() > 1e4
    assert (co[vis, 3] < 1.02 / 255).sum() > 100
    # and blended pixels reach the outer part of their boxes (thin supports get
    # wider margins, so the ratio stays below 1 / (1.02 + 4e-6 kappa))
    rel = np.maximum(np.abs(px - mx) / ex, np.abs(py - my) / ey)
    assert (rel > 0.75).sum() > 0


@pytest.mark.parametrize("seed", [7, 9])
def test_backward_culling_drops_no_blended_pair(seed):
    """The backward replays, per 8x4 block, only the entries that pass the
    box and exponent tests, and collects I_i = sum of the weights it
    replays.  A blended (pixel, entry) pair culled by mistake would leave
    that Gaussian's collected I_i short of the forward's (a pair weighs at
    least alpha_min T); on thin, faint needles the two sums must agree."""
    _need_gpu()
    sc = scenes.needle_scene(4000, seed=seed)
    cams = [scenes.origin_camera(512, 512, 512.0), scenes.origin_camera(300, 200, 300.0)]
    g = raster.GaussianTensors.from_scene(sc)
    fr = raster.forward(g, cams)
    grads = raster.alloc_grads(g)
    grads["weight_sum"] = torch.zeros(int(fr.plan.n_items), device="cuda")
    dL = torch.rand_like(fr.outs["image"]) - 0.5
    raster.render_bwd(fr.plan, g.struct(), fr.cfg, fr.pre_ws, fr.sort_ws, dL, fr.outs["image"],
                      fr.outs["n_contrib"], grads)
    a = grads["weight_sum"].double().cpu()
    b = fr.outs["weight_sum"].double().cpu()
    assert (b > 0).sum() > 2000
    assert torch.all((a - b).abs() <= 2e-6 + 1e-5 * b.abs())


def test_culling_past_the_validated_condition_number():
    """The box margin is argued only up to a 2-D condition number of 2e5.
    Long, extremely thin needles crossing the view (condition numbers from
    4e4 to above 1e6) must get unbounded boxes past the bound (the culling
    then rests on the exact exponent test alone) and finite ones below it,
    and the backward must still replay every pair the forward blended: its
    collected I_i equals the forward's, also for the Gaussians past the bound."""
    _need_gpu()
    sc = scenes.crossing_needles_scene(200, seed=0)
    cams = [scenes.origin_camera(512, 512, 1024.0)]
    g = raster.GaussianTensors.from_scene(sc)
    fr = raster.forward(g, cams)
    st = raster.inspect_preprocess(fr)
    co = st["conic_o"].numpy().astype(np.float64)
    vis = st["tiles"].numpy() > 0
    A, B, C = co[:, 0], co[:, 1], co[:, 2]
    disc = np.sqrt(((A - C) / 2) ** 2 + B ** 2)
    with np.errstate(divide="ignore", invalid="ignore"):
        kappa = ((A + C) / 2 + disc) / ((A + C) / 2 - disc)
    ex, ey = _unpack_extents(st["rgb"].numpy()[:, 3])
    past = vis & (kappa > 2.1e5)
    within = vis & (kappa < 1.9e5)
    assert past.sum() >= 50 and within.sum() >= 50, (past.sum(), within.sum())
    assert np.isinf(ex[past]).all() and np.isinf(ey[past]).all()
    assert np.isfinite(ex[within]).all() and np.isfinite(ey[within]).all()
    grads = raster.alloc_grads(g)
    grads["weight_sum"] = torch.zeros(int(fr.plan.n_items), device="cuda")
    dL = torch.rand_like(fr.outs["image"]) - 0.5
    raster.render_bwd(fr.plan, g.struct(), fr.cfg, fr.pre_ws, fr.sort_ws, dL, fr.outs["image"],
                      fr.outs["n_contrib"], grads)
    torch.cuda.synchronize()
    a = grads["weight_sum"].double().cpu().numpy()
    b = fr.outs["weight_sum"].double().cpu().numpy()
    assert np.all(np.abs(a - b) <= 2e-6 + 1e-5 * np.abs(b))
    assert (b[past] > 1.0).sum() >= 50, (b[past] > 1.0).sum()
