"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Stage by stage: projection (tolerance), binning / sort order / tile ranges
(bit-exact, decided by the oracle on the CUDA path's own FP32 state), render
outputs (tolerance, near-threshold pixels excluded and counted) and gradients
(relative tolerance).  Tolerances, derived from FP32 arithmetic:
  colour, T, w_max            max-abs 1e-4
  depth d^mid, d^center        max-abs 1e-4  (values reach ~35)
  depth d^blend               1e-4 * max(1, |d^blend|)  (weights' error times depth, see _depth_tol)
  I_i (summed weights)        1e-4 + 1e-5 * I      (sums of up to ~1e4 terms)
  gradients                   |g - g_ref| <= 1e-3 max(|g_ref|, 1e-2 ||g_ref||_inf)
"""
import math

import numpy as np
import pytest
import torch

from oracle import OracleConfig, binning as OB, project as OP, render as OR
from paper_2411_12788_gb300 import _lib, raster, scenes

pytestmark = pytest.mark.gpu
CFG = OracleConfig()


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _oracle_view(sc, cam, pix=None, want_depth=True, cfg=None):
    with torch.no_grad():
        pr = OP.project(sc.means, sc.scales, sc.rotations, sc.opacities, sc.sh, sc.sh_degree, cam)
        out = OR.render_view(pr, cam, cfg=cfg, pix=pix, want_depth=want_depth)
    return pr, out


def _gpu_pixels(fr, v, name):
    t = fr.outs[name]
    off, h, w = raster.view_slice(fr.plan, v)
    return t[off: off + h * w].cpu()


def _gpu_colour(fr, v):
    return raster.view_image(fr.outs["image"], fr.plan, v).cpu().double().permute(1, 2, 0).reshape(-1, 3)


def _multiview_cams():
    # three ragged views (sizes not multiples of 16) around the box scene
    sizes = [(50, 37), (64, 64), (33, 20)]
    eyes = [(0.0, 0.0, 0.0), (0.4, -0.2, 0.3), (-0.5, 0.3, -0.2)]
    cams = []
    for (w, h), e in zip(sizes, eyes):
        R, t = scenes.look_at(e, (0.0, 0.0, 4.0))
        cams.append(scenes.fov_camera(R, t, w, h, 50.0))
    return cams


SCENES = {
    "box1024_deg0": lambda: (scenes.box_scene(1024, seed=0, sh_degree=0), [scenes.origin_camera()]),
    "box512_deg3_multiview": lambda: (scenes.box_scene(512, seed=4, sh_degree=3), _multiview_cams()),
}
def _tall_cams(k):
    # k views 40 x 1040 (65 tile rows each) from eyes spread around the box
    cams = []
    for i in range(k):
        R, t = scenes.look_at((0.08 * (i - k / 2), 0.05 * i, -0.1 * (i % 3)), (0.0, 0.0, 4.0))
        cams.append(scenes.fov_camera(R, t, 40, 1040, 20.0))
    return cams


# binning cases: also a view 1,026 tiles across, whose lists gs_bin_sort builds
# by sorting the entries by tile id (the other scenes take the pair sort); and
# tall views whose 325 or 585 tile rows make the pair sort one 9-bit pass or
# an 8-bit and a 2-bit pass (the small scenes' few rows take one narrow pass)
SORT_SCENES = dict(SCENES, box600_wide_strip=lambda: (scenes.box_scene(600, seed=9, sh_degree=1),
                                                      [scenes.origin_camera(16410, 24, 2400.0),
                                                       scenes.origin_camera(64, 48, 64.0)]),
                   box400_tall_325_rows=lambda: (scenes.box_scene(400, seed=5, sh_degree=1), _tall_cams(5)),
                   box400_tall_585_rows=lambda: (scenes.box_scene(400, seed=6, sh_degree=1), _tall_cams(9)))


# ---------------------------------------------------------------- stage P
@pytest.mark.parametrize("case", list(SCENES))
def test_preprocess_matches_oracle(case):
    _need_gpu()
    sc, cams = SCENES[case]()
    g = raster.GaussianTensors.from_scene(sc)
    fr = raster.forward(g, cams)
    st = raster.inspect_preprocess(fr)
    n = sc.n
    for v, cam in enumerate(cams):
        sl = slice(v * n, (v + 1) * n)
        vis = st["tiles"][sl].numpy() > 0
        with torch.no_grad():
            pr = OP.project(sc.means, sc.scales, sc.rotations, sc.opacities, sc.sh, sc.sh_degree, cam)
        assert vis.sum() > 0
        assert np.all(pr["valid"].numpy()[vis])
        xy = st["xy_tau_z"][sl].double().numpy()
        co = st["conic_o"][sl].double().numpy()
        rgb = st["rgb"][sl].double().numpy()
        ref_m = pr["mean2d"].numpy()
        np.testing.assert_allclose(xy[vis, :2], ref_m[vis], rtol=1e-5, atol=1e-3)
        np.testing.assert_allclose(xy[vis, 3], pr["z"].numpy()[vis], rtol=1e-6)
        np.testing.assert_allclose(xy[vis, 2], pr["tau"].numpy()[vis], rtol=1e-5, atol=1e-5)
        ref_c = pr["conic"].numpy()
        scale = np.abs(ref_c[vis]).max(axis=1, keepdims=True)
        assert np.all(np.abs(co[vis, :3] - ref_c[vis]) <= 2e-5 * scale + 1e-7)
        np.testing.assert_allclose(co[vis, 3], sc.opacities[vis], rtol=0, atol=0)
        np.testing.assert_allclose(rgb[vis, :3], pr["rgb"].numpy()[vis], atol=2e-6)


# ---------------------------------------------------------------- stage B
@pytest.mark.parametrize("case", list(SORT_SCENES))
def test_binning_sort_ranges_bit_exact(case):
    """Tile lists: the oracle decides membership in float64 from the CUDA
    path's FP32 state; they must agree except within 1e-4 of the boundary.
    Order: stable (tile, float32 z, item) order of the CUDA path's own entries,
    bit-exact; ranges bit-exact; scanned offsets bit-exact."""
    _need_gpu()
    sc, cams = SORT_SCENES[case]()
    g = raster.GaussianTensors.from_scene(sc)
    fr = raster.forward(g, cams)
    torch.cuda.synchronize()
    assert raster.device_status(fr.plan, fr.pre_ws) == 0
    assert raster.lists_path(fr.plan) == (case != "box600_wide_strip")
    st = raster.inspect_preprocess(fr)
    so = raster.inspect_sort(fr)
    n = sc.n
    bases, total_tiles = OB.view_tile_bases([(c.width, c.height) for c in cams])
    assert total_tiles == fr.plan.total_tiles
    tiles_ids = so["tile_ids"].numpy().astype(np.int64)
    items = so["items"].numpy().astype(np.int64)
    E = int(fr.plan.n_entries)
    assert len(items) == E and E > 0
    gpu_set = set(zip(tiles_ids.tolist(), items.tolist()))
    assert len(gpu_set) == E                      # no duplicated entry
    xyz = st["xy_tau_z"].numpy()
    co = st["conic_o"].numpy()
    cnt = st["tiles"].numpy().astype(np.int64)
    near_total = 0
    for v, cam in enumerate(cams):
        sl = slice(v * n, (v + 1) * n)
        vis = cnt[sl] > 0
        gg, tt, near, rg, rt = OB.tile_lists(xyz[sl, :2], co[sl, :3], co[sl, 3], vis, cam.width, cam.height)
        exp = set(zip((tt + bases[v]).tolist(), (gg + v * n).tolist()))
        upper = bases[v + 1] if v + 1 < len(cams) else total_tiles
        got = {(t, i) for (t, i) in gpu_set if bases[v] <= t < upper}
        allowed = set(zip((tt[near] + bases[v]).tolist(), (gg[near] + v * n).tolist())) | \
            set(zip((rt + bases[v]).tolist(), (rg + v * n).tolist()))
        diff = exp ^ got
        assert diff <= allowed, list(diff - allowed)[:5]
        near_total += len(diff)
    assert near_total <= max(2, 1e-3 * E)
    # per-item counts and the depth-order scan
    per_item = np.bincount(items, minlength=len(cnt))
    np.testing.assert_array_equal(per_item, cnt)
    order = st["sorted_items"].numpy().astype(np.int64)
    zf = xyz[:, 3].astype(np.float32)
    vis_all = cnt > 0
    ref_order = np.nonzero(vis_all)[0][np.lexsort((np.nonzero(vis_all)[0], zf[vis_all]))]
    np.testing.assert_array_equal(order[:len(ref_order)], ref_order)
    if raster.lists_path(fr.plan):
        # pair offsets: scanned band sizes (tile rows of each visible item)
        rect = st["rect"].numpy().astype(np.int64)
        band = ((rect[:, 1] >> 16) & 0xFFFF) - ((rect[:, 0] >> 16) & 0xFFFF) + 1
        np.testing.assert_array_equal(st["pair_offsets"].numpy()[:len(ref_order)],
                                      OB.exclusive_scan(band[ref_order]))
        assert int(fr.plan.n_pairs) == int(band[ref_order].sum())
    else:
        np.testing.assert_array_equal(st["offsets"].numpy()[:len(ref_order)], OB.exclusive_scan(cnt[ref_order]))
    # order of the entries: stable by (tile, z bits) over (item-major) input
    inp = np.lexsort((tiles_ids, items))              # input order: item, then tile
    # items within the same (tile, z) keep ascending item order
    perm = OB.sort_entries(tiles_ids[inp], zf[items[inp]], None)
    np.testing.assert_array_equal(tiles_ids[inp][perm], tiles_ids)
    np.testing.assert_array_equal(items[inp][perm], items)
    np.testing.assert_array_equal(so["ranges"].numpy(), OB.tile_ranges(tiles_ids, total_tiles))


# ---------------------------------------------------------------- stage R
def _depth_tol(name, ref):
    """d^mid (Eq. 2) and d^center: max-abs 1e-4.  d^blend = sum_i w_i z_i:
    1e-4 max(1, |d^blend|).  The blending weights are held to the colour bar
    (max-abs 1e-4 on sum_i w_i c_i, colours of order 1); they carry the FP32
    projection's rounding (the conic, in a Gaussian's far tail) through the
    transmittance, and the blended depth multiplies their error by depths of
    up to ~35.  Measured on the 500k scene: a pixel with three blended
    entries, no stop, |dT| 1.2e-5 and colour error 6.8e-6, has d^blend 3.55
    at a mean depth of 14.7 and errs by 1.8e-4 = |dT| x 14.7, so max-abs
    1e-4 is out of reach for FP32 weights at depths past about 8."""
    if name == "depth_blend":
        return 1e-4 * np.maximum(1.0, np.abs(ref))
    return 1e-4


def _check_render(sc, cams, fr, max_flag_frac=2e-3, cfg=None):
    """Render outputs of every view against the oracle; returns the largest
    depth errors seen (d^mid, d^center, d^blend)."""
    n = sc.n
    worst = {}
    for v, cam in enumerate(cams):
        pr, out = _oracle_view(sc, cam, cfg=cfg)
        ok = out["flags"].numpy() == 0
        assert ok.mean() >= 1 - max_flag_frac, ok.mean()
        col = _gpu_colour(fr, v).numpy()
        ref = out["colour"].numpy()
        assert np.abs(col - ref)[ok].max() <= 1e-4
        T = _gpu_pixels(fr, v, "final_T").double().numpy()
        assert np.abs(T - out["t_final"].numpy())[ok].max() <= 1e-4
        wmax = _gpu_pixels(fr, v, "wmax").double().numpy()
        assert np.abs(wmax - out["wmax"].numpy())[ok].max() <= 1e-4
        imax = _gpu_pixels(fr, v, "imax").numpy()
        np.testing.assert_array_equal(imax[ok], out["imax"].numpy()[ok])
        if "n_blended" in fr.outs:
            nbl = _gpu_pixels(fr, v, "n_blended").numpy()
            np.testing.assert_array_equal(nbl[ok], out["n_blended"].numpy()[ok])
        # depths (values reach ~35): d^mid and d^center max-abs 1e-4; d^blend
        # max-abs 1e-4 + 1e-5 |d^blend| (FP32 transmittances: see _DEPTH_TOL)
        for name in ("depth", "depth_center", "depth_blend"):
            d = _gpu_pixels(fr, v, name).double().numpy()
            ref = out[name].numpy()
            err = np.abs(d - ref)[ok]
            worst[name] = max(worst.get(name, 0.0), float(err.max()) if err.size else 0.0)
            assert np.all(err <= _depth_tol(name, ref[ok])), (name, err.max())
        # n_contrib points at the last blended Gaussian in the tile's list
        nc = _gpu_pixels(fr, v, "n_contrib").numpy().astype(np.int64)
        last = out["last"].numpy()
        so = raster.inspect_sort(fr)
        rngs = so["ranges"].numpy()
        items = so["items"].numpy()
        base = fr.plan.tile_base[v]
        tx_n = (cam.width + 15) // 16
        uu, vv = out["u"].numpy(), out["v"].numpy()
        tile = base + (vv // 16) * tx_n + uu // 16
        has = (nc > 0) & ok
        gpu_last = items[rngs[tile[has], 0] + nc[has] - 1] - v * n
        np.testing.assert_array_equal(gpu_last, last[has])
        assert np.all(last[(nc == 0) & ok] == -1)
        # per-Gaussian sums of this view, compared where no flagged pixel is involved
        bad = OR.contributors(pr, np.stack([uu[~ok], vv[~ok]], 1), CFG.alpha_min)
        keep = np.ones(n, bool)
        keep[bad] = False
        ws = fr.outs["weight_sum"][v * n:(v + 1) * n].cpu().double().numpy()
        wr = out["weight_sum"].numpy()
        assert np.all(np.abs(ws - wr)[keep] <= 1e-4 + 1e-5 * np.abs(wr[keep]))
        ma = fr.outs["max_area"][v * n:(v + 1) * n].cpu().numpy()
        np.testing.assert_array_equal(ma[keep], out["max_area"].numpy()[keep])
    print(f"largest depth errors: {worst}")
    return worst


@pytest.mark.parametrize("case", list(SCENES))
def test_render_matches_oracle(case):
    _need_gpu()
    sc, cams = SCENES[case]()
    g = raster.GaussianTensors.from_scene(sc)
    fr = raster.forward(g, cams)
    torch.cuda.synchronize()
    assert raster.device_status(fr.plan, fr.pre_ws) == 0
    _check_render(sc, cams, fr)


@pytest.mark.parametrize("case", list(SCENES))
def test_three_sigma_extent_matches_oracle(case):
    """GS_FLAG_EXTENT_3SIGMA: every Gaussian is listed in the tiles its 3-sigma
    square meets (the same entries as the oracle's, except entries whose
    membership a 1e-5 relative change of the radius or centre would flip),
    and the render equals the oracle's render with the support truncated to
    those tiles."""
    _need_gpu()
    sc, cams = SCENES[case]()
    g = raster.GaussianTensors.from_scene(sc)
    fr = raster.forward(g, cams, cfg=raster.make_config(flags=_lib.GS_FLAG_EXTENT_3SIGMA))
    torch.cuda.synchronize()
    assert raster.device_status(fr.plan, fr.pre_ws) == 0
    st = raster.inspect_preprocess(fr)
    so = raster.inspect_sort(fr)
    n = sc.n
    bases, total_tiles = OB.view_tile_bases([(c.width, c.height) for c in cams])
    gpu_set = set(zip(so["tile_ids"].numpy().astype(np.int64).tolist(), so["items"].numpy().astype(np.int64).tolist()))
    assert len(gpu_set) == int(fr.plan.n_entries) > 0
    xyz, co, cnt = st["xy_tau_z"].numpy(), st["conic_o"].numpy(), st["tiles"].numpy().astype(np.int64)
    differ = 0
    for v, cam in enumerate(cams):
        sl = slice(v * n, (v + 1) * n)
        gg, tt, near, rg, rt = OB.tile_lists(xyz[sl, :2], co[sl, :3], co[sl, 3], cnt[sl] > 0, cam.width,
                                             cam.height, extent="3sigma")
        exp = set(zip((tt + bases[v]).tolist(), (gg + v * n).tolist()))
        upper = bases[v + 1] if v + 1 < len(cams) else total_tiles
        got = {(t, i) for (t, i) in gpu_set if bases[v] <= t < upper}
        allowed = set(zip((tt[near] + bases[v]).tolist(), (gg[near] + v * n).tolist())) | \
            set(zip((rt + bases[v]).tolist(), (rg + v * n).tolist()))
        assert (exp ^ got) <= allowed, list((exp ^ got) - allowed)[:5]
        differ += len(exp ^ got)
    assert differ <= max(2, 1e-3 * len(gpu_set))
    # the exact-support lists differ (the square is another extent)
    fe = raster.forward(g, cams)
    ex = raster.inspect_sort(fe)
    assert set(zip(ex["tile_ids"].numpy().tolist(), ex["items"].numpy().tolist())) != gpu_set
    _check_render(sc, cams, fr, cfg=OracleConfig(extent="3sigma"))


def test_render_is_deterministic():
    _need_gpu()
    sc, cams = SCENES["box512_deg3_multiview"]()
    g = raster.GaussianTensors.from_scene(sc)
    a = raster.forward(g, cams).outs
    b = raster.forward(g, cams).outs
    for k in ("image", "final_T", "n_contrib", "imax", "depth", "max_area"):
        assert torch.equal(a[k], b[k]), k


# ---------------------------------------------------------------- gradients
def _grad_case(seed=2, n=256, deg=3, size=64):
    sc = scenes.box_scene(n, seed=seed, sh_degree=deg)
    cam = scenes.origin_camera(size, size, float(size))
    target = scenes.target_images([cam], seed=1)[0]
    return sc, cam, target


def _oracle_grads(sc, cam, target, cfg=None):
    params = [torch.tensor(np.asarray(a, np.float64), requires_grad=True)
              for a in (sc.means, sc.scales, sc.rotations, sc.opacities, sc.sh)]
    pr = OP.project(*params, sc.sh_degree, cam)
    out = OR.render_view(pr, cam, cfg=cfg, want_depth=False)
    img = OR.planar(out["colour"], cam)
    L = torch.abs(img - torch.as_tensor(target, dtype=torch.float64)).mean()
    L.backward()
    return L.item(), [p.grad.numpy() for p in params], out, pr


def _assert_grad_close(name, g, ref, keep):
    g = g[keep].reshape(-1)
    ref = ref[keep].reshape(-1)
    floor = 1e-2 * np.abs(ref).max()
    bad = np.abs(g - ref) > 1e-3 * np.maximum(np.abs(ref), floor)
    assert not bad.any(), (name, int(bad.sum()), g[bad][:4], ref[bad][:4])


@pytest.mark.parametrize("deg,seed,extent", [(3, 2, "exact"), (0, 0, "exact"), (1, 5, "exact"), (3, 7, "3sigma")])
def test_backward_matches_oracle(deg, seed, extent):
    _need_gpu()
    sc, cam, target = _grad_case(seed=seed, deg=deg)
    g = raster.GaussianTensors.from_scene(sc)
    three = extent == "3sigma"
    fr = raster.forward(g, [cam], cfg=raster.make_config(flags=_lib.GS_FLAG_EXTENT_3SIGMA) if three else None)
    img = fr.outs["image"]
    tgt = torch.as_tensor(target.reshape(-1)).cuda()
    loss = torch.zeros(1, device="cuda")
    dL = torch.empty_like(img)
    raster.loss_l1(img, tgt, loss, dL)
    grads = raster.backward(g, fr, dL)
    torch.cuda.synchronize()
    L, ref, out, pr = _oracle_grads(sc, cam, target, cfg=OracleConfig(extent=extent))
    assert abs(loss.item() - L) <= 1e-6
    ok = out["flags"].numpy() == 0
    uu, vv = out["u"].numpy(), out["v"].numpy()
    bad = OR.contributors(pr, np.stack([uu[~ok], vv[~ok]], 1), CFG.alpha_min)
    keep = np.ones(sc.n, bool)
    keep[bad] = False
    assert keep.mean() > 0.9
    names = ["d_means", "d_scales", "d_rotations", "d_opacities", "d_sh"]
    for name, r in zip(names, ref):
        gg = grads[name].cpu().double().numpy()
        _assert_grad_close(name, gg, r, keep)


def test_mean2d_abs_gradient_matches_oracle():
    """d_mean2d_abs: per view the length of dL/d(projected centre), summed over
    the views (the densification statistic of 3DGS); two ragged views against
    the oracle's autograd derivative of each view's mean2d."""
    _need_gpu()
    sc = scenes.box_scene(384, seed=6, sh_degree=1)
    cams = _multiview_cams()[:2]
    targets = scenes.target_images(cams, seed=3)
    g = raster.GaussianTensors.from_scene(sc)
    fr = raster.forward(g, cams)
    img = fr.outs["image"]
    tgt = torch.cat([torch.as_tensor(t.reshape(-1)) for t in targets]).cuda()
    loss = torch.zeros(1, device="cuda")
    dL = torch.empty_like(img)
    raster.loss_l1(img, tgt, loss, dL)
    grads = raster.backward(g, fr, dL)
    torch.cuda.synchronize()
    params = [torch.tensor(np.asarray(a, np.float64), requires_grad=True)
              for a in (sc.means, sc.scales, sc.rotations, sc.opacities, sc.sh)]
    total = sum(3 * c.width * c.height for c in cams)
    L = 0.0
    prs, keep = [], np.ones(sc.n, bool)
    for cam, t in zip(cams, targets):
        pr = OP.project(*params, sc.sh_degree, cam)
        pr["mean2d"].retain_grad()
        out = OR.render_view(pr, cam, want_depth=False)
        L = L + torch.abs(OR.planar(out["colour"], cam) - torch.as_tensor(t, dtype=torch.float64)).sum() / total
        ok = out["flags"].numpy() == 0
        bad = OR.contributors(pr, np.stack([out["u"].numpy()[~ok], out["v"].numpy()[~ok]], 1), CFG.alpha_min)
        keep[bad] = False
        prs.append(pr)
    L.backward()
    assert abs(loss.item() - L.item()) <= 1e-6
    ref = sum(pr["mean2d"].grad.norm(dim=1).numpy() for pr in prs)
    assert keep.mean() > 0.9 and (ref[keep] > 0).sum() > 50
    _assert_grad_close("d_mean2d_abs", grads["d_mean2d_abs"].cpu().double().numpy(), ref, keep)


def test_backward_collects_the_forward_weight_sums():
    """I_i collected by the backward pass equals the forward's I_i."""
    _need_gpu()
    sc, cams = SCENES["box512_deg3_multiview"]()
    g = raster.GaussianTensors.from_scene(sc)
    fr = raster.forward(g, cams)
    grads = raster.alloc_grads(g)
    grads["weight_sum"] = torch.zeros(int(fr.plan.n_items), device="cuda")
    dL = torch.rand_like(fr.outs["image"]) - 0.5
    raster.render_bwd(fr.plan, g.struct(), fr.cfg, fr.pre_ws, fr.sort_ws, dL, fr.outs["image"],
                      fr.outs["n_contrib"], grads)
    a = grads["weight_sum"].double().cpu()
    b = fr.outs["weight_sum"].double().cpu()
    assert b.max() > 1.0
    assert torch.all((a - b).abs() <= 1e-4 + 1e-5 * b.abs())


def test_fixed_point_weight_sums_are_reproducible():
    """weight_sum_fixed (I_i in units of 2^-24, integer sums): bit-identical over
    repeated forward and backward passes, and within the per-pixel rounding of
    the float I_i; the backward's equals the forward's within the same bound."""
    _need_gpu()
    sc, cams = SCENES["box512_deg3_multiview"]()
    g = raster.GaussianTensors.from_scene(sc)
    want = raster.FWD_OUTPUTS + ("weight_sum_fixed",)
    runs = [raster.forward(g, cams, want=want) for _ in range(3)]
    fx = [fr.outs["weight_sum_fixed"].cpu() for fr in runs]
    assert all(torch.equal(fx[0], f) for f in fx[1:])
    fl = runs[0].outs["weight_sum"].double().cpu()
    fixed = fx[0].double() / 2.0 ** 24
    assert fl.max() > 1.0
    assert torch.all((fixed - fl).abs() <= 1e-4 + 1e-5 * fl.abs())
    fr = runs[0]
    dL = torch.rand_like(fr.outs["image"]) - 0.5
    bw = []
    for _ in range(2):
        grads = raster.alloc_grads(g)
        grads["weight_sum_fixed"] = torch.zeros(int(fr.plan.n_items), dtype=torch.int64, device="cuda")
        raster.render_bwd(fr.plan, g.struct(), fr.cfg, fr.pre_ws, fr.sort_ws, dL, fr.outs["image"],
                          fr.outs["n_contrib"], grads)
        bw.append(grads["weight_sum_fixed"].cpu())
    assert torch.equal(bw[0], bw[1])
    assert torch.all((bw[0].double() / 2.0 ** 24 - fixed).abs() <= 1e-4 + 1e-5 * fixed.abs())


def test_autograd_function_and_recompute():
    """The torch.autograd.Function gives the same gradients whether the sorted
    lists are kept or rebuilt in backward."""
    _need_gpu()
    sc, cam, target = _grad_case(seed=3, deg=1)
    g = raster.GaussianTensors.from_scene(sc)
    tgt = torch.as_tensor(target.reshape(-1)).cuda()
    res = []
    for recompute in (False, True):
        ps = [t.clone().requires_grad_(True) for t in (g.means, g.scales, g.rotations, g.opacities, g.sh)]
        st = raster.RasterSettings([cam], 1, recompute_sort=recompute)
        img, depth, imax, wsum, area = raster.rasterize(*ps, st)
        L = torch.abs(img - tgt).mean()
        L.backward()
        res.append([p.grad.clone() for p in ps])
    for a, b in zip(*res):
        assert torch.allclose(a, b, rtol=1e-5, atol=1e-7)


# ---------------------------------------------------------------- edge cases
def test_edge_cases():
    _need_gpu()
    cam = scenes.origin_camera(37, 21, 40.0)
    # empty scene
    sc = scenes.box_scene(0, seed=1)
    g = raster.GaussianTensors.from_scene(sc)
    fr = raster.forward(g, [cam])
    assert fr.plan.n_entries == 0
    assert torch.all(fr.outs["image"] == 0) and torch.all(fr.outs["final_T"] == 1)
    assert torch.all(fr.outs["imax"] == -1)
    # everything behind the camera or too transparent
    sc = scenes.box_scene(64, seed=1)
    sc.means[:32, 2] = -3.0
    sc.opacities[32:] = 1.0 / 512
    fr = raster.forward(raster.GaussianTensors.from_scene(sc), [cam])
    assert fr.plan.n_entries == 0
    # one huge Gaussian covering every tile, plus the termination stack
    zs = 4.0 + 0.25 * np.arange(20)
    sc = scenes.box_scene(21, seed=1)
    sc.means[:20, 2] = zs
    sc.means[:20, 0] = (17 + 0.5 - 18.5) * zs / 40.0
    sc.means[:20, 1] = (9 + 0.5 - 10.5) * zs / 40.0
    sc.scales[:20] = 0.02
    sc.opacities[:20] = 0.5
    sc.rotations[:20] = [1, 0, 0, 0]
    sc.means[20] = [0, 0, 30.0]
    sc.scales[20] = 5.0
    sc.opacities[20] = 0.3
    g = raster.GaussianTensors.from_scene(sc)
    fr = raster.forward(g, [cam])
    _check_render(sc, [cam], fr)
    assert fr.plan.n_entries >= fr.plan.total_tiles


def test_loss_l1_kernel():
    _need_gpu()
    rng = np.random.default_rng(0)
    a = torch.tensor(rng.uniform(0, 1, 100003), dtype=torch.float32, device="cuda")
    b = torch.tensor(rng.uniform(0, 1, 100003), dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, device="cuda")
    dL = torch.empty_like(a)
    raster.loss_l1(a, b, loss, dL)
    ref = torch.abs(a.double() - b.double()).mean().item()
    assert abs(loss.item() - ref) <= 1e-6
    assert torch.equal(dL, torch.sign(a - b) / a.numel())


# ---------------------------------------------------------------- full size
def test_training_scale_sampled_pixels():
    """500k Gaussians (SH 3), one 1600x1063 ring view: the oracle evaluates 96
    sampled pixels one by one; sort invariants checked on the whole list."""
    _need_gpu()
    sc = scenes.cluster_scene(500_000, 64, seed=0, sh_degree=3)
    cam = scenes.ring_camera(0.3, 1600, 1063)
    g = raster.GaussianTensors.from_scene(sc)
    fr = raster.forward(g, [cam])
    torch.cuda.synchronize()
    assert raster.device_status(fr.plan, fr.pre_ws) == 0
    rng = np.random.default_rng(7)
    pix = np.stack([rng.integers(0, cam.width, 96), rng.integers(0, cam.height, 96)], 1)
    _, out = _oracle_view(sc, cam, pix=pix)
    ok = out["flags"].numpy() == 0
    assert ok.sum() >= 90
    lin = pix[:, 1] * cam.width + pix[:, 0]
    col = _gpu_colour(fr, 0).numpy()[lin]
    assert np.abs(col - out["colour"].numpy())[ok].max() <= 1e-4
    T = _gpu_pixels(fr, 0, "final_T").double().numpy()[lin]
    t_err = np.abs(T - out["t_final"].numpy())
    c_err = np.abs(col - out["colour"].numpy()).max(axis=1)
    for name in ("depth", "depth_center", "depth_blend"):
        d = _gpu_pixels(fr, 0, name).double().numpy()[lin]
        ref = out[name].numpy()
        err = np.abs(d - ref)[ok]
        k = int(np.argmax(err))
        msg = f"{name}: largest error {err.max():.3e} (at depth {ref[ok][k]:.2f}) over {ok.sum()} sampled pixels"
        if name == "depth_blend":
            # the blended depth's error is the weights' error times the depth:
            # report the transmittance and colour errors of that pixel and its
            # mean blended depth d^blend / (1 - T)
            t_ref = out["t_final"].numpy()[ok][k]
            msg += (f"; there |dT| {t_err[ok][k]:.2e}, colour error {c_err[ok][k]:.2e}, "
                    f"mean depth {ref[ok][k] / max(1.0 - t_ref, 1e-12):.2f}")
        print(msg)
        assert np.all(err <= _depth_tol(name, ref[ok])), (name, err.max())
    np.testing.assert_array_equal(_gpu_pixels(fr, 0, "imax").numpy()[lin][ok], out["imax"].numpy()[ok])
    so = raster.inspect_sort(fr)
    st = raster.inspect_preprocess(fr)
    t = so["tile_ids"].numpy().astype(np.int64)
    it = so["items"].numpy().astype(np.int64)
    assert np.all(np.diff(t) >= 0)
    z = st["xy_tau_z"][:, 3].numpy()[it]
    same = np.diff(t) == 0
    dz = np.diff(z.view(np.uint32).astype(np.int64))
    assert np.all(dz[same] >= 0)
    assert np.all(np.diff(it)[same & (dz == 0)] > 0)
    # a permutation of the duplicated entries: every item as often as the
    # tiles it was counted on, and every entry in its own tile's range
    np.testing.assert_array_equal(np.bincount(it, minlength=sc.n), st["tiles"].numpy().astype(np.int64))
    rg = so["ranges"].numpy().astype(np.int64)
    nonempty = rg[:, 1] > rg[:, 0]
    assert rg[nonempty, 0].min() == 0 and rg[nonempty, 1].max() == fr.plan.n_entries
    assert np.all(t[rg[nonempty, 0]] == np.nonzero(nonempty)[0]) and np.all(t[rg[nonempty, 1] - 1] == np.nonzero(nonempty)[0])
    assert int((rg[nonempty, 1] - rg[nonempty, 0]).sum()) == fr.plan.n_entries


# ---------------------------------------------------------------- gradient buffer modes
@pytest.mark.parametrize("deg,wide", [(0, True), (3, True), (1, False), (3, False)])
def test_backward_overwrite_mode_equals_accumulate_into_zeros(deg, wide):
    """GS_FLAG_ZERO_ACCUM writes every attribute gradient (the buffers' old
    contents, here NaN, are never read); without it the gradients are added
    to what the buffers hold.  With SH rows stored wider than the degree and
    with rows of exactly the degree's width (degrees 1 and 3 then take the
    128-bit staging and write-out of the SH rows)."""
    _need_gpu()
    sc = scenes.cluster_scene(30000, 16, seed=17, sh_degree=deg)
    if wide:
        sc.sh = np.concatenate([sc.sh, np.zeros((sc.n, 2, 3), np.float32)], 1)    # stored rows wider than the degree
    cams = [scenes.ring_camera(0.5, 96, 80), scenes.ring_camera(2.6, 64, 48)]
    g = raster.GaussianTensors.from_scene(sc)
    fr = raster.forward(g, cams)
    dL = torch.randn_like(fr.outs["image"])
    ref = raster.alloc_grads(g)                      # zeros, accumulate mode
    raster.render_bwd(fr.plan, g.struct(), fr.cfg, fr.pre_ws, fr.sort_ws, dL, fr.outs["image"],
                      fr.outs["n_contrib"], ref)
    nan = {k: torch.full_like(v, float("nan")) for k, v in ref.items()}
    cfg = raster.make_config(flags=raster._lib.GS_FLAG_ZERO_ACCUM)
    raster.render_bwd(fr.plan, g.struct(), cfg, fr.pre_ws, fr.sort_ws, dL, fr.outs["image"],
                      fr.outs["n_contrib"], nan)
    ones = {k: torch.ones_like(v) for k, v in ref.items()}
    raster.render_bwd(fr.plan, g.struct(), fr.cfg, fr.pre_ws, fr.sort_ws, dL, fr.outs["image"],
                      fr.outs["n_contrib"], ones)
    torch.cuda.synchronize()
    # the per-item 2-D gradients are summed with float atomics, whose order
    # differs between runs: equal up to rounding
    for k in ref:
        tol = 1e-5 * (1e-3 + ref[k].abs().max().item())
        assert not torch.isnan(nan[k]).any(), k
        assert torch.allclose(nan[k], ref[k], rtol=0, atol=tol), k
        assert torch.allclose(ones[k], ref[k] + 1, rtol=0, atol=tol + 1e-6), k
    # Gaussians rendered in no view get exact zeros
    unseen = ref["d_means"].abs().sum(1) == 0
    assert unseen.any() and (nan["d_means"][unseen] == 0).all() and (nan["d_sh"][unseen] == 0).all()
    # coefficients beyond the degree: zero in both modes
    K = (deg + 1) ** 2
    assert (nan["d_sh"][:, K:] == 0).all() and (ones["d_sh"][:, K:] == 1).all()


def test_backward_over_many_views_is_the_sum_of_single_view_passes():
    """40 ragged views in one batch, more than a warp has lanes: each view's
    image equals the view rendered alone, and the batched gradients
    (d_mean2d_abs included) equal the sum over the views of the single-view
    backward passes, which the tests above pin to the oracle."""
    _need_gpu()
    sc = scenes.cluster_scene(4000, 16, seed=23, sh_degree=3)
    cams = [scenes.ring_camera(2 * math.pi * v / 40, 40 + 7 * (v % 3), 30 + 3 * (v % 5)) for v in range(40)]
    g = raster.GaussianTensors.from_scene(sc)
    fr = raster.forward(g, cams)
    gen = torch.Generator(device="cuda").manual_seed(5)
    dL = torch.randn(fr.outs["image"].shape, generator=gen, device="cuda")
    batched = raster.backward(g, fr, dL)
    total = raster.alloc_grads(g)
    for v, cam in enumerate(cams):
        one = raster.forward(g, [cam])
        off, h, w = raster.view_slice(fr.plan, v)
        assert torch.equal(one.outs["image"], fr.outs["image"][3 * off: 3 * (off + h * w)]), v
        for k, t in raster.backward(g, one, dL[3 * off: 3 * (off + h * w)]).items():
            total[k] += t
    torch.cuda.synchronize()
    late = fr.outs["image"][3 * int(fr.plan.pixel_base[32]):]
    assert late.abs().max().item() > 0.1          # the views past the first 32 see the scene
    # the per-item 2-D gradients are summed with float atomics: equal up to rounding
    for k in total:
        tol = 1e-5 * (1e-3 + total[k].abs().max().item())
        assert torch.allclose(batched[k], total[k], rtol=1e-4, atol=tol), k


# ---------------------------------------------------------------- failure detection
def test_bounded_wait_reports_timeout_and_context_survives():
    """The sort's and the scan's look-back waits, each over a predecessor that
    never publishes, give up after their bounds and report GS_ERR_TIMEOUT;
    the context keeps working."""
    _need_gpu()
    import time
    t0 = time.perf_counter()
    st = raster.selftest_wait_timeout()
    dt = time.perf_counter() - t0
    assert st == raster._lib.GS_ERR_TIMEOUT
    assert dt < 30.0
    sc = scenes.box_scene(256, seed=3)
    g = raster.GaussianTensors.from_scene(sc)
    fr = raster.forward(g, [scenes.origin_camera(64, 64, 64.0)])
    torch.cuda.synchronize()
    assert raster.device_status(fr.plan, fr.pre_ws) == 0
    assert torch.isfinite(fr.outs["image"]).all()
