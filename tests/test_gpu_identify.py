"""gs_identify (Sec. 4.1, 4.3, 5.1, 5.2) against the oracle.

The selections are decided on the GPU forward pass's own FP32 statistics (S_i,
I_i, i_max, w_max, whose parity with the oracle renderer is tested
elsewhere), so the comparison is bit-exact: the oracle decides on the same
numbers in float64, which orders them identically.
"""
import numpy as np
import pytest
import torch

from oracle import identify as OI
from paper_2411_12788_gb300 import _lib, raster, scenes

pytestmark = pytest.mark.gpu


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _cams():
    sizes = [(200, 150), (160, 160), (97, 61)]
    return [scenes.ring_camera(a, w, h) for a, (w, h) in zip((0.0, 1.1, 2.5), sizes)]


def _oracle_flags(plan, cams, I, S, imax, wmax, cfg):
    n = int(plan.n)
    flags = np.zeros(n * len(cams), np.uint8)
    for v, cam in enumerate(cams):
        sl = slice(v * n, (v + 1) * n)
        p0, p1 = int(plan.pixel_base[v]), int(plan.pixel_base[v + 1])
        f = (OI.blur_split(S[sl], cam.height, cam.width, cfg.theta_blur) * raster.ID_BLUR
             | OI.intersected(S[sl]) * raster.ID_INTERSECT
             | OI.visible(I[sl], cfg.keep_visible) * raster.ID_VISIBLE
             | OI.critical(imax[p0:p1], wmax[p0:p1], cfg.keep_critical, n) * raster.ID_CRITICAL)
        flags[sl] = f.astype(np.uint8)
    return flags


def _counts(flags, n, V):
    f = flags.reshape(V, n)
    return np.stack([(f & b).astype(bool).sum(1) for b in (1, 2, 4, 8)], 1)


@pytest.mark.parametrize("q", [0.99, 0.5])
def test_identify_matches_oracle_on_gpu_statistics(q):
    _need_gpu()
    sc = scenes.cluster_scene(20000, 16, seed=5, sh_degree=1)
    cams = _cams()
    g = raster.GaussianTensors.from_scene(sc)
    fr = raster.forward(g, cams)
    cfg = raster.make_identify_config(keep_visible=q, keep_critical=q)
    out = raster.identify(fr.plan, fr.outs["weight_sum"], fr.outs["max_area"], fr.outs["imax"], fr.outs["wmax"], cfg)
    torch.cuda.synchronize()
    I = fr.outs["weight_sum"].cpu().numpy()
    S = fr.outs["max_area"].cpu().numpy().astype(np.int64)
    imax = fr.outs["imax"].cpu().numpy()
    wmax = fr.outs["wmax"].cpu().numpy()
    ref = _oracle_flags(fr.plan, cams, I, S, imax, wmax, cfg)
    got = out["flags"].cpu().numpy()
    assert np.array_equal(got, ref)
    assert np.array_equal(out["visible_mask"].cpu().numpy(), (ref & raster.ID_VISIBLE) // raster.ID_VISIBLE)
    assert np.array_equal(out["counts"].cpu().numpy(), _counts(ref, sc.n, len(cams)))
    # every selection is non-trivial on this scene
    c = out["counts"].cpu().numpy()
    assert (c > 0).all()
    assert (c[:, 2] < (I.reshape(len(cams), -1) > 0).sum(1)).all()


@pytest.mark.parametrize("q", [0.99, 0.5, 0.0, 1.0])
def test_identify_ties_on_synthetic_statistics(q):
    _need_gpu()
    rng = np.random.default_rng(11)
    n = 1000
    cams = [scenes.origin_camera(40, 30, 40.0), scenes.origin_camera(25, 20, 25.0)]
    plan = raster.make_plan(n, cams)
    P = int(plan.total_pixels)
    I = rng.integers(0, 6, 2 * n).astype(np.float32) * np.float32(0.25)        # many ties and zeros
    S = rng.integers(0, 4, 2 * n).astype(np.int32)
    imax = rng.integers(-1, n, P).astype(np.int32)
    wmax = np.where(imax >= 0, rng.integers(1, 5, P) * np.float32(0.125), 0).astype(np.float32)
    cfg = raster.make_identify_config(theta_blur=1e-3, keep_visible=q, keep_critical=q)
    dev = lambda a: torch.from_numpy(a).cuda()
    out = raster.identify(plan, dev(I), dev(S), dev(imax), dev(wmax), cfg)
    torch.cuda.synchronize()
    ref = _oracle_flags(plan, cams, I, S.astype(np.int64), imax, wmax, cfg)
    assert np.array_equal(out["flags"].cpu().numpy(), ref)
    assert np.array_equal(out["counts"].cpu().numpy(), _counts(ref, n, 2))


def test_visibility_mask_culls_in_preprocess():
    _need_gpu()
    sc = scenes.cluster_scene(20000, 16, seed=6, sh_degree=0)
    cam = _cams()[0]
    g = raster.GaussianTensors.from_scene(sc)
    fr = raster.forward(g, [cam])
    out = raster.identify(fr.plan, fr.outs["weight_sum"], fr.outs["max_area"], fr.outs["imax"], fr.outs["wmax"])
    mask = out["visible_mask"]
    keep = torch.nonzero(mask).flatten().to(torch.int32)
    assert 0 < keep.numel() < sc.n
    masked = raster.forward(g, [cam], mask=mask)
    st = raster.inspect_preprocess(masked)
    assert (st["tiles"].numpy()[mask.cpu().numpy() == 0] == 0).all()
    # the masked render is the render of the visible subset (same order, same arithmetic)
    sub = raster.forward(raster.gather_scene(g, keep), [cam])
    for k in ("image", "final_T", "n_contrib", "depth"):
        assert torch.equal(masked.outs[k], sub.outs[k]), k
    assert masked.plan.n_entries < fr.plan.n_entries


def test_bit_mask_culls_like_the_byte_mask():
    """GS_FLAG_MASK_BITS: the mask packed by gs_pack_mask (one bit per
    Gaussian and view, rows padded to 32-bit words) culls exactly what the
    byte mask culls; the packed bits are the byte mask's, padding zero."""
    _need_gpu()
    n = 3001                                       # rows end in a partial word
    sc = scenes.cluster_scene(n, 16, seed=8, sh_degree=1)
    cams = _cams()
    g = raster.GaussianTensors.from_scene(sc)
    rng = np.random.default_rng(9)
    byte = (rng.random(n * len(cams)) < 0.7).astype(np.uint8)
    mask = torch.as_tensor(byte).cuda()
    bits = raster.pack_mask(mask, n, len(cams))
    words = bits.cpu().numpy().view(np.uint32)
    assert words.shape == (len(cams), (n + 31) // 32)
    unpacked = ((words[:, :, None] >> np.arange(32, dtype=np.uint32)) & 1).reshape(len(cams), -1)
    np.testing.assert_array_equal(unpacked[:, :n].reshape(-1), byte)
    assert not unpacked[:, n:].any()
    a = raster.forward(g, cams, mask=mask)
    b = raster.forward(g, cams, cfg=raster.make_config(flags=_lib.GS_FLAG_MASK_BITS), mask=bits.contiguous())
    assert a.plan.n_entries == b.plan.n_entries
    np.testing.assert_array_equal(raster.inspect_preprocess(a)["tiles"].numpy(), raster.inspect_preprocess(b)["tiles"].numpy())
    for k in ("image", "final_T", "n_contrib", "imax", "depth"):
        assert torch.equal(a.outs[k], b.outs[k]), k


def test_identify_view_that_sees_nothing():
    _need_gpu()
    sc = scenes.box_scene(512, seed=1)
    R, t = scenes.look_at((0.0, 0.0, 0.0), (0.0, 0.0, -4.0))      # facing away from the scene
    cams = [scenes.origin_camera(64, 64, 64.0), scenes.fov_camera(R, t, 48, 32)]
    g = raster.GaussianTensors.from_scene(sc)
    fr = raster.forward(g, cams)
    out = raster.identify(fr.plan, fr.outs["weight_sum"], fr.outs["max_area"], fr.outs["imax"], fr.outs["wmax"])
    c = out["counts"].cpu().numpy()
    assert c[1].tolist() == [0, 0, 0, 0] and c[0, 1] > 0
    assert not out["flags"].cpu().numpy()[sc.n:].any()
