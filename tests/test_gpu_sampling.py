"""Primitive sampling and depth-reinitialization seeds (Sec. 4.2, 4.3)
against the oracle, through the C ABI.  The random draws are inputs, so the
drawn indices are compared exactly; reprojected points to FP32 rounding."""
import numpy as np
import pytest
import torch

from oracle import sampling as OS
from paper_2411_12788_gb300 import raster, scenes

pytestmark = pytest.mark.gpu


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("k", [0, 1, 1000, 100000, 190000])
def test_weighted_sampling_matches_oracle(k):
    _need_gpu()
    rng = np.random.default_rng(21)
    n = 200000
    I = rng.gamma(0.5, 1.0, n).astype(np.float32)
    I[rng.uniform(size=n) < 0.3] = 0.0                        # no weight: never drawn
    I[:2000] = np.float32(0.75)                                # ties
    E = rng.exponential(size=n).astype(np.float32)
    E[:1000] = np.float32(1.5)
    got = raster.sample_gaussians(torch.from_numpy(I).cuda(), torch.from_numpy(E).cuda(), k).cpu().numpy()
    ref = OS.weighted_sample(I, E, k)
    assert np.array_equal(got.astype(np.int64), ref)
    assert len(ref) == min(k, int((I > 0).sum()))


def test_weighted_sampling_on_rendered_importance():
    _need_gpu()
    sc = scenes.cluster_scene(50000, 16, seed=8, sh_degree=0)
    cams = [scenes.ring_camera(0.4, 240, 160)]
    g = raster.GaussianTensors.from_scene(sc)
    fr = raster.forward(g, cams)
    I = fr.outs["weight_sum"]
    E = torch.from_numpy(np.random.default_rng(9).exponential(size=sc.n).astype(np.float32)).cuda()
    k = int((I > 0).sum().item()) // 2
    got = raster.sample_gaussians(I, E, k).cpu().numpy()
    assert np.array_equal(got.astype(np.int64), OS.weighted_sample(I.cpu().numpy(), E.cpu().numpy(), k))


@pytest.mark.parametrize("k", [1, 5000, 10 ** 7])
def test_depth_points_match_oracle(k):
    _need_gpu()
    sc = scenes.cluster_scene(30000, 16, seed=10, sh_degree=1)
    cams = [scenes.ring_camera(0.0, 200, 150), scenes.ring_camera(1.9, 97, 61)]
    g = raster.GaussianTensors.from_scene(sc)
    fr = raster.forward(g, cams)
    rng = np.random.default_rng(12)
    for v, cam in enumerate(cams):
        off, h, w = raster.view_slice(fr.plan, v)
        target = rng.uniform(size=(3, h, w)).astype(np.float32)
        u = (1.0 - rng.uniform(size=h * w)).astype(np.float32)       # in (0, 1]
        out = raster.depth_points(fr.plan, v, fr.outs["depth"], fr.outs["imax"], torch.from_numpy(target).cuda(),
                                  torch.from_numpy(u).cuda(), k)
        depth = fr.outs["depth"][off: off + h * w].cpu().numpy()
        imax = fr.outs["imax"][off: off + h * w].cpu().numpy()
        ref = OS.depth_points(depth, imax, target, u, cam, k)
        assert np.array_equal(out["pixel_idx"].cpu().numpy().astype(np.int64), ref["pixel_idx"])
        assert len(ref["pixel_idx"]) == min(k, int(((imax >= 0) & (depth > 0)).sum()))
        np.testing.assert_array_equal(out["colours"].cpu().numpy(), ref["colours"].astype(np.float32))
        # FP32 reprojection: a few ulp of the largest term (|p| up to the depth)
        scale = max(1.0, float(depth.max()))
        np.testing.assert_allclose(out["points"].cpu().numpy(), ref["points"], rtol=0, atol=1e-6 * scale)
