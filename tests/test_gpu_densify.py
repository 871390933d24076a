"""Aggressive clone (Sec. 5.1) through the C ABI against the oracle."""
import numpy as np
import pytest
import torch

from oracle import densify as OD
from paper_2411_12788_gb300 import raster, scenes

pytestmark = pytest.mark.gpu


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("k", [0, 1, 3000])
def test_clone_matches_oracle(k):
    _need_gpu()
    sc = scenes.cluster_scene(10000, 8, seed=13, sh_degree=2)
    rng = np.random.default_rng(14)
    sc.opacities[:] = rng.uniform(1e-3, 0.995, sc.n).astype(np.float32)
    idx = rng.permutation(sc.n)[:k].astype(np.int32)              # distinct, any order
    g = raster.GaussianTensors.from_scene(sc)
    out = raster.clone_gaussians(g, torch.from_numpy(idx).cuda())
    ref = OD.clone(sc.means, sc.scales, sc.rotations, sc.opacities, sc.sh, idx)
    for name in ("means", "rotations", "sh"):
        assert np.array_equal(getattr(out, name).cpu().numpy(), ref[name].astype(np.float32)), name
    np.testing.assert_allclose(out.opacities.cpu().numpy(), ref["opacities"], rtol=2e-6, atol=0)
    np.testing.assert_allclose(out.scales.cpu().numpy(), ref["scales"], rtol=3e-6, atol=0)


def test_critical_gaussians_clone_and_render():
    _need_gpu()
    sc = scenes.cluster_scene(20000, 16, seed=15, sh_degree=0)
    cam = scenes.ring_camera(0.3, 160, 120)
    g = raster.GaussianTensors.from_scene(sc)
    fr = raster.forward(g, [cam])
    ids = raster.identify(fr.plan, fr.outs["weight_sum"], fr.outs["max_area"], fr.outs["imax"], fr.outs["wmax"])
    crit = torch.nonzero(ids["flags"] & raster.ID_CRITICAL).flatten().to(torch.int32)
    assert crit.numel() > 0
    g2 = raster.clone_gaussians(g, crit)
    assert g2.n == sc.n + crit.numel()
    fr2 = raster.forward(g2, [cam])
    img = fr2.outs["image"]
    assert torch.isfinite(img).all() and fr2.plan.n_entries > fr.plan.n_entries
