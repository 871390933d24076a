"""Importance pruning (MSv2-D, Sec. 6.1) on the GPU against the oracle:
selection of the k largest accumulated weights (ties to the lower index) is
integer work decided on the same FP32 values, so it must be bit-exact; the
gathered scene must equal the rows it names; the re-render of the kept set
follows the render tolerances."""
import math

import numpy as np
import pytest
import torch

from oracle import prune as OPR, project as OP, render as OR
from paper_2411_12788_gb300 import raster, scenes

pytestmark = pytest.mark.gpu


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("n,k,kind", [(1000, 250, "uniform"), (100_003, 25_001, "ties"), (64, 0, "uniform"),
                                      (64, 64, "uniform"), (5000, 1, "ties"), (5000, 4999, "zeros"),
                                      (1 << 20, 1 << 18, "ties"),
                                      # the flag scans' tiles hold 8,192 counts: one full tile, one
                                      # plus a single count, and 301 tiles with a 3-count tail, whose
                                      # look-back walks more than two windows of 128 predecessors
                                      (8192, 4096, "ties"), (8193, 1, "uniform"), (300 * 8192 + 3, 614_400, "ties")])
def test_prune_select_matches_oracle(n, k, kind):
    _need_gpu()
    rng = np.random.default_rng(n + k)
    if kind == "uniform":
        w = rng.uniform(0, 10, n).astype(np.float32)
    elif kind == "ties":
        w = (rng.integers(0, 50, n) * 0.25).astype(np.float32)      # many exact ties
    else:
        w = np.zeros(n, np.float32)
        w[rng.integers(0, n, 10)] = 1.0
    got = raster.prune_select(torch.tensor(w, device="cuda"), k).cpu().numpy().astype(np.int64)
    ref = OPR.keep_top_k(w, k)
    assert len(ref) == k
    np.testing.assert_array_equal(got, ref)


def test_gather_scene_rows():
    _need_gpu()
    sc = scenes.box_scene(3000, seed=2, sh_degree=2)
    g = raster.GaussianTensors.from_scene(sc)
    idx = torch.tensor(np.sort(np.random.default_rng(0).choice(3000, 777, replace=False)), dtype=torch.int32,
                       device="cuda")
    h = raster.gather_scene(g, idx)
    ii = idx.long()
    for name in ("means", "scales", "rotations", "opacities", "sh"):
        assert torch.equal(getattr(h, name), getattr(g, name)[ii]), name


def test_dense_phase_prune_and_rerender():
    """3M Gaussians (256 clusters, SH 3), one 1920x1080 view: render, keep
    the top 25 % by accumulated weight, gather, re-render; the oracle checks
    the selection exactly and 64 sampled pixels of the re-render."""
    _need_gpu()
    sc = scenes.cluster_scene(3_000_000, 256, seed=0, sh_degree=3)
    cam = scenes.ring_camera(0.3, 1920, 1080)
    g = raster.GaussianTensors.from_scene(sc)
    fr = raster.forward(g, [cam])
    wsum = fr.outs["weight_sum"]
    k = math.ceil(0.25 * sc.n)
    keep = raster.prune_select(wsum, k)
    ref = OPR.keep_top(wsum.cpu().numpy(), 0.25)
    np.testing.assert_array_equal(keep.cpu().numpy().astype(np.int64), ref)
    h = raster.gather_scene(g, keep)
    fr2 = raster.forward(h, [cam])
    torch.cuda.synchronize()
    sub = sc.subset(ref)
    rng = np.random.default_rng(9)
    pix = np.stack([rng.integers(0, cam.width, 64), rng.integers(0, cam.height, 64)], 1)
    with torch.no_grad():
        pr = OP.project(sub.means, sub.scales, sub.rotations, sub.opacities, sub.sh, 3, cam)
        out = OR.render_view(pr, cam, pix=pix, want_depth=False)
    ok = out["flags"].numpy() == 0
    assert ok.sum() >= 56, np.bincount(out["flags"].numpy(), minlength=32)
    img = raster.view_image(fr2.outs["image"], fr2.plan, 0).cpu().double()
    col = img[:, pix[:, 1], pix[:, 0]].T.numpy()
    assert np.abs(col - out["colour"].numpy())[ok].max() <= 1e-4
