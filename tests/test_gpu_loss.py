"""The fused L1 + D-SSIM loss (the C1 training objective) through the C ABI
against the float64 oracle: loss to 1e-5 relative, gradient element by
element to 2e-4 of its largest magnitude (FP32 windowed moments)."""
import numpy as np
import pytest
import torch

from oracle import loss as OL
from paper_2411_12788_gb300 import raster, scenes

pytestmark = pytest.mark.gpu


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("lam", [0.2, 0.0, 1.0])
def test_l1_ssim_matches_oracle(lam):
    _need_gpu()
    sizes = [(50, 37), (64, 64), (33, 20), (200, 150)]
    cams = [scenes.origin_camera(w, h, float(w)) for w, h in sizes]
    plan = raster.make_plan(10, cams)
    rng = np.random.default_rng(31)
    imgs = [rng.uniform(size=(3, h, w)) for w, h in sizes]
    # targets: correlated with the images so that SSIM is far from 0 and 1
    tgts = [np.clip(a + rng.normal(0, 0.2, a.shape), 0, 1) for a in imgs]
    imgs[1][:, 10:20, 10:20] = tgts[1][:, 10:20, 10:20]       # exact matches: L1 sign(0) = 0
    x = torch.from_numpy(np.concatenate([a.reshape(-1) for a in imgs]).astype(np.float32)).cuda()
    y = torch.from_numpy(np.concatenate([a.reshape(-1) for a in tgts]).astype(np.float32)).cuda()
    L = torch.zeros(1, device="cuda")
    parts = torch.zeros(2, device="cuda")
    g = torch.empty_like(x)
    raster.loss_l1_ssim(plan, x, y, L, g, lam, l1_ssim=parts)
    torch.cuda.synchronize()
    xs = [torch.from_numpy(a.astype(np.float32)).double().requires_grad_(True) for a in imgs]
    ys = [torch.from_numpy(a.astype(np.float32)).double() for a in tgts]
    Lr, l1r, ssr = OL.l1_ssim(xs, ys, lam)
    grads = torch.autograd.grad(Lr, xs)
    gr = torch.cat([t.reshape(-1) for t in grads]).numpy()
    assert abs(L.item() - Lr.item()) <= 1e-5 * abs(Lr.item())
    assert abs(parts[0].item() - l1r.item()) <= 1e-5 * l1r.item()
    assert abs(parts[1].item() - ssr.item()) <= 1e-5 * abs(ssr.item())
    gg = g.cpu().numpy()
    assert np.abs(gg - gr).max() <= 2e-4 * np.abs(gr).max()


def test_l1_ssim_on_rendered_views_in_the_training_step():
    _need_gpu()
    sc = scenes.cluster_scene(20000, 16, seed=16, sh_degree=1)
    cams = [scenes.ring_camera(0.2, 120, 90), scenes.ring_camera(2.0, 77, 45)]
    g = raster.GaussianTensors.from_scene(sc)
    fr = raster.forward(g, cams)
    tg = scenes.target_images(cams, seed=1)
    y = torch.as_tensor(np.concatenate([t.reshape(-1) for t in tg])).cuda()
    L = torch.zeros(1, device="cuda")
    d = torch.empty_like(fr.outs["image"])
    raster.loss_l1_ssim(fr.plan, fr.outs["image"], y, L, d, 0.2)
    grads = raster.backward(g, fr, d)
    torch.cuda.synchronize()
    imgs = [raster.view_image(fr.outs["image"], fr.plan, v).cpu().double() for v in range(2)]
    ys = [torch.from_numpy(t).double() for t in tg]
    Lr, _, _ = OL.l1_ssim(imgs, ys, 0.2)
    assert abs(L.item() - Lr.item()) <= 1e-5 * Lr.item()
    assert all(torch.isfinite(v).all() for v in grads.values())


def test_training_step_with_l1_ssim_at_full_size():
    """500k Gaussians (SH 3), one 1600x1063 view, 0.8 L1 + 0.2 D-SSIM against
    the seeded target: the loss and its image gradient match the oracle
    evaluated on the rendered image, and the backward returns finite
    gradients and the forward's I_i."""
    _need_gpu()
    sc = scenes.cluster_scene(500_000, 64, seed=0, sh_degree=3)
    cam = scenes.ring_camera(0.3, 1600, 1063)
    g = raster.GaussianTensors.from_scene(sc)
    fr = raster.forward(g, [cam])
    tg = scenes.target_images([cam], seed=1)[0]
    y = torch.from_numpy(tg.reshape(-1)).cuda()
    L = torch.zeros(1, device="cuda")
    d = torch.empty_like(fr.outs["image"])
    raster.loss_l1_ssim(fr.plan, fr.outs["image"], y, L, d, 0.2)
    grads = raster.alloc_grads(g)
    grads["weight_sum"] = torch.zeros(int(fr.plan.n_items), device="cuda")
    raster.render_bwd(fr.plan, g.struct(), fr.cfg, fr.pre_ws, fr.sort_ws, d, fr.outs["image"],
                      fr.outs["n_contrib"], grads)
    torch.cuda.synchronize()
    x = raster.view_image(fr.outs["image"], fr.plan, 0).cpu().double().requires_grad_(True)
    Lr, _, _ = OL.l1_ssim([x], [torch.from_numpy(tg).double()], 0.2)
    (gr,) = torch.autograd.grad(Lr, [x])
    assert abs(L.item() - Lr.item()) <= 1e-5 * Lr.item()
    gg = d.cpu().double().reshape(gr.shape)
    assert (gg - gr).abs().max().item() <= 2e-4 * gr.abs().max().item()
    assert all(torch.isfinite(v).all() for v in grads.values())
    a, b = grads["weight_sum"].double().cpu(), fr.outs["weight_sum"].double().cpu()
    assert torch.all((a - b).abs() <= 1e-4 + 1e-5 * b.abs())
