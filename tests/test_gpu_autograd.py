"""The torch.autograd.Function (raster.rasterize) against the oracle.

Gradients of a loss through rasterize() (SH degree 3, two views of different
sizes, one batch) are compared with the float64 oracle's autograd derivative
of the same loss, with the sorted lists kept from the forward and with them
rebuilt in the backward (recompute_sort).  The loss is a fixed seeded linear
functional of the image, zero on the pixels where the oracle sees an event
that FP32 can flip (threshold, stop, depth-order tie, clamp), so no Gaussian
has to be excluded.  Bars: image max-abs 1e-4; gradients
|g - g_ref| <= 1e-3 max(|g_ref|, 1e-2 ||g_ref||_inf) (Eq. 1 and its exact
derivative).
"""
import numpy as np
import pytest
import torch

from oracle import project as OP, render as OR
from paper_2411_12788_gb300 import raster, scenes

pytestmark = pytest.mark.gpu


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _case():
    sc = scenes.box_scene(256, seed=2, sh_degree=3)
    cams = [scenes.origin_camera(64, 64, 64.0),
            scenes.fov_camera(*scenes.look_at((0.4, -0.2, 0.3), (0.0, 0.0, 4.0)), 48, 40, 50.0)]
    return sc, cams


def _oracle(sc, cams, seed=4):
    rng = np.random.default_rng(seed)
    params = [torch.tensor(np.asarray(a, np.float64), requires_grad=True)
              for a in (sc.means, sc.scales, sc.rotations, sc.opacities, sc.sh)]
    weights, colours, flagged = [], [], 0
    for cam in cams:
        pr = OP.project(*params, sc.sh_degree, cam)
        out = OR.render_view(pr, cam, want_depth=False)
        ok = out["flags"].numpy() == 0
        flagged += int((~ok).sum())
        w = rng.standard_normal((cam.height * cam.width, 3)) * ok[:, None]
        (out["colour"] * torch.as_tensor(w)).sum().backward()
        weights.append(w)
        colours.append((out["colour"].detach().numpy(), ok))
    return params, weights, colours, flagged


def _planar(rows, cam):
    return rows.reshape(cam.height, cam.width, 3).transpose(2, 0, 1).reshape(-1)


@pytest.mark.parametrize("recompute", [False, True])
def test_rasterize_gradients_match_oracle(recompute):
    _need_gpu()
    sc, cams = _case()
    params, weights, colours, flagged = _oracle(sc, cams)
    assert flagged <= 2e-3 * sum(c.width * c.height for c in cams)
    ps = [torch.tensor(np.asarray(a, np.float32), device="cuda", requires_grad=True)
          for a in (sc.means, sc.scales, sc.rotations, sc.opacities, sc.sh)]
    st = raster.RasterSettings(cams, sc.sh_degree, recompute_sort=recompute)
    img, depth, imax, wsum, area = raster.rasterize(*ps, st)
    wt = torch.as_tensor(np.concatenate([_planar(w, c) for w, c in zip(weights, cams)])).float().cuda()
    (img * wt).sum().backward()
    torch.cuda.synchronize()
    plan = st.last_plan
    for v, (cam, (ref, ok)) in enumerate(zip(cams, colours)):
        got = raster.view_image(img.detach(), plan, v).permute(1, 2, 0).reshape(-1, 3).cpu().double().numpy()
        assert np.abs(got - ref)[ok].max() <= 1e-4
    for name, p, r in zip(["means", "scales", "rotations", "opacities", "sh"], ps, params):
        g = p.grad.cpu().double().numpy().reshape(-1)
        ref = r.grad.numpy().reshape(-1)
        floor = 1e-2 * np.abs(ref).max()
        bad = np.abs(g - ref) > 1e-3 * np.maximum(np.abs(ref), floor)
        assert not bad.any(), (name, int(bad.sum()), g[bad][:4], ref[bad][:4])


def test_l1_loss_function():
    """raster.l1_loss (gs_loss_l1 behind a torch.autograd.Function): the
    mean absolute difference and its gradient sign(image - target) / count,
    scaled by the incoming gradient."""
    _need_gpu()
    rng = np.random.default_rng(1)
    a = torch.tensor(rng.uniform(0, 1, 70001), dtype=torch.float32, device="cuda", requires_grad=True)
    b = torch.tensor(rng.uniform(0, 1, 70001), dtype=torch.float32, device="cuda")
    L = raster.l1_loss(a, b)
    (3.0 * L).backward()
    assert abs(L.item() - torch.abs(a.detach().double() - b.double()).mean().item()) <= 1e-6
    assert torch.equal(a.grad, 3.0 * (torch.sign(a.detach() - b) / a.numel()))
