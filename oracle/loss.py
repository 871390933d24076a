"""Photometric losses for the training step (test infrastructure).

The paper trains with the 3DGS photometric objective (Sec. 6.2) without
restating it; the readings used here are the mean absolute error over all
channels and pixels of all views (L1), and (1 - lambda) L1 + lambda
(1 - SSIM) with lambda = 0.2 and the SSIM below.  Gradients are
torch.autograd of these float64 definitions (conv2d is the library step of
the windowed sums).
"""
from __future__ import annotations

import torch


def l1(images, targets):
    """Mean |image - target| over every element of every view (float64).
    The L1 term of the 3DGS objective the paper trains with (Sec. 6.2)."""
    num = sum(torch.abs(a.to(torch.float64) - b.to(torch.float64)).sum()
              for a, b in zip(images, targets))
    den = sum(a.numel() for a in images)
    return num / den


# SSIM as the 3DGS objective uses it (the paper does not restate it; reading):
# per channel, an 11 x 11 Gaussian window with sigma 1.5 normalised to sum 1,
# zero padding at the image border, C1 = 0.01^2, C2 = 0.03^2 (data range 1),
# and the mean of the SSIM map over every pixel and channel of every view.
SSIM_C1 = 0.01 ** 2
SSIM_C2 = 0.03 ** 2


def gaussian_window(size: int = 11, sigma: float = 1.5) -> torch.Tensor:
    """The 11x11 SSIM window (sigma 1.5, normalised) of the D-SSIM term (Sec. 6.2 reading)."""
    r = size // 2
    g = torch.exp(-torch.arange(-r, r + 1, dtype=torch.float64) ** 2 / (2 * sigma * sigma))
    g = g / g.sum()
    return torch.outer(g, g)


def ssim_map(x: torch.Tensor, y: torch.Tensor) -> torch.Tensor:
    """SSIM map of planar [C, H, W] images (float64, zero padding).
    The SSIM of the D-SSIM term (Sec. 6.2 reading)."""
    x = x.to(torch.float64)[:, None]
    y = y.to(torch.float64)[:, None]
    w = gaussian_window()[None, None]
    conv = lambda t: torch.nn.functional.conv2d(t, w, padding=w.shape[-1] // 2)
    mx, my = conv(x), conv(y)
    sxx = conv(x * x) - mx * mx
    syy = conv(y * y) - my * my
    sxy = conv(x * y) - mx * my
    s = ((2 * mx * my + SSIM_C1) * (2 * sxy + SSIM_C2)) / ((mx * mx + my * my + SSIM_C1) * (sxx + syy + SSIM_C2))
    return s[:, 0]


def l1_ssim(images, targets, lam: float = 0.2):
    """(1 - lam) L1 + lam (1 - SSIM), both means over every element of every
    view (the views' maps concatenated), float64.
    The photometric objective of the training step (Sec. 6.2 reading)."""
    den = sum(a.numel() for a in images)
    l1v = sum(torch.abs(a.to(torch.float64) - b.to(torch.float64)).sum() for a, b in zip(images, targets)) / den
    ss = sum(ssim_map(a, b).sum() for a, b in zip(images, targets)) / den
    return (1 - lam) * l1v + lam * (1 - ss), l1v, ss
