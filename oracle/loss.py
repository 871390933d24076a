"""Photometric losses for the training step (test infrastructure).

The paper trains with the 3DGS photometric objective (Sec. 6.2) without
restating it; the readings used here are the mean absolute error over all
channels and pixels of all views (L1) and its gradient.
"""
from __future__ import annotations

import torch


def l1(images, targets):
    """Mean |image - target| over every element of every view (float64)."""
    num = sum(torch.abs(a.to(torch.float64) - b.to(torch.float64)).sum()
              for a, b in zip(images, targets))
    den = sum(a.numel() for a in images)
    return num / den
