"""CPU oracle for the tile-based Gaussian-splatting rasterizer (TEST INFRASTRUCTURE).

This package is the slow, plain, obviously-correct reference that the CUDA
path is checked against.  It is test infrastructure only: the tests, the
smoke check and the benchmark's CPU-baseline leg may import it; the product
path (the C-ABI library and its Python binding) never does.

Everything is float64 PyTorch CPU code (or numpy), written from the paper's
definitions:
  * Sec. 3.1: the Gaussian primitive, depth ordering by distance to the image
    plane, the local affine (EWA) projection to 2-D and alpha blending, Eq. 1.
  * Sec. 3.2: the importance score I_i = sum of blending weights over rays.
  * Sec. 3.3, Eq. 2 and Sec. 4.1: the rendered index i_max = argmax_i w_i and
    the midpoint depth of the ray-ellipsoid chord d^mid_{i_max}; the blended
    depth sum_i w_i d_i; the maximum-contribution area S_i.
  * Sec. 4.1, 4.3, 5.1, 5.2: blur-split candidates, intersected, visible and
    critical Gaussians of a rendered view.
  * Sec. 4.2, 4.3: depth-reinitialization seeds and importance sampling.
  * Sec. 5.1: the aggressive clone of critical Gaussians.
Gradients are the exact derivatives of this forward, taken by torch.autograd.

Module map:
  oracle.project   step P: per (view, Gaussian) projection and colour
  oracle.render    step R: per-pixel compositing and its side outputs
  oracle.binning   step B: tile lists, sort order and tile ranges
  oracle.prune     top-fraction selection by blending weight
  oracle.identify  per-view selections of Gaussians (Sec. 4-5)
  oracle.sampling  primitive sampling and depth-reinitialization seeds
  oracle.densify   aggressive clone
  oracle.loss      photometric losses used by the training step
"""
from .config import OracleConfig
from . import project, render, binning, prune, loss, identify, sampling, densify

__all__ = ["OracleConfig", "project", "render", "binning", "prune", "loss", "identify", "sampling", "densify"]
