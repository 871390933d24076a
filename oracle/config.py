"""Numeric conventions of the rasterizer (oracle side; test infrastructure).

The paper fixes the blending rule (Eq. 1) but not these constants; the values
below are the readings this implementation adopts:
  znear      Gaussians whose camera-space z is at or below this are culled
  lowpass    isotropic 2-D dilation added to the projected covariance (px^2)
  clamp      the Jacobian of the local affine approximation is taken at the
             centre's x/z, y/z clamped to +-clamp * half-FOV tangent
  alpha_max  opacity clamp (alpha = min(alpha_max, o * G))
  alpha_min  an entry whose alpha is below this is skipped
  t_min      compositing stops before the entry that would bring the
             transmittance below this; that entry is not blended
  bg         background colour added as T_final * bg
  extent     "exact": a Gaussian reaches every pixel where alpha >= alpha_min;
             "3sigma": only the pixels of the tiles its 3-sigma square meets
             (the tile extent of the 3DGS rasterizer, Sec. 3.1; see
             oracle.binning)
"""
from __future__ import annotations

from dataclasses import dataclass, field


@dataclass
class OracleConfig:
    znear: float = 0.2
    lowpass: float = 0.3
    clamp: float = 1.3
    alpha_max: float = 0.99
    alpha_min: float = 1.0 / 255.0
    t_min: float = 1e-4
    bg: tuple = field(default_factory=lambda: (0.0, 0.0, 0.0))
    tile: int = 16
    extent: str = "exact"
