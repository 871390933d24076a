"""Step P of the oracle: per (view, Gaussian) projection and colour (test infrastructure).

Follows Sec. 3.1 of the paper: a Gaussian has centre p_i, covariance Sigma_i and
opacity; it is projected to a 2-D Gaussian by the local affine (EWA)
approximation of the perspective map, ordered by the depth of its centre
from the image plane, and coloured by spherical harmonics evaluated in the
viewing direction.  All arithmetic is float64; every function accepts
tensors that require grad so that torch.autograd gives the exact gradient.

Conventions (readings where the paper is silent):
  * covariance Sigma = R(q) diag(s^2) R(q)^T with q a (w, x, y, z) quaternion,
    normalised here (the input need not be unit);
  * camera: p_c = R p + t, x right, y down, z forward; the pixel (u, v)
    is sampled at its centre (u + 0.5, v + 0.5);
  * the projected covariance gets `lowpass` * I added;
  * colour = max(0, sum_lm sh_lm Y_lm(dir) + 0.5), dir the unit vector from
    the camera centre to p_i; Y_lm real SH with the Condon-Shortley phase,
    ordered m = -l..l inside band l.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from .config import OracleConfig

f64 = torch.float64


# --------------------------------------------------------------------------
# quaternions
# --------------------------------------------------------------------------
def _hamilton(a: torch.Tensor, b: torch.Tensor) -> torch.Tensor:
    """Quaternion product a*b, (w, x, y, z) along the last axis."""
    aw, ax, ay, az = a.unbind(-1)
    bw, bx, by, bz = b.unbind(-1)
    return torch.stack([
        aw * bw - ax * bx - ay * by - az * bz,
        aw * bx + ax * bw + ay * bz - az * by,
        aw * by - ax * bz + ay * bw + az * bx,
        aw * bz + ax * by - ay * bx + az * bw,
    ], dim=-1)


def rotation_matrix(q: torch.Tensor) -> torch.Tensor:
    """R(q) for (possibly unnormalised) quaternions q [..., 4] -> [..., 3, 3].

    Column k of R is the rotation of the basis vector e_k, computed as the
    sandwich product q_hat e_k q_hat^*.  The rotation of the covariance R(q) diag(s^2) R(q)^T (Sec. 3.1)."""
    qh = q / torch.linalg.norm(q, dim=-1, keepdim=True)
    conj = qh * torch.tensor([1.0, -1.0, -1.0, -1.0], dtype=qh.dtype)
    cols = []
    for k in range(3):
        e = torch.zeros(qh.shape[:-1] + (4,), dtype=qh.dtype)
        e[..., k + 1] = 1.0
        v = _hamilton(_hamilton(qh, e), conj)
        cols.append(v[..., 1:])
    return torch.stack(cols, dim=-1)


# --------------------------------------------------------------------------
# real spherical harmonics from their definition
# --------------------------------------------------------------------------
def _legendre_derivative_coeffs(l: int, m: int) -> np.ndarray:
    """Power-series coefficients of d^m/dz^m P_l(z)."""
    c = np.zeros(l + 1)
    c[l] = 1.0
    poly = np.polynomial.legendre.leg2poly(c)
    return np.polynomial.polynomial.polyder(poly, m) if m > 0 else poly


def sh_basis(degree: int, dirs: torch.Tensor) -> torch.Tensor:
    """Real SH Y_lm(d) for unit vectors d [..., 3] -> [..., (degree+1)^2].

    With z = cos(theta) and x + i y = sin(theta) e^{i phi}:
      Y_l0     = K_l0 P_l(z)
      Y_l(+m)  = sqrt2 K_lm (-1)^m Re((x+iy)^m) P_l^(m)(z)   (m > 0)
      Y_l(-m)  = sqrt2 K_lm (-1)^m Im((x+iy)^m) P_l^(m)(z)
    K_lm = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!), P_l^(m) the m-th derivative of
    the Legendre polynomial; the (-1)^m is the Condon-Shortley phase.
    The spherical-harmonic colour basis (Sec. 3.1)."""
    x, y, z = dirs.unbind(-1)
    out = []
    # powers of (x + i y): re/im parts by repeated complex multiplication
    re = [torch.ones_like(x)]
    im = [torch.zeros_like(x)]
    for m in range(1, degree + 1):
        r_prev, i_prev = re[-1], im[-1]
        re.append(r_prev * x - i_prev * y)
        im.append(r_prev * y + i_prev * x)
    for l in range(degree + 1):
        band = {}
        for m in range(0, l + 1):
            k = math.sqrt((2 * l + 1) / (4 * math.pi)
                          * math.factorial(l - m) / math.factorial(l + m))
            coeffs = _legendre_derivative_coeffs(l, m)
            pz = torch.zeros_like(z)
            for c in coeffs[::-1]:
                pz = pz * z + float(c)
            if m == 0:
                band[0] = k * pz
            else:
                s = math.sqrt(2.0) * k * (-1.0) ** m
                band[m] = s * re[m] * pz
                band[-m] = s * im[m] * pz
        out.extend(band[m] for m in range(-l, l + 1))
    return torch.stack(out, dim=-1)


# --------------------------------------------------------------------------
# projection
# --------------------------------------------------------------------------
def _t(a, dtype=f64):
    if isinstance(a, torch.Tensor):
        return a.to(dtype)
    return torch.as_tensor(np.asarray(a), dtype=dtype)


def project(means, scales, rotations, opacities, sh, sh_degree: int, cam,
            cfg: OracleConfig | None = None, mask=None) -> dict:
    """Per-Gaussian projected state for one camera.

    Returns a dict of float64 tensors (length N unless stated):
      p_c [N,3], z            camera-space centre and its depth
      cov3c [N,3,3]           camera-space 3-D covariance R Sigma R^T
      cov2d [N,2,2]           J cov3c J^T + lowpass I
      conic [N,3]             (A, B, C) of inverse(cov2d) = [[A, B], [B, C]]
      mean2d [N,2]            projected centre in pixels
      rgb [N,3]               SH colour, clamped at 0
      opacity [N]             as given
      tau [N]                 support bound: pixel x has o*G(x) >= alpha_min
                              iff q(x) <= tau = 2 ln(o / alpha_min)
      ell [N,3,3]             camera-frame ellipsoid matrix inverse(cov3c)
      valid [N] bool          z > znear, det > 0, mask (if given)
    """
    cfg = cfg or OracleConfig()
    p = _t(means)
    s = _t(scales)
    q = _t(rotations)
    o = _t(opacities)
    shc = _t(sh)
    R = _t(cam.R)
    tv = _t(cam.t)
    p_c = p @ R.T + tv
    x, y, z = p_c.unbind(-1)

    Rq = rotation_matrix(q)
    M = Rq * s.unsqueeze(-2)                       # R(q) diag(s)
    cov3 = M @ M.transpose(-1, -2)                 # Sigma = R diag(s^2) R^T
    cov3c = R @ cov3 @ R.T

    # Jacobian of (u, v) = (fx x/z + cx, fy y/z + cy) at the clamped centre
    limx = cfg.clamp * (cam.width / (2.0 * cam.fx))
    limy = cfg.clamp * (cam.height / (2.0 * cam.fy))
    zs = torch.where(z > cfg.znear, z, torch.ones_like(z))
    xc = torch.minimum(torch.maximum(x / zs, -limx * torch.ones_like(z)),
                       limx * torch.ones_like(z)) * zs
    yc = torch.minimum(torch.maximum(y / zs, -limy * torch.ones_like(z)),
                       limy * torch.ones_like(z)) * zs
    zero = torch.zeros_like(z)
    J = torch.stack([
        torch.stack([cam.fx / zs, zero, -cam.fx * xc / (zs * zs)], -1),
        torch.stack([zero, cam.fy / zs, -cam.fy * yc / (zs * zs)], -1),
    ], dim=-2)
    cov2d = J @ cov3c @ J.transpose(-1, -2) + cfg.lowpass * torch.eye(2, dtype=f64)
    a, b, c = cov2d[:, 0, 0], cov2d[:, 0, 1], cov2d[:, 1, 1]
    det = a * c - b * b
    dets = torch.where(det > 0, det, torch.ones_like(det))
    conic = torch.stack([c / dets, -b / dets, a / dets], -1)
    mean2d = torch.stack([cam.fx * x / zs + cam.cx, cam.fy * y / zs + cam.cy], -1)

    cam_centre = -(R.T @ tv)
    d = p - cam_centre
    d = d / torch.linalg.norm(d, dim=-1, keepdim=True)
    Y = sh_basis(sh_degree, d)                     # [N, K]
    K = (sh_degree + 1) ** 2
    rgb = torch.einsum("nk,nkc->nc", Y, shc[:, :K, :]) + 0.5
    rgb = torch.clamp(rgb, min=0.0)

    tau = 2.0 * torch.log(o / cfg.alpha_min)
    valid = (z > cfg.znear) & (det > 0)
    if mask is not None:
        valid = valid & torch.as_tensor(np.asarray(mask)).bool()
    ell = torch.linalg.inv(cov3c.detach())         # depth is not differentiated
    return dict(p_c=p_c, z=z, cov3c=cov3c, cov2d=cov2d, conic=conic, mean2d=mean2d,
                rgb=rgb, opacity=o, tau=tau, ell=ell, valid=valid)


def midpoint_depth(p_c: torch.Tensor, ell: torch.Tensor, u, v, cam) -> torch.Tensor:
    """d^mid for the pixel ray through (u + 0.5, v + 0.5) (Sec. 4.1, Eq. 2).

    The ray is r(t) = t d with d = ((u+.5-cx)/fx, (v+.5-cy)/fy, 1); the
    ellipsoid is (x - p_c)^T E (x - p_c) = 1 with E the inverse camera-space
    covariance (the unit ellipsoid of the paper's scale frame).  Its two
    intersections solve t^2 d'Ed - 2t d'Ep_c + p_c'Ep_c - 1 = 0, whose
    midpoint is t = d'E p_c / d'E d.  Because d_z = 1 the midpoint's camera
    z equals t, which is returned."""
    dx = (_t(u) + 0.5 - cam.cx) / cam.fx
    dy = (_t(v) + 0.5 - cam.cy) / cam.fy
    dvec = torch.stack([dx, dy, torch.ones_like(dx)], -1)
    Ed = torch.einsum("...ij,...j->...i", ell, dvec)
    return (Ed * p_c).sum(-1) / (Ed * dvec).sum(-1)


def midpoint_discriminant(p_c, ell, u, v, cam) -> torch.Tensor:
    """(d'Ep_c)^2 - (d'Ed)(p_c'Ep_c - 1): >= 0 iff the pixel ray meets the
    unit ellipsoid (the hit criterion the paper mentions in Sec. 4.1)."""
    dx = (_t(u) + 0.5 - cam.cx) / cam.fx
    dy = (_t(v) + 0.5 - cam.cy) / cam.fy
    dvec = torch.stack([dx, dy, torch.ones_like(dx)], -1)
    Ed = torch.einsum("...ij,...j->...i", ell, dvec)
    Ep = torch.einsum("...ij,...j->...i", ell, p_c)
    b = (Ed * p_c).sum(-1)
    return b * b - (Ed * dvec).sum(-1) * ((Ep * p_c).sum(-1) - 1.0)
