"""Seeded synthetic inputs: Gaussian scenes, pinhole cameras and target images.

This module is shared by the tests, the benchmark and the smoke run, and by
the CPU oracle's tests.  It draws random numbers and builds input geometry
(camera poses); it holds none of the rasterizer's arithmetic (no projection,
no colour evaluation, no compositing).

Scene layout (all float32, numpy, C-contiguous):
  means      [N, 3]   world-space centres p_i
  scales     [N, 3]   linear (activated) per-axis standard deviations s
  rotations  [N, 4]   unit quaternions, (w, x, y, z) order
  opacities  [N]      opacity in (0, 1)
  sh         [N, K, 3] spherical-harmonic coefficients, K = (degree+1)^2,
                      band-major (l = 0..degree, m = -l..l), RGB last
Camera: world->camera rotation R (row-major 3x3), translation t, focal
lengths fx, fy, principal point cx, cy, image width and height.  Camera axes
follow the usual vision convention: x right, y down, z forward.

The workload shapes follow the paper's training scenes (0.3-5 M Gaussians,
views about 1.6 K pixels wide, Sec. 6.2-6.3 and the resource table); the
datasets themselves are not used.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Real SH band-0 basis value 1/(2*sqrt(pi)); the generators store a DC colour
# c as the coefficient (c - 0.5) / Y00 so that a degree-0 render shows c.
_Y00 = 0.5 / math.sqrt(math.pi)


@dataclass
class Camera:
    R: np.ndarray           # [3, 3] float64, world -> camera rotation
    t: np.ndarray           # [3] float64
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int

    @property
    def n_pixels(self) -> int:
        return self.width * self.height


@dataclass
class Scene:
    means: np.ndarray
    scales: np.ndarray
    rotations: np.ndarray
    opacities: np.ndarray
    sh: np.ndarray
    sh_degree: int
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def subset(self, idx) -> "Scene":
        idx = np.asarray(idx)
        return Scene(self.means[idx].copy(), self.scales[idx].copy(),
                     self.rotations[idx].copy(), self.opacities[idx].copy(),
                     self.sh[idx].copy(), self.sh_degree, dict(self.meta))

    def save(self, path) -> None:
        """Writes the scene as flat arrays (numpy .npz): a checkpoint of the
        Gaussians that `load` reads back exactly."""
        np.savez(path, means=self.means, scales=self.scales, rotations=self.rotations,
                 opacities=self.opacities, sh=self.sh, sh_degree=np.int64(self.sh_degree))


def load(path) -> Scene:
    """A scene written by Scene.save (or any .npz with the same arrays)."""
    with np.load(path) as z:
        return Scene(z["means"], z["scales"], z["rotations"], z["opacities"], z["sh"], int(z["sh_degree"]))


def scene_from_tensors(g) -> Scene:
    """The host copy of device Gaussians (raster.GaussianTensors), e.g. to save
    a trained or pruned scene."""
    f = lambda t: t.detach().cpu().numpy().astype(np.float32)
    return Scene(f(g.means), f(g.scales), f(g.rotations), f(g.opacities), f(g.sh), int(g.sh_degree))


def _unit_quaternions(rng: np.random.Generator, n: int) -> np.ndarray:
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


def _sigmoid(x: np.ndarray) -> np.ndarray:
    return 1.0 / (1.0 + np.exp(-x))


def _sh_from_colour(rng: np.random.Generator, n: int, degree: int,
                    high_std: float) -> np.ndarray:
    k = (degree + 1) ** 2
    sh = np.zeros((n, k, 3), dtype=np.float64)
    colour = rng.uniform(0.0, 1.0, size=(n, 3))
    sh[:, 0, :] = (colour - 0.5) / _Y00
    if k > 1:
        sh[:, 1:, :] = rng.normal(0.0, high_std, size=(n, k - 1, 3))
    return sh


def _finish(means, scales, quats, opac, sh, degree, meta) -> Scene:
    f = np.float32
    return Scene(np.ascontiguousarray(means, f), np.ascontiguousarray(scales, f),
                 np.ascontiguousarray(quats, f), np.ascontiguousarray(opac, f),
                 np.ascontiguousarray(sh, f), degree, meta)


def box_scene(n: int = 1024, seed: int = 0, sh_degree: int = 0) -> Scene:
    """Plain forward+backward scene: means uniform in [-1,1]x[-1,1]x[2,6],
    log-scales N(-3, 0.5), uniform unit quaternions, opacity sigmoid(N(0,1)),
    DC colour uniform in [0,1] (RGB), in front of a camera at the origin."""
    rng = np.random.default_rng(seed)
    means = np.stack([rng.uniform(-1, 1, n), rng.uniform(-1, 1, n),
                      rng.uniform(2, 6, n)], axis=1)
    scales = np.exp(rng.normal(-3.0, 0.5, size=(n, 3)))
    quats = _unit_quaternions(rng, n)
    opac = _sigmoid(rng.normal(0.0, 1.0, size=n))
    sh = _sh_from_colour(rng, n, sh_degree, 0.05)
    return _finish(means, scales, quats, opac, sh, sh_degree,
                   {"kind": "box", "seed": seed})


def needle_scene(n: int = 4000, seed: int = 0, long_range=(0.02, 0.5), faint_frac: float = 0.5) -> Scene:
    """Adversarial scene for the support-box margins: means uniform in
    [-1.5,1.5]^2 x [2,8], long axis log-uniform in `long_range` (default
    [0.02, 0.5]), the other two shorter by a log-uniform ratio in [1, 1000]
    (x U[0.5, 2] for the third), uniform unit quaternions, a fraction
    `faint_frac` (default half) of the opacities just above 1/255
    ((1 + U[1e-4, 1e-2]) / 255) and the rest U[0.05, 0.99], DC colour U[0,1]."""
    rng = np.random.default_rng(seed)
    means = np.stack([rng.uniform(-1.5, 1.5, n), rng.uniform(-1.5, 1.5, n),
                      rng.uniform(2, 8, n)], axis=1)
    long = np.exp(rng.uniform(np.log(long_range[0]), np.log(long_range[1]), n))
    short = long / np.exp(rng.uniform(0.0, np.log(1e3), n))
    scales = np.stack([long, short, short * rng.uniform(0.5, 2.0, n)], axis=1)
    quats = _unit_quaternions(rng, n)
    faint = rng.uniform(size=n) < faint_frac
    opac = np.where(faint, (1.0 + rng.uniform(1e-4, 1e-2, n)) / 255.0, rng.uniform(0.05, 0.99, n))
    sh = _sh_from_colour(rng, n, 0, 0.05)
    return _finish(means, scales, quats, opac, sh, 0, {"kind": "needles", "seed": seed})


def crossing_needles_scene(n: int = 200, seed: int = 0) -> Scene:
    """Long, extremely thin needles lying nearly in the image plane of a
    camera at the origin looking down +z, all passing close to the optical
    axis (so that they cross the image and one another): means
    U([-0.3,0.3]^2 x [3,5]), long axis log-uniform in [0.5, 2], the other two
    1e-4 of it, rotations about the viewing axis by a uniform angle (tilted
    by N(0, 0.05) quaternion components), opacity U[0.3, 0.9], DC colour
    U[0,1].  Seen at focal lengths near 1000 px their projected
    covariances have condition numbers from 1e4 to above 1e6."""
    rng = np.random.default_rng(seed)
    means = np.stack([rng.uniform(-0.3, 0.3, n), rng.uniform(-0.3, 0.3, n), rng.uniform(3, 5, n)], axis=1)
    long = np.exp(rng.uniform(np.log(0.5), np.log(2.0), n))
    scales = np.stack([long, 1e-4 * long, 1e-4 * long], axis=1)
    th = rng.uniform(0.0, 2 * np.pi, n)
    quats = np.stack([np.cos(th / 2), rng.normal(0, 0.05, n), rng.normal(0, 0.05, n), np.sin(th / 2)], axis=1)
    quats /= np.linalg.norm(quats, axis=1, keepdims=True)
    opac = rng.uniform(0.3, 0.9, n)
    sh = _sh_from_colour(rng, n, 0, 0.05)
    return _finish(means, scales, quats, opac, sh, 0, {"kind": "crossing-needles", "seed": seed})


def cluster_scene(n: int, n_clusters: int = 64, seed: int = 0,
                  sh_degree: int = 3) -> Scene:
    """Training-shaped scene: 80 % of the means from a mixture of anisotropic
    3-D Gaussian clusters (centres N(0, 0.8^2 I), per-axis std log-uniform in
    [0.05, 0.4], random orientation, equal weights), 20 % on a background
    shell (uniform direction, radius U[10, 30]).  Log-scales N(-4, 0.7),
    opacity sigmoid(N(0, 1.5)), uniform unit quaternions, DC colour U[0,1],
    higher SH bands N(0, 0.05)."""
    rng = np.random.default_rng(seed)
    n_shell = n // 5
    n_clu = n - n_shell
    centres = rng.normal(0.0, 0.8, size=(n_clusters, 3))
    stds = np.exp(rng.uniform(math.log(0.05), math.log(0.4), size=(n_clusters, 3)))
    # random cluster orientations: orthogonal factors of Gaussian matrices
    crot = np.linalg.qr(rng.standard_normal((n_clusters, 3, 3)))[0]
    which = rng.integers(0, n_clusters, size=n_clu)
    local = rng.standard_normal((n_clu, 3)) * stds[which]
    clu = centres[which] + np.einsum("nij,nj->ni", crot[which], local)
    d = rng.standard_normal((n_shell, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    shell = d * rng.uniform(10.0, 30.0, size=(n_shell, 1))
    means = np.concatenate([clu, shell], axis=0)
    perm = rng.permutation(n)
    means = means[perm]
    scales = np.exp(rng.normal(-4.0, 0.7, size=(n, 3)))
    quats = _unit_quaternions(rng, n)
    opac = _sigmoid(rng.normal(0.0, 1.5, size=n))
    sh = _sh_from_colour(rng, n, sh_degree, 0.05)
    return _finish(means, scales, quats, opac, sh, sh_degree,
                   {"kind": "cluster", "seed": seed, "clusters": n_clusters})


def look_at(eye, target=(0.0, 0.0, 0.0), down=(0.0, 1.0, 0.0)):
    """World->camera (R, t) for a camera at `eye` looking at `target`, with
    the image y axis along the world direction `down` (x right, z forward)."""
    eye = np.asarray(eye, np.float64)
    fwd = np.asarray(target, np.float64) - eye
    fwd /= np.linalg.norm(fwd)
    dn = np.asarray(down, np.float64)
    right = np.cross(dn, fwd)
    if np.linalg.norm(right) < 1e-6:          # looking along `down`
        right = np.cross(np.array([0.0, 0.0, 1.0]), fwd)
    right /= np.linalg.norm(right)
    dn2 = np.cross(fwd, right)
    R = np.stack([right, dn2, fwd], axis=0)
    t = -R @ eye
    return R, t


def fov_camera(R, t, width: int, height: int, fovx_deg: float = 60.0) -> Camera:
    fx = width / (2.0 * math.tan(math.radians(fovx_deg) / 2.0))
    return Camera(np.asarray(R, np.float64), np.asarray(t, np.float64), fx, fx,
                  width / 2.0, height / 2.0, int(width), int(height))


def origin_camera(width: int = 128, height: int = 128, f: float = 128.0) -> Camera:
    """Pinhole camera at the origin looking down +z (R = I, t = 0)."""
    return Camera(np.eye(3), np.zeros(3), f, f, width / 2.0, height / 2.0,
                  int(width), int(height))


def ring_camera(angle: float, width: int, height: int, radius: float = 4.0,
                fovx_deg: float = 60.0) -> Camera:
    """Camera on the y = 0 ring of the given radius, looking at the origin,
    image 'down' along world +y."""
    eye = (radius * math.sin(angle), 0.0, -radius * math.cos(angle))
    R, t = look_at(eye)
    return fov_camera(R, t, width, height, fovx_deg)


MULTIVIEW_SIZES = [(800, 800), (800, 800), (1280, 720), (1280, 720), (1280, 720),
                   (1600, 1063), (1600, 1063), (1920, 1080)]


def multiview_cameras(sizes=None) -> list[Camera]:
    """Eight ring views at angles 2*pi*k/8 with uneven sizes
    (2x 800x800, 3x 1280x720, 2x 1600x1063, 1x 1920x1080)."""
    sizes = MULTIVIEW_SIZES if sizes is None else sizes
    nv = len(sizes)
    return [ring_camera(2 * math.pi * k / nv, w, h) for k, (w, h) in enumerate(sizes)]


SERVE_SIZES = [(640, 480), (1280, 720), (1920, 1080), (3840, 2160)]


def sphere_camera(rng: np.random.Generator, sizes=None) -> Camera:
    """Random pose on a sphere of radius U[3, 6] looking at the origin, with a
    resolution drawn uniformly from `sizes` (fovx 60 degrees)."""
    sizes = SERVE_SIZES if sizes is None else sizes
    d = rng.standard_normal(3)
    d /= np.linalg.norm(d)
    eye = d * rng.uniform(3.0, 6.0)
    R, t = look_at(eye)
    w, h = sizes[int(rng.integers(0, len(sizes)))]
    return fov_camera(R, t, w, h)


def target_images(cams, seed: int = 1) -> list[np.ndarray]:
    """Uniform-noise target images, planar [3, H, W] float32 per view."""
    rng = np.random.default_rng(seed)
    return [rng.uniform(0.0, 1.0, size=(3, c.height, c.width)).astype(np.float32)
            for c in cams]
