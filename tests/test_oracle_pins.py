"""Pins of the CPU oracle against closed forms, library routines, invariants
and brute force (no GPU).  Each test names the passage of the paper whose
definition it checks.  None of these re-types the oracle's own formula."""
import math

import numpy as np
import pytest
import torch

from oracle import OracleConfig
from oracle import binning, densify, identify, project as P, render as R, prune, loss, sampling
from paper_2411_12788_gb300 import scenes

CFG = OracleConfig()


def _one_scene(means, scales, quats, opac, colours, sh_degree=0):
    n = len(means)
    k = (sh_degree + 1) ** 2
    sh = np.zeros((n, k, 3))
    sh[:, 0, :] = (np.asarray(colours, np.float64) - 0.5) / (0.5 / math.sqrt(math.pi))
    return scenes.Scene(np.asarray(means, np.float64), np.asarray(scales, np.float64),
                        np.asarray(quats, np.float64), np.asarray(opac, np.float64),
                        sh, sh_degree)


# ---------------------------------------------------------------- step P pins
def test_rotation_matches_scipy():
    """Sec. 3.1 covariance from a rotation: R(q) against scipy's quaternion
    conversion, plus orthonormality."""
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(5)
    q = rng.standard_normal((64, 4)) * rng.uniform(0.3, 3.0, (64, 1))  # unnormalised
    Rm = P.rotation_matrix(torch.tensor(q)).numpy()
    ref = Rotation.from_quat(q[:, [1, 2, 3, 0]]).as_matrix()
    np.testing.assert_allclose(Rm, ref, atol=1e-12)
    np.testing.assert_allclose(Rm @ Rm.transpose(0, 2, 1), np.broadcast_to(np.eye(3), Rm.shape), atol=1e-12)


def test_sh_basis_matches_scipy_complex_harmonics():
    """Sec. 3.1 view-dependent SH colour: the real basis equals sqrt2 Re/Im of
    scipy's complex Y_l^m (Condon-Shortley phase) and Y_00."""
    from scipy.special import sph_harm_y
    rng = np.random.default_rng(6)
    d = rng.standard_normal((200, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    Y = P.sh_basis(3, torch.tensor(d)).numpy()
    theta = np.arccos(np.clip(d[:, 2], -1, 1))
    phi = np.arctan2(d[:, 1], d[:, 0])
    for l in range(4):
        for m in range(-l, l + 1):
            c = sph_harm_y(l, abs(m), theta, phi)
            ref = c.real if m == 0 else math.sqrt(2) * (c.real if m > 0 else c.imag)
            np.testing.assert_allclose(Y[:, l * l + l + m], ref, atol=1e-12)


def test_sh_basis_orthonormal_by_quadrature():
    """Orthonormality of the real SH basis on the sphere (Gauss-Legendre in
    cos(theta) x uniform phi), degree 3 -> 16x16 identity Gram matrix."""
    xg, wg = np.polynomial.legendre.leggauss(16)
    nphi = 32
    phi = (np.arange(nphi) + 0.5) * 2 * math.pi / nphi
    ct, ph = np.meshgrid(xg, phi, indexing="ij")
    st = np.sqrt(1 - ct ** 2)
    d = np.stack([st * np.cos(ph), st * np.sin(ph), ct], -1).reshape(-1, 3)
    w = (wg[:, None] * np.full(nphi, 2 * math.pi / nphi)[None, :]).reshape(-1)
    Y = P.sh_basis(3, torch.tensor(d)).numpy()
    G = (Y * w[:, None]).T @ Y
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)


def test_degree0_colour_is_generated_colour():
    sc = scenes.box_scene(64, seed=3)
    cam = scenes.origin_camera()
    pr = P.project(sc.means, sc.scales, sc.rotations, sc.opacities, sc.sh, 0, cam)
    c = sc.sh[:, 0, :].astype(np.float64) * (0.5 / math.sqrt(math.pi)) + 0.5
    np.testing.assert_allclose(pr["rgb"].numpy(), c, atol=1e-6)


def test_covariance_eigen_structure():
    """Sigma = R diag(s^2) R^T: eigenvalues s^2, eigenvectors the columns of R(q)."""
    rng = np.random.default_rng(7)
    q = rng.standard_normal((16, 4))
    s = rng.uniform(0.1, 1.0, (16, 3))
    cam = scenes.origin_camera()
    pr = P.project(np.zeros((16, 3)) + [0, 0, 3], s, q, np.full(16, 0.5),
                   np.zeros((16, 1, 3)), 0, cam)
    cov = pr["cov3c"].numpy()   # camera R = I
    Rm = P.rotation_matrix(torch.tensor(q)).numpy()
    for k in range(16):
        np.testing.assert_allclose(Rm[k].T @ cov[k] @ Rm[k], np.diag(s[k] ** 2), atol=1e-12)


def test_ewa_jacobian_is_projection_derivative():
    """Sec. 3.1 local affine approximation: cov2d - lowpass I equals J cov J^T
    with J the numerical derivative of the pinhole map at the centre (inside
    the clamp), and the clamped Jacobian equals the one at the clamped point."""
    cam = scenes.fov_camera(*scenes.look_at((0.3, -0.2, -3.0)), 320, 240)
    rng = np.random.default_rng(8)
    n = 32
    means = rng.uniform(-0.5, 0.5, (n, 3))
    s = rng.uniform(0.01, 0.2, (n, 3))
    q = rng.standard_normal((n, 4))
    pr = P.project(means, s, q, np.full(n, 0.5), np.zeros((n, 1, 3)), 0, cam)
    pc = pr["p_c"].numpy()

    def proj(x):
        return np.array([cam.fx * x[0] / x[2] + cam.cx, cam.fy * x[1] / x[2] + cam.cy])
    for k in range(n):
        h = 1e-6
        J = np.stack([(proj(pc[k] + h * e) - proj(pc[k] - h * e)) / (2 * h) for e in np.eye(3)], 1)
        ref = J @ pr["cov3c"][k].numpy() @ J.T + CFG.lowpass * np.eye(2)
        np.testing.assert_allclose(pr["cov2d"][k].numpy(), ref, rtol=1e-6, atol=1e-6)
    # a centre far outside the frustum edge: J taken at the clamped direction
    far = np.array([[5.0, 0.1, 2.0]])
    prf = P.project(far, [[0.1, 0.1, 0.1]], [[1, 0, 0, 0]], [0.5], np.zeros((1, 1, 3)), 0,
                    scenes.origin_camera())
    lim = 1.3 * (128 / (2 * 128.0))
    xc = lim * 2.0
    J = np.array([[128 / 2.0, 0, -128 * xc / 4.0], [0, 128 / 2.0, -128 * 0.1 / 4.0]])
    ref = J @ (0.01 * np.eye(3)) @ J.T + CFG.lowpass * np.eye(2)
    np.testing.assert_allclose(prf["cov2d"][0].numpy(), ref, rtol=1e-12)


def test_midpoint_equals_max_density_and_discriminant():
    """Sec. 4.1: the chord midpoint of the unit ellipsoid equals the t of
    maximum Gaussian density along the ray (golden-section search), and the
    discriminant is >= 0 exactly when the ray meets the ellipsoid."""
    rng = np.random.default_rng(9)
    cam = scenes.origin_camera()
    n = 24
    means = np.stack([rng.uniform(-0.3, 0.3, n), rng.uniform(-0.3, 0.3, n), rng.uniform(2, 5, n)], 1)
    s = np.exp(rng.normal(-2.0, 0.6, (n, 3)))
    q = rng.standard_normal((n, 4))
    pr = P.project(means, s, q, np.full(n, 0.5), np.zeros((n, 1, 3)), 0, cam)
    u = rng.integers(40, 88, n)
    v = rng.integers(40, 88, n)
    dm = P.midpoint_depth(pr["p_c"], pr["ell"], u, v, cam).numpy()
    disc = P.midpoint_discriminant(pr["p_c"], pr["ell"], u, v, cam).numpy()
    for k in range(n):
        d = np.array([(u[k] + 0.5 - cam.cx) / cam.fx, (v[k] + 0.5 - cam.cy) / cam.fy, 1.0])
        E = np.linalg.inv(pr["cov3c"][k].numpy())
        p = pr["p_c"][k].numpy()
        f = lambda t: (t * d - p) @ E @ (t * d - p)      # -2 log density
        a, b = 0.0, 20.0
        g = (math.sqrt(5) - 1) / 2
        for _ in range(200):
            c1, c2 = b - g * (b - a), a + g * (b - a)
            if f(c1) < f(c2):
                b = c2
            else:
                a = c1
        assert abs(0.5 * (a + b) - dm[k]) < 1e-7 * max(1.0, dm[k])
        assert (disc[k] >= 0) == (f(0.5 * (a + b)) <= 1.0)


# ---------------------------------------------------------------- step R pins
def _iso_setup(o=0.8, s=0.02, z0=4.0, lowpass=0.3):
    sc = _one_scene([[0, 0, z0]], [[s, s, s]], [[1, 0, 0, 0]], [o], [[0.9, 0.4, 0.2]])
    return sc, scenes.origin_camera()


@pytest.mark.parametrize("o", [0.8, 0.999])
def test_single_isotropic_gaussian_closed_form(o):
    """Eq. 1 for one Gaussian on the optical axis: colour = alpha c with
    alpha = min(0.99, o exp(-r^2 / (2 sigma^2))), sigma^2 = (f s / z0)^2 + lowpass;
    I = sum of those alphas; d^mid = z0 / (1 + |r/f|^2) (Eq. 2)."""
    s, z0, f = 0.02, 4.0, 128.0
    sc, cam = _iso_setup(o=o, s=s, z0=z0)
    out = R.render(sc, [cam])[0]
    vv, uu = np.meshgrid(np.arange(128), np.arange(128), indexing="ij")
    dx = uu.reshape(-1) + 0.5 - 64
    dy = vv.reshape(-1) + 0.5 - 64
    sig2 = (f * s / z0) ** 2 + CFG.lowpass
    a = np.minimum(0.99, o * np.exp(-(dx ** 2 + dy ** 2) / (2 * sig2)))
    a = np.where(a >= 1 / 255, a, 0.0)
    col = out["colour"].numpy()
    np.testing.assert_allclose(col, a[:, None] * np.array([0.9, 0.4, 0.2])[None], atol=1e-12)
    np.testing.assert_allclose(out["t_final"].numpy(), 1 - a, atol=1e-12)
    np.testing.assert_allclose(out["weight_sum"].numpy()[0], a.sum(), rtol=1e-12)
    hit = a > 0
    assert out["max_area"][0].item() == hit.sum()
    assert np.all(out["imax"].numpy() == np.where(hit, 0, -1))
    d_ref = z0 / (1 + (dx / f) ** 2 + (dy / f) ** 2)
    np.testing.assert_allclose(out["depth"].numpy()[hit], d_ref[hit], rtol=1e-12)
    np.testing.assert_allclose(out["depth_blend"].numpy(), a * z0, rtol=1e-12)
    # d^center is the centre's depth wherever the Gaussian is the max-weight one
    np.testing.assert_array_equal(out["depth_center"].numpy(), np.where(hit, z0, 0.0))
    if o >= 0.99 / math.exp(-(0.5 ** 2 * 2) / (2 * sig2)):
        # the four central pixels are clamped to exactly alpha_max
        centre = (np.abs(dx) == 0.5) & (np.abs(dy) == 0.5)
        np.testing.assert_array_equal(col[centre, 0], 0.99 * 0.9)


def test_two_gaussians_front_to_back():
    """Eq. 1 with two overlapping Gaussians: c = a1 c1 + (1 - a1) a2 c2 where
    the nearer one is first, whatever the input order."""
    c1, c2 = [0.9, 0.1, 0.1], [0.1, 0.1, 0.9]
    sc = _one_scene([[0, 0, 6.0], [0, 0, 3.0]], [[0.05] * 3, [0.03] * 3],
                    [[1, 0, 0, 0]] * 2, [0.7, 0.6], [c2, c1])
    cam = scenes.origin_camera()
    out = R.render(sc, [cam])[0]
    vv, uu = np.meshgrid(np.arange(128), np.arange(128), indexing="ij")
    r2 = (uu.reshape(-1) + 0.5 - 64) ** 2 + (vv.reshape(-1) + 0.5 - 64) ** 2

    def alpha(o, s, z):
        a = np.minimum(0.99, o * np.exp(-r2 / (2 * ((128 * s / z) ** 2 + 0.3))))
        return np.where(a >= 1 / 255, a, 0.0)
    a_front, a_back = alpha(0.6, 0.03, 3.0), alpha(0.7, 0.05, 6.0)
    ref = a_front[:, None] * np.array(c1) + ((1 - a_front) * a_back)[:, None] * np.array(c2)
    np.testing.assert_allclose(out["colour"].numpy(), ref, atol=1e-12)


def test_order_invariance_for_disjoint_supports():
    """Eq. 1 is order-independent when no two supports overlap: permuting the
    Gaussians and their depths gives the same image."""
    rng = np.random.default_rng(11)
    grid = [(x, y) for x in np.linspace(-0.8, 0.8, 5) for y in np.linspace(-0.8, 0.8, 5)]
    n = len(grid)
    z = rng.uniform(3, 5, n)
    means = np.array([[gx * zz / 2, gy * zz / 2, zz] for (gx, gy), zz in zip(grid, z)])
    sc = _one_scene(means, np.full((n, 3), 0.01), rng.standard_normal((n, 4)),
                    rng.uniform(0.3, 0.9, n), rng.uniform(0, 1, (n, 3)))
    cam = scenes.origin_camera()
    a = R.render(sc, [cam])[0]["colour"].numpy()
    perm = rng.permutation(n)
    sc2 = sc.subset(perm)
    # move every Gaussian along its own ray to a new depth: same image footprint
    newz = rng.uniform(3, 5, n)
    sc2.means = sc2.means * (newz / sc2.means[:, 2])[:, None]
    sc2.scales = sc2.scales * (newz / sc.subset(perm).means[:, 2])[:, None]
    b = R.render(sc2, [cam])[0]["colour"].numpy()
    np.testing.assert_allclose(a, b, atol=1e-12)


def test_alpha_skip_threshold():
    """alpha < 1/255 is skipped, alpha >= 1/255 is blended: a Gaussian at the
    exact centre of pixel (63, 63) whose opacity sits just below / above."""
    cam = scenes.origin_camera()
    z = 4.0
    x = -z / 256.0                    # fx * x / z + cx = 63.5 exactly
    for o, blended in [(1 / 255 * (1 - 1e-9), False), (1 / 255 * (1 + 1e-9), True)]:
        sc = _one_scene([[x, x, z]], [[0.02] * 3], [[1, 0, 0, 0]], [o], [[1, 1, 1]])
        out = R.render(sc, [cam], pix=[np.array([[63, 63]])])[0]
        assert (out["n_blended"][0].item() == 1) == blended


def test_termination_stack_blends_13():
    """Early termination: 20 Gaussians of opacity 0.5 centred exactly on a
    pixel centre give alpha = 0.5 each; 0.5^13 >= 1e-4 > 0.5^14, so exactly 13
    are blended and the colour is sum_k 0.5^k c_k."""
    cam = scenes.origin_camera()
    zs = 4.0 + 0.25 * np.arange(20)
    means = np.stack([-zs / 256, -zs / 256, zs], 1)
    rng = np.random.default_rng(12)
    cols = rng.uniform(0, 1, (20, 3))
    sc = _one_scene(means, np.full((20, 3), 0.02), [[1, 0, 0, 0]] * 20, np.full(20, 0.5), cols)
    out = R.render(sc, [cam], pix=[np.array([[63, 63]])])[0]
    assert out["n_blended"][0].item() == 13
    ref = sum(0.5 ** (k + 1) * cols[k] for k in range(13))
    np.testing.assert_allclose(out["colour"][0].numpy(), ref, atol=1e-15)
    assert out["t_final"][0].item() == 0.5 ** 13
    assert out["last"][0].item() == 12
    assert out["imax"][0].item() == 0          # equal first weight 0.5 > later


def test_argmax_tie_keeps_front():
    """i_max = argmax w (Eq. 2); an exact tie keeps the nearer Gaussian:
    alpha 0.5 then alpha 1.0 clamped to... use 0.5 and 1.0 -> weights 0.5, 0.495."""
    cam = scenes.origin_camera()
    zs = np.array([4.0, 4.5])
    means = np.stack([-zs / 256, -zs / 256, zs], 1)
    # front alpha a1, back alpha a2 with (1 - a1) a2 == a1  -> a2 = a1 / (1 - a1)
    a1 = 0.25
    a2 = a1 / (1 - a1)
    sc = _one_scene(means, np.full((2, 3), 0.02), [[1, 0, 0, 0]] * 2, [a1, a2],
                    [[1, 0, 0], [0, 0, 1]])
    out = R.render(sc, [cam], pix=[np.array([[63, 63]])])[0]
    assert out["wmax"][0].item() == pytest.approx(0.25, abs=1e-15)
    assert out["imax"][0].item() == 0


def _brute_pixel(mean2d, conic, opac, rgb, z, u, v, cfg):
    """Sequential per-pixel loop of Eq. 1 (stops before the entry that would
    bring T below t_min)."""
    order = sorted(range(len(z)), key=lambda i: (np.float32(z[i]), i))
    T, C, wmax, imax, db = 1.0, np.zeros(3), 0.0, -1, 0.0
    wsum = np.zeros(len(z))
    for i in order:
        dx, dy = u + 0.5 - mean2d[i][0], v + 0.5 - mean2d[i][1]
        qq = conic[i][0] * dx * dx + 2 * conic[i][1] * dx * dy + conic[i][2] * dy * dy
        a = min(cfg.alpha_max, opac[i] * math.exp(-0.5 * qq))
        if a < cfg.alpha_min:
            continue
        if T * (1 - a) < cfg.t_min:
            break
        w = a * T
        C += w * rgb[i]
        db += w * z[i]
        wsum[i] += w
        if w > wmax:
            wmax, imax = w, i
        T *= 1 - a
    return C, T, imax, wmax, db, wsum


def test_dense_renderer_matches_sequential_loop():
    """Brute force: the vectorised oracle equals a plain per-pixel loop on a
    small random scene with heavy overlap (high opacities)."""
    rng = np.random.default_rng(13)
    n = 24
    sc = _one_scene(np.stack([rng.uniform(-0.3, 0.3, n), rng.uniform(-0.3, 0.3, n), rng.uniform(2, 4, n)], 1),
                    np.exp(rng.normal(-2.0, 0.4, (n, 3))), rng.standard_normal((n, 4)),
                    rng.uniform(0.5, 1.0, n), rng.uniform(0, 1, (n, 3)))
    cam = scenes.origin_camera(24, 24, 40.0)
    pr = P.project(sc.means, sc.scales, sc.rotations, sc.opacities, sc.sh, 0, cam)
    out = R.render_view(pr, cam)
    m2, cn, op, rgb, z = (pr[k].detach().numpy() for k in ("mean2d", "conic", "opacity", "rgb", "z"))
    wsum = np.zeros(n)
    for p, (u, v) in enumerate(zip(out["u"].numpy(), out["v"].numpy())):
        C, T, imax, wmax, db, ws = _brute_pixel(m2, cn, op, rgb, z, u, v, CFG)
        np.testing.assert_allclose(out["colour"][p].numpy(), C, atol=1e-13)
        assert abs(out["t_final"][p].item() - T) < 1e-13
        assert out["imax"][p].item() == imax
        assert abs(out["depth_blend"][p].item() - db) < 1e-12
        wsum += ws
    np.testing.assert_allclose(out["weight_sum"].numpy(), wsum, atol=1e-12)
    assert (out["n_blended"] > 3).float().mean() > 0.3     # the case is not trivial
    assert (out["t_final"] < 1e-3).any()                    # and some pixels stop early


# ---------------------------------------------------------------- step B pins
def test_rect_min_q_against_dense_sampling():
    """Exact min of the conic quadratic over a tile rectangle against dense
    sampling of the rectangle (never below it, and within the grid step)."""
    rng = np.random.default_rng(14)
    for _ in range(200):
        L = np.tril(rng.normal(0, 1, (2, 2)))
        Sig = L @ L.T + 0.1 * np.eye(2)
        Ci = np.linalg.inv(Sig)
        mx, my = rng.uniform(-40, 56, 2)
        xs = np.linspace(0.5, 15.5, 301)
        X, Y = np.meshgrid(xs, xs, indexing="ij")
        dx, dy = X - mx, Y - my
        qd = Ci[0, 0] * dx * dx + 2 * Ci[0, 1] * dx * dy + Ci[1, 1] * dy * dy
        m = binning.rect_min_q(Ci[0, 0], Ci[0, 1], Ci[1, 1], mx, my, 0.5, 15.5, 0.5, 15.5)
        assert m <= qd.min() + 1e-9
        # the grid misses the true minimiser by at most half a step
        assert qd.min() - m <= 1e-3 * max(1.0, qd.min()) + 0.2 * np.abs(Ci).max() * 0.05 * 40


def test_tile_lists_cover_every_supporting_pixel():
    """Every pixel with o G >= alpha_min (per-pixel brute force) lies in a
    kept tile of that Gaussian, and every kept tile has its rectangle's min q
    <= tau (no tile is kept for nothing)."""
    sc = scenes.box_scene(200, seed=15)
    cam = scenes.origin_camera(96, 80, 100.0)
    pr = P.project(sc.means, sc.scales, sc.rotations, sc.opacities, sc.sh, 0, cam)
    m2, cn = pr["mean2d"].numpy(), pr["conic"].numpy()
    g, t, near, _, _ = binning.tile_lists(m2, cn, sc.opacities, pr["valid"].numpy(), 96, 80)
    kept = set(zip(g.tolist(), t.tolist()))
    vv, uu = np.meshgrid(np.arange(80), np.arange(96), indexing="ij")
    uu, vv = uu.reshape(-1), vv.reshape(-1)
    tx_n = 6
    for i in range(200):
        if not pr["valid"][i]:
            continue
        dx, dy = uu + 0.5 - m2[i, 0], vv + 0.5 - m2[i, 1]
        q = cn[i, 0] * dx * dx + 2 * cn[i, 1] * dx * dy + cn[i, 2] * dy * dy
        a = sc.opacities[i] * np.exp(-0.5 * q)
        sup = a >= 1 / 255
        for tt in set(((vv[sup] // 16) * tx_n + uu[sup] // 16).tolist()):
            assert (i, tt) in kept
    assert len(g) > 200


def test_three_sigma_radius_against_eigvalsh():
    """lambda_max in closed form agrees with numpy's symmetric eigensolver, and
    r = ceil(3 sqrt(lambda_max)) on matrices with known eigenvalues."""
    rng = np.random.default_rng(21)
    for _ in range(200):
        L = rng.normal(size=(2, 2)) * rng.uniform(0.1, 30)
        S = L @ L.T + 0.3 * np.eye(2)
        ref = np.linalg.eigvalsh(S)[-1]
        assert abs(binning.lambda_max(S[0, 0], S[1, 1], S[0, 1]) - ref) <= 1e-12 * ref
    # eigenvalues (4, 1): diagonal and rotated by 45 degrees; (2, 2)
    assert binning.three_sigma_radius(4.0, 1.0, 0.0) == 6.0
    assert binning.three_sigma_radius(2.5, 2.5, 1.5) == 6.0
    assert binning.three_sigma_radius(2.0, 2.0, 0.0) == math.ceil(3 * math.sqrt(2))


def test_square_tile_range_brute_force():
    """The tiles whose pixel centres meet [m - r, m + r], by enumerating the
    centres, equal the closed-form range (clipped to the grid)."""
    rng = np.random.default_rng(22)
    for _ in range(500):
        n = int(rng.integers(1, 12))
        m = rng.uniform(-40, 16 * n + 40)
        r = float(rng.integers(1, 40))
        lo, hi = binning.square_tile_range(m, r, n)
        centres = np.arange(16 * n) + 0.5
        hit = np.abs(centres - m) <= r
        ref = sorted(set((np.nonzero(hit)[0] // 16).tolist()))
        got = list(range(int(lo), int(hi) + 1))
        assert got == ref, (m, r, n, got, ref)


def test_three_sigma_extent_truncates_the_support():
    """One opaque Gaussian whose exact support (3.33 sigma at o = 0.99) reaches
    past its 3-sigma square: in the 3sigma extent the pixels of tiles the
    square misses get the background, the others the exact-extent colour;
    the tile lists are the square's tiles."""
    s, z0 = 0.1, 4.0
    # sigma^2 = (128 s / z0)^2 + 0.3 = 10.54 px^2: r = ceil(3 sigma) = 10 px
    # while the exact support reaches sigma sqrt(2 ln(0.99 * 255)) = 10.8 px;
    # centred at (54, 54) the square ends at 64 < 64.5, the first pixel
    # centre of the next tile, which the exact support still reaches
    sc = _one_scene([[(54.0 - 64.0) * z0 / 128.0, (54.0 - 64.0) * z0 / 128.0, z0]], [[s, s, s]],
                    [[1, 0, 0, 0]], [0.99], [[0.9, 0.4, 0.2]])
    cam = scenes.origin_camera()
    exact = R.render(sc, [cam])[0]
    tri = R.render(sc, [cam], cfg=OracleConfig(extent="3sigma"))[0]
    pr = P.project(sc.means, sc.scales, sc.rotations, sc.opacities, sc.sh, 0, cam)
    cov = pr["cov2d"].numpy()[0]
    r = binning.three_sigma_radius(cov[0, 0], cov[1, 1], cov[0, 1])
    m = pr["mean2d"].numpy()[0]
    assert r == 10.0 and np.allclose(m, 54.0)
    x0, x1 = binning.square_tile_range(m[0], r, 8)
    y0, y1 = binning.square_tile_range(m[1], r, 8)
    u, v = tri["u"].numpy(), tri["v"].numpy()
    inside = (u // 16 >= x0) & (u // 16 <= x1) & (v // 16 >= y0) & (v // 16 <= y1)
    ce, ct = exact["colour"].numpy(), tri["colour"].numpy()
    np.testing.assert_array_equal(ct[inside], ce[inside])
    assert np.all(ct[~inside] == 0.0)
    assert (ce[~inside, 0] > 0).sum() > 0           # the exact support reaches past the square's tiles
    g, t, _, _, _ = binning.tile_lists(pr["mean2d"].numpy(), pr["conic"].numpy(), [0.99], [True], 128, 128,
                                       extent="3sigma")
    assert sorted(t.tolist()) == sorted(ty * 8 + tx for ty in range(y0, y1 + 1) for tx in range(x0, x1 + 1))


def test_sort_and_ranges_on_handmade_keys():
    """Stable (tile, z) order and [start, end) ranges on a hand-made list."""
    tile = np.array([3, 1, 3, 0, 1, 3])
    z = np.array([2.0, 5.0, 1.0, 9.0, 5.0, 1.0], np.float32)
    order = binning.sort_entries(tile, z, None)
    assert order.tolist() == [3, 1, 4, 2, 5, 0]     # equal z keep input order
    rng_ = binning.tile_ranges(tile[order], 5)
    assert rng_.tolist() == [[0, 1], [1, 3], [3, 3], [3, 6], [6, 6]]
    assert binning.exclusive_scan([3, 0, 2, 5]).tolist() == [0, 3, 3, 5]


# ---------------------------------------------------------------- misc pins
def test_keep_top_ties_by_index():
    w = np.array([0.5, 2.0, 0.5, 1.0, 0.5, 3.0])
    assert prune.keep_top(w, 0.5).tolist() == [1, 3, 5]
    assert prune.keep_top(w, 0.6).tolist() == [0, 1, 3, 5]      # ceil(3.6) = 4


def test_keep_quantile_by_hand():
    # M = 5 positive values, q = 0.5 -> ceil(2.5) = 3 kept: the 3, 3 and 2
    v = np.array([0.0, 3.0, 1.0, 3.0, 2.0, 0.5])
    assert identify.keep_quantile(v, 0.5).tolist() == [False, True, False, True, True, False]
    # ties at the boundary go to the lower index; zeros are never kept
    t = np.array([1.0, 2.0, 2.0, 2.0, 0.0, 1.0])
    # (q in single precision: 0.3f * 5 = 1.50000006 -> 2; 0.4f * 5 = 2.00000003 -> 3)
    assert np.nonzero(identify.keep_quantile(t, 0.3))[0].tolist() == [1, 2]
    assert np.nonzero(identify.keep_quantile(t, 0.4))[0].tolist() == [1, 2, 3]
    assert np.nonzero(identify.keep_quantile(t, 0.61))[0].tolist() == [0, 1, 2, 3]  # 4th: the lower-index 1
    assert not identify.keep_quantile(np.zeros(7), 0.99).any()
    assert identify.keep_quantile(t, 1.0).sum() == 5 and not identify.keep_quantile(t, 0.0).any()
    # q is the single-precision 0.99 (0.99000000953...): 1000 values keep 991, 100 keep all 100
    assert identify.keep_count(1000, 0.99) == 991 and identify.keep_count(100, 0.99) == 100
    assert identify.keep_quantile(np.arange(1.0, 1001.0), 0.99).sum() == 991
    assert not identify.keep_quantile(np.arange(1.0, 1001.0), 0.99)[:9].any()


def test_blur_split_threshold_by_hand():
    # theta = 2e-4 in single precision is 1.99999995e-4: 100 x 100 -> S > 1.99999995,
    # 400 x 250 -> S > 19.9999995
    assert identify.blur_split([0, 1, 2, 3, 10], 100, 100).tolist() == [False, False, True, True, True]
    assert identify.blur_split([19, 20], 250, 400).tolist() == [False, True]
    assert identify.intersected([0, 1, 5]).tolist() == [False, True, True]


def test_critical_by_hand():
    imax = np.array([0, 0, 1, -1, 2, 2])
    wmax = np.array([0.9, 0.2, 0.5, 0.0, 0.1, 0.05])
    # 5 pixels with a contributor, q = 0.5 keeps 3: w 0.9 (G0), 0.5 (G1), 0.2 (G0)
    assert identify.critical(imax, wmax, 0.5, 4).tolist() == [True, True, False, False]
    assert identify.critical(imax, wmax, 1.0, 4).tolist() == [True, True, True, False]


def test_identify_on_rendered_separated_gaussians():
    # Disjoint isotropic Gaussians: every touched pixel has one contributor, so
    # S_i is the number of pixels with o exp(-q/2) >= 1/255 (counted by brute
    # force here) and I_i the sum of those alphas.
    W = H = 256
    cam = scenes.origin_camera(W, H, 256.0)
    cx = np.array([-0.6, 0.0, 0.6])
    sig = np.array([0.004, 0.02, 0.06])          # world std at z = 4 -> 0.26, 1.3, 3.8 px
    o = np.array([0.1, 0.5, 0.8])
    means = np.stack([cx * 4 / 4, np.zeros(3), np.full(3, 4.0)], 1)
    sc = scenes.Scene(means.astype(np.float32), np.repeat(sig[:, None], 3, 1).astype(np.float32),
                      np.tile(np.array([1.0, 0, 0, 0], np.float32), (3, 1)), o.astype(np.float32),
                      (np.full((3, 1, 3), 0.3, np.float32)), 0)
    with torch.no_grad():
        pr = P.project(sc.means, sc.scales, sc.rotations, sc.opacities, sc.sh, 0, cam)
        out = R.render_view(pr, cam)
    S = out["max_area"].numpy()
    u, v = np.meshgrid(np.arange(W) + 0.5, np.arange(H) + 0.5)
    for i in range(3):
        m = pr["mean2d"][i].numpy()
        A, B, C = pr["conic"][i].numpy()
        dx, dy = u - m[0], v - m[1]
        a = o[i] * np.exp(-0.5 * (A * dx * dx + 2 * B * dx * dy + C * dy * dy))
        assert S[i] == np.sum(a >= 1 / 255)
    # threshold 2e-4 * 256^2 = 13.1 px: the two larger ones are blur-split candidates
    assert identify.blur_split(S, H, W).tolist() == [False, True, True]
    I = out["weight_sum"].numpy()
    vis = identify.visible(I, 0.5)                 # ceil(1.5) = 2 of 3
    assert vis.tolist() == (I >= np.sort(I)[1]).tolist()


def test_weighted_sample_first_draw_is_proportional():
    # exponential clocks: the first to ring is i with probability I_i / sum I
    rng = np.random.default_rng(3)
    I = np.array([1.0, 2.0, 3.0, 4.0, 0.0])
    T = 200000
    E = rng.exponential(size=(T, 5)).astype(np.float32)
    first = np.argmax((I.astype(np.float32) / E), axis=1)
    freq = np.bincount(first, minlength=5) / T
    assert np.allclose(freq, I / I.sum(), atol=4e-3)
    # and the oracle's draw of one is that Gaussian
    for t in range(50):
        assert sampling.weighted_sample(I, E[t], 1).tolist() == [first[t]]


def test_weighted_sample_two_draws_match_sequential_law():
    # inclusion probability of i in two successive proportional draws without
    # replacement: p_i + sum_{j != i} p_j p_i / (1 - p_j)
    rng = np.random.default_rng(4)
    I = np.array([5.0, 1.0, 3.0, 1.0])
    p = I / I.sum()
    incl = np.array([p[i] + sum(p[j] * p[i] / (1 - p[j]) for j in range(4) if j != i) for i in range(4)])
    T = 60000
    counts = np.zeros(4)
    E = rng.exponential(size=(T, 4)).astype(np.float32)
    for t in range(T):
        counts[sampling.weighted_sample(I, E[t], 2)] += 1
    assert np.allclose(counts / T, incl, atol=6e-3)


def test_weighted_sample_edges():
    I = np.array([0.0, 2.0, 0.0, 1.0, 3.0])
    E = np.ones(5, np.float32)
    assert sampling.weighted_sample(I, E, 10).tolist() == [1, 3, 4]      # zeros never drawn
    assert sampling.weighted_sample(I, E, 2).tolist() == [1, 4]
    assert sampling.weighted_sample(I, E, 0).tolist() == []
    # equal keys: the lower index first
    assert sampling.weighted_sample([1.0, 1.0, 1.0], np.ones(3, np.float32), 2).tolist() == [0, 1]


def test_reprojection_inverts_the_pinhole_projection():
    R, t = scenes.look_at((0.7, -0.4, 0.2), (0.0, 0.0, 4.0))
    cam = scenes.fov_camera(R, t, 64, 48, 55.0)
    rng = np.random.default_rng(5)
    pix = rng.integers(0, 64 * 48, 40)
    depth = np.zeros(64 * 48)
    depth[pix] = rng.uniform(1.0, 9.0, 40)
    P = sampling.reproject(depth, pix, cam)
    pc = P @ np.asarray(cam.R, np.float64).T + np.asarray(cam.t, np.float64)
    assert np.allclose(pc[:, 2], depth[pix], rtol=1e-12)
    assert np.allclose(cam.fx * pc[:, 0] / pc[:, 2] + cam.cx, pix % 64 + 0.5, atol=1e-9)
    assert np.allclose(cam.fy * pc[:, 1] / pc[:, 2] + cam.cy, pix // 64 + 0.5, atol=1e-9)


def test_depth_points_draws_among_valid_pixels():
    cam = scenes.origin_camera(8, 4, 8.0)
    rng = np.random.default_rng(6)
    depth = rng.uniform(1, 3, 32)
    depth[[3, 9]] = 0.0
    imax = np.where(np.arange(32) % 5 == 0, -1, 7)
    u = rng.uniform(size=32)
    target = rng.uniform(size=(3, 4, 8))
    out = sampling.depth_points(depth, imax, target, u, cam, 6)
    valid = (imax >= 0) & (depth > 0)
    sel = out["pixel_idx"]
    assert len(sel) == 6 and valid[sel].all()
    assert u[sel].min() >= u[valid & ~np.isin(np.arange(32), sel)].max()
    assert np.array_equal(out["colours"], target.reshape(3, -1)[:, sel].T)
    assert len(sampling.depth_points(depth, imax, target, u, cam, 1000)["pixel_idx"]) == valid.sum()


@pytest.mark.parametrize("o", [0.02, 0.3, 0.75, 0.99])
def test_clone_pair_keeps_peak_opacity_and_line_integral(o):
    # two coincident clones composite to 1 - (1 - o')^2 = o at the centre
    on = densify.clone_opacity(o)
    assert abs(1 - (1 - on) ** 2 - o) < 1e-14
    # and along a line through the centre (1-D profile g(x) = exp(-x^2 / 2s^2))
    # the pair's composited opacity integrates to the original's
    s = 1.7
    f = densify.clone_scale_factor(o)
    x = np.linspace(-40, 40, 400001)
    g1 = np.exp(-0.5 * (x / (f * s)) ** 2)
    pair = 1 - (1 - on * g1) ** 2
    assert abs(np.trapezoid(pair, x) - np.trapezoid(o * np.exp(-0.5 * (x / s) ** 2), x)) < 1e-9


def test_clone_by_hand():
    # o = 0.75: o' = 0.5, scale factor 0.75 / (1 - 0.25 / sqrt 2)
    assert abs(densify.clone_opacity(0.75) - 0.5) < 1e-15
    assert abs(densify.clone_scale_factor(0.75) - 0.75 / (1 - 0.25 / np.sqrt(2))) < 1e-15
    m = np.arange(12.0).reshape(4, 3)
    out = densify.clone(m, np.ones((4, 3)), np.tile([1.0, 0, 0, 0], (4, 1)), np.array([0.1, 0.75, 0.2, 0.5]),
                        np.zeros((4, 1, 3)), [1, 3])
    assert out["means"].shape == (6, 3) and np.array_equal(out["means"][4], m[1]) and np.array_equal(out["means"][5], m[3])
    assert np.allclose(out["opacities"], [0.1, 0.5, 0.2, 1 - np.sqrt(0.5), 0.5, 1 - np.sqrt(0.5)])
    assert np.allclose(out["scales"][[0, 2]], 1.0)


def test_ssim_window_closed_form():
    w = loss.gaussian_window()
    g = w[5] / w[5].sum()
    assert abs(float(w.sum()) - 1) < 1e-14 and torch.allclose(w, w.T) and torch.allclose(g, g.flip(0))
    assert abs(float(g[5] / g[6]) - np.exp(1 / 4.5)) < 1e-12 and abs(float(g[5] / g[0]) - np.exp(25 / 4.5)) < 1e-9


def test_ssim_of_identical_images_is_one():
    x = torch.rand(3, 23, 17, dtype=torch.float64, generator=torch.Generator().manual_seed(1))
    assert torch.allclose(loss.ssim_map(x, x), torch.ones(3, 23, 17, dtype=torch.float64), atol=1e-14)


def test_ssim_constant_images_closed_form():
    # away from the border (window fully inside) mu = a, b and every sigma is 0
    a, b = 0.3, 0.7
    s = loss.ssim_map(torch.full((1, 20, 20), a, dtype=torch.float64), torch.full((1, 20, 20), b, dtype=torch.float64))
    ref = (2 * a * b + loss.SSIM_C1) / (a * a + b * b + loss.SSIM_C1)
    assert torch.allclose(s[0, 5:15, 5:15], torch.full((10, 10), ref, dtype=torch.float64), atol=1e-14)


def test_ssim_matches_explicit_window_sums():
    # brute force: every window sum written out pixel by pixel, zero padding
    rng = np.random.default_rng(2)
    x, y = rng.uniform(size=(2, 1, 9, 13))
    g1 = np.exp(-np.arange(-5, 6) ** 2 / 4.5)
    g1 /= g1.sum()
    H, W = 9, 13
    ref = np.zeros((H, W))
    for i in range(H):
        for j in range(W):
            m = np.zeros(5)
            for di in range(-5, 6):
                for dj in range(-5, 6):
                    u, v = i + di, j + dj
                    if 0 <= u < H and 0 <= v < W:
                        w = g1[di + 5] * g1[dj + 5]
                        xv, yv = x[0, u, v], y[0, u, v]
                        m += w * np.array([xv, yv, xv * xv, yv * yv, xv * yv])
            mx, my, exx, eyy, exy = m
            ref[i, j] = ((2 * mx * my + 1e-4) * (2 * (exy - mx * my) + 9e-4)) / (
                (mx * mx + my * my + 1e-4) * (exx - mx * mx + eyy - my * my + 9e-4))
    got = loss.ssim_map(torch.from_numpy(x), torch.from_numpy(y))[0].numpy()
    assert np.allclose(got, ref, atol=1e-13)


def test_l1_ssim_gradient_matches_central_differences():
    rng = np.random.default_rng(3)
    x = torch.from_numpy(rng.uniform(size=(3, 7, 8))).requires_grad_(True)
    y = torch.from_numpy(rng.uniform(size=(3, 7, 8)))
    L, _, _ = loss.l1_ssim([x], [y], 0.2)
    (g,) = torch.autograd.grad(L, x)
    h = 1e-6
    for idx in [(0, 0, 0), (1, 3, 4), (2, 6, 7), (0, 2, 5)]:
        xp, xm = x.detach().clone(), x.detach().clone()
        xp[idx] += h
        xm[idx] -= h
        fd = (loss.l1_ssim([xp], [y], 0.2)[0] - loss.l1_ssim([xm], [y], 0.2)[0]) / (2 * h)
        assert abs(float(fd) - float(g[idx])) < 1e-7


def test_l1_loss_closed_form():
    a = torch.zeros(3, 2, 2)
    b = torch.ones(3, 2, 2) * 0.25
    assert loss.l1([a], [b]).item() == 0.25


# ---------------------------------------------------------------- gradients
def _event_signature(pr, cam, cfg):
    out = R.render_view(pr, cam, cfg, want_depth=False)
    return out


def test_autograd_gradient_matches_central_differences():
    """The oracle's gradient (autograd of the forward) against central finite
    differences (h = 1e-4 in float64) of the L1 loss, for every parameter
    kind; parameters whose +-h changes a discrete event (skip, stop, clamp)
    are excluded and must be rare."""
    rng = np.random.default_rng(16)
    n = 12
    sc = _one_scene(np.stack([rng.uniform(-0.25, 0.25, n), rng.uniform(-0.25, 0.25, n), rng.uniform(2, 4, n)], 1),
                    np.exp(rng.normal(-2.6, 0.4, (n, 3))), rng.standard_normal((n, 4)),
                    rng.uniform(0.3, 0.95, n), rng.uniform(0, 1, (n, 3)), sh_degree=1)
    sc.sh[:, 1:, :] = rng.normal(0, 0.2, (n, 3, 3))
    cam = scenes.fov_camera(*scenes.look_at((0.2, 0.1, -0.5), (0, 0, 3)), 24, 20)
    target = torch.tensor(rng.uniform(0, 1, (20 * 24, 3)))
    params = [torch.tensor(np.asarray(a, np.float64), requires_grad=True)
              for a in (sc.means, sc.scales, sc.rotations, sc.opacities, sc.sh)]

    def lossf(ps, events=False):
        pr = P.project(*ps, 1, cam)
        out = R.render_view(pr, cam, want_depth=False)
        L = torch.abs(out["colour"] - target).mean()
        if events:
            alpha = None
            return L, out
        return L
    L = lossf(params)
    grads = torch.autograd.grad(L, params)
    _, base = lossf([p.detach() for p in params], events=True)

    def events(ps):
        with torch.no_grad():
            pr = P.project(*ps, 1, cam)
            o = R.render_view(pr, cam, want_depth=False)
        return (o["n_blended"].numpy().copy(), o["last"].numpy().copy(),
                torch.sign(o["colour"] - target).numpy().copy())
    ev0 = events([p.detach() for p in params])
    h = 1e-4
    checked = excluded = 0
    for pi, (p, g) in enumerate(zip(params, grads)):
        flat = p.detach().reshape(-1)
        for j in range(flat.numel()):
            vals = []
            evs = []
            for sgn in (1, -1):
                ps = [q.detach().clone() for q in params]
                ps[pi].view(-1)[j] += sgn * h
                with torch.no_grad():
                    vals.append(lossf(ps).item())
                evs.append(events(ps))
            same = all(all(np.array_equal(a, b) for a, b in zip(ev0, e)) for e in evs)
            if not same:
                excluded += 1
                continue
            fd = (vals[0] - vals[1]) / (2 * h)
            an = g.reshape(-1)[j].item()
            assert abs(fd - an) <= 1e-6 + 1e-4 * abs(an), (pi, j, fd, an)
            checked += 1
    assert excluded <= 0.02 * (checked + excluded)
    assert checked > 200


def test_conic_and_centre_of_projected_gaussian():
    """Sec. 3.1: the 2-D Gaussian's quadratic form is the inverse of the
    projected covariance, and its centre is the pinhole image of p_i."""
    sc = scenes.box_scene(64, seed=17)
    cam = scenes.fov_camera(*scenes.look_at((0.4, 0.3, -1.0), (0, 0, 4)), 200, 150)
    pr = P.project(sc.means, sc.scales, sc.rotations, sc.opacities, sc.sh, 0, cam)
    A, B, C = pr["conic"].numpy().T
    con = np.stack([np.stack([A, B], -1), np.stack([B, C], -1)], -2)
    np.testing.assert_allclose(con @ pr["cov2d"].numpy(), np.broadcast_to(np.eye(2), con.shape), atol=1e-9)
    pc = sc.means.astype(np.float64) @ cam.R.T + cam.t
    uv = np.stack([cam.fx * pc[:, 0] / pc[:, 2] + cam.cx, cam.fy * pc[:, 1] / pc[:, 2] + cam.cy], 1)
    np.testing.assert_allclose(pr["mean2d"].numpy(), uv, rtol=1e-12)


def test_sh_view_direction_points_from_camera_to_gaussian():
    """Sec. 3.1 view-dependent colour: with only band-1 coefficients the colour
    is 0.5 + sqrt(3/(4 pi)) (-y, z, -x) . coefficients of the unit vector from the
    camera centre (-R^T t) to the Gaussian."""
    ang = 0.7
    cam = scenes.ring_camera(ang, 64, 64)
    eye = np.array([4 * math.sin(ang), 0.0, -4 * math.cos(ang)])
    p = np.array([[0.3, -0.2, 0.1]])
    sh = np.zeros((1, 4, 3))
    sh[0, 1, 0] = 1.0       # m = -1 -> red channel
    sh[0, 2, 1] = 1.0       # m = 0  -> green
    sh[0, 3, 2] = 1.0       # m = +1 -> blue
    pr = P.project(p, [[0.1] * 3], [[1, 0, 0, 0]], [0.5], sh, 1, cam)
    d = (p[0] - eye) / np.linalg.norm(p[0] - eye)
    k = math.sqrt(3 / (4 * math.pi))
    ref = np.maximum(0.0, 0.5 + k * np.array([-d[1], d[2], -d[0]]))
    np.testing.assert_allclose(pr["rgb"][0].numpy(), ref, atol=1e-12)


def test_anisotropic_alpha_field():
    """Eq. 1 weights of one anisotropic Gaussian: alpha at every pixel equals
    o exp(-0.5 d^T cov2d^{-1} d) (linear solve), clamped and thresholded."""
    rng = np.random.default_rng(18)
    sc = _one_scene([[0.1, -0.05, 3.0]], [[0.15, 0.04, 0.01]], [rng.standard_normal(4)], [0.9], [[1, 1, 1]])
    cam = scenes.origin_camera()
    pr = P.project(sc.means, sc.scales, sc.rotations, sc.opacities, sc.sh, 0, cam)
    out = R.render_view(pr, cam)
    vv, uu = np.meshgrid(np.arange(128), np.arange(128), indexing="ij")
    d = np.stack([uu.reshape(-1) + 0.5, vv.reshape(-1) + 0.5], 1) - pr["mean2d"][0].numpy()
    sol = np.linalg.solve(pr["cov2d"][0].numpy(), d.T).T
    a = np.minimum(0.99, 0.9 * np.exp(-0.5 * (d * sol).sum(1)))
    a = np.where(a >= 1 / 255, a, 0)
    np.testing.assert_allclose(out["colour"][:, 0].numpy(), a, atol=1e-12)
    assert (a > 0).sum() > 40
