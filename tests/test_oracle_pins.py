"""Pins of the FP64 oracle to things other than itself: closed forms,
library routines, brute force and invariants (CPU only).

Each test names the passage of CityGaussianV2 (arXiv 2411.00771) or of the
definition it checks, and is built so that a plausible slip in the oracle (a
dropped term, a wrong sign or index, a transposed operand) fails one of them.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy.ndimage import correlate
from scipy.spatial.transform import Rotation
from scipy.special import sph_harm_y

import oracle
from paper_2411_00771_gb300 import synthetic as syn
from tests.scenes import camera, make_scene, pixel_grid

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
ALPHA_MIN = 1.0 / 255.0


def _render(scene, cam, **kw):
    return oracle.render(scene, cam, **kw)


# --------------------------------------------------------------------------
# Geometry: ray-splat intersection and the low-pass max (Sec. 3.1 surfel
# model; Sec. 3.2 antialiasing filter)

def test_fronto_parallel_single_splat_closed_form():
    """A disk facing the camera on the optical axis: rho_obj = |d|^2 z0^2 /
    (f^2 s^2) per axis, rho_scr = 2 |d|^2, alpha = o exp(-min/2)."""
    cam = camera(64, 64, 64.0)
    z0, su, sv, o = 3.0, 0.21, 0.13, 0.8
    sc = make_scene([dict(mu=(0, 0, z0), scale=(su, sv), opacity=o, rgb=(0.9, 0.4, 0.1))])
    r = _render(sc, cam)
    x, y = pixel_grid(cam)
    dx, dy = x - 32.0, y - 32.0
    rho_obj = (dx * z0 / (64.0 * su)) ** 2 + (dy * z0 / (64.0 * sv)) ** 2
    rho_scr = 2.0 * (dx * dx + dy * dy)
    rho = np.minimum(rho_obj, rho_scr)
    alpha = np.minimum(0.99, o * np.exp(-0.5 * rho))
    blended = (rho <= 9.0) & (alpha >= ALPHA_MIN)
    exp_alpha = np.where(blended, alpha, 0.0)
    assert np.abs(r["out"][3] - exp_alpha).max() < 1e-12
    assert np.array_equal(r["count"], blended.astype(np.int32))
    # colour = alpha * rgb, depth = alpha * z0, normal faces the camera
    assert np.abs(r["out"][0] - 0.9 * exp_alpha).max() < 1e-12
    assert np.abs(r["out"][2] - 0.1 * exp_alpha).max() < 1e-12
    assert np.abs(r["out"][4] - z0 * exp_alpha).max() < 1e-12
    assert np.abs(r["out"][5] - exp_alpha / z0).max() < 1e-12
    assert np.abs(r["out"][9] + exp_alpha).max() < 1e-12
    assert np.abs(r["out"][11] - (1 - exp_alpha)).max() < 1e-12
    assert np.abs(r["out"][6] - np.where(blended, z0, 0.0)).max() < 1e-12


def _independent_rho(mu, quat_wxyz, scale, cam, x, y):
    """Ray-plane intersection written independently: t = (n.mu)/(n.r)."""
    R = Rotation.from_quat([quat_wxyz[1], quat_wxyz[2], quat_wxyz[3], quat_wxyz[0]]).as_matrix()
    tu, tv, n = R[:, 0], R[:, 1], R[:, 2]
    r = np.stack([(x - cam["cx"]) / cam["fx"], (y - cam["cy"]) / cam["fy"], np.ones_like(x)], -1)
    t = (n @ mu) / (r @ n)
    P = t[..., None] * r
    u = ((P - mu) @ tu) / scale[0]
    v = ((P - mu) @ tv) / scale[1]
    return u * u + v * v, t


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_tilted_splat_matches_ray_plane_intersection(seed):
    rng = np.random.default_rng(100 + seed)
    cam = camera(48, 40, 50.0, cx=23.3, cy=19.1)
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    mu = np.array([rng.uniform(-0.2, 0.2), rng.uniform(-0.2, 0.2), rng.uniform(2.5, 3.5)])
    scale = np.array([rng.uniform(0.1, 0.3), rng.uniform(0.1, 0.3)])
    o = 0.7
    sc = make_scene([dict(mu=mu, quat=q, scale=scale, opacity=o)])
    r = _render(sc, cam)
    x, y = pixel_grid(cam)
    rho_obj, zobj = _independent_rho(mu, q, scale, cam, x, y)
    c = np.array([cam["fx"] * mu[0] / mu[2] + cam["cx"], cam["fy"] * mu[1] / mu[2] + cam["cy"]])
    rho_scr = 2 * ((x - c[0]) ** 2 + (y - c[1]) ** 2)
    rho = np.minimum(rho_obj, rho_scr)
    z = np.where(rho_obj <= rho_scr, zobj, mu[2])
    alpha = o * np.exp(-0.5 * rho)
    blended = (rho <= 9) & (alpha >= ALPHA_MIN)
    assert blended.sum() > 20
    assert np.abs(r["out"][3] - np.where(blended, alpha, 0)).max() < 1e-10
    assert np.abs(r["out"][4] - np.where(blended, alpha * z, 0)).max() < 1e-9


def test_subpixel_splat_is_screen_filter():
    """s -> 0: only the screen-space filter remains, G = exp(-|x - c|^2)."""
    cam = camera(32, 32, 40.0)
    mu = np.array([0.013, -0.021, 3.0])
    sc = make_scene([dict(mu=mu, scale=(1e-6, 1e-6), opacity=0.9,
                          quat=(0.9, 0.3, -0.2, 0.1))])
    r = _render(sc, cam)
    x, y = pixel_grid(cam)
    c = (40 * mu[0] / mu[2] + 16, 40 * mu[1] / mu[2] + 16)
    d2 = (x - c[0]) ** 2 + (y - c[1]) ** 2
    alpha = 0.9 * np.exp(-d2)
    blended = (2 * d2 <= 9) & (alpha >= ALPHA_MIN)
    assert np.abs(r["out"][3] - np.where(blended, alpha, 0)).max() < 1e-12
    # depth is the centre depth when the screen filter wins
    assert np.abs(r["out"][4] - np.where(blended, alpha * 3.0, 0)).max() < 1e-12


def test_near_plane_cull():
    """A disk whose 3-sigma extent reaches the near plane (0.2) is culled."""
    cam = camera(32, 32, 32.0)
    q = Rotation.from_euler("x", 60, degrees=True).as_quat()  # x y z w
    quat = (q[3], q[0], q[1], q[2])
    ok = make_scene([dict(mu=(0, 0, 1.0), quat=quat, scale=(0.1, 0.2), opacity=0.9)])
    bad = make_scene([dict(mu=(0, 0, 1.0), quat=quat, scale=(0.1, 0.4), opacity=0.9)])
    # min depth of the 3-sigma disk = z - 3 * |(s_u t_u.z, s_v t_v.z)|
    tvz = Rotation.from_quat(q).as_matrix()[2, 1]
    assert 1.0 - 3 * abs(0.2 * tvz) > 0.2 and 1.0 - 3 * abs(0.4 * tvz) < 0.2
    assert oracle.preprocess(ok, cam)["live"][0] == 1
    assert oracle.preprocess(bad, cam)["live"][0] == 0
    assert _render(bad, cam)["count"].sum() == 0


# --------------------------------------------------------------------------
# Compositing (Eq. 1) and the rendered auxiliaries

def _two_splats(z1, z2, o1, o2):
    big = (5.0, 5.0)
    return make_scene([dict(mu=(0, 0, z1), scale=big, opacity=o1, rgb=(1, 0, 0)),
                       dict(mu=(0, 0, z2), scale=big, opacity=o2, rgb=(0, 0, 1))])


def test_two_splats_closed_form_and_order():
    cam = camera(16, 16, 16.0)
    z1, z2, o1, o2 = 2.0, 3.0, 0.3, 0.6
    r = _render(_two_splats(z1, z2, o1, o2), cam)
    # centre pixel: rho is tiny but not zero; read the exact alphas back
    x, y = 8.5, 8.5
    d2 = (x - 8) ** 2 + (y - 8) ** 2
    a1 = o1 * math.exp(-0.5 * d2 * (z1 / (16 * 5.0)) ** 2)
    a2 = o2 * math.exp(-0.5 * d2 * (z2 / (16 * 5.0)) ** 2)
    w1, w2 = a1, a2 * (1 - a1)
    p = (8, 8)
    out = r["out"][:, p[0], p[1]]
    assert abs(out[0] - w1) < 1e-14 and abs(out[2] - w2) < 1e-14
    assert abs(out[11] - (1 - a1) * (1 - a2)) < 1e-14
    assert abs(out[4] - (w1 * z1 + w2 * z2)) < 1e-13
    assert abs(out[10] - 2 * w1 * w2 * abs(z1 - z2)) < 1e-13
    assert abs(r["dexact"][p] - 2 * w1 * w2 * abs(z1 - z2)) < 1e-13
    # both entered with T > 0.5 (1 and 1 - a1 = 0.7): median is the second
    assert out[6] == z2
    # swapping the depths swaps the order
    r2 = _render(_two_splats(z2, z1, o1, o2), cam)
    o2_ = r2["out"][:, p[0], p[1]]
    b2 = o2 * math.exp(-0.5 * d2 * (z1 / 80.0) ** 2)
    b1 = o1 * math.exp(-0.5 * d2 * (z2 / 80.0) ** 2)
    assert abs(o2_[2] - b2) < 1e-14 and abs(o2_[0] - b1 * (1 - b2)) < 1e-14


def test_median_pivot():
    cam = camera(16, 16, 16.0)
    r = _render(_two_splats(2.0, 3.0, 0.6, 0.6), cam)
    assert r["out"][6, 8, 8] == 2.0  # second pair entered with T = 0.4 < 0.5


def test_transmittance_stop_and_alpha_clamp():
    cam = camera(16, 16, 16.0)
    big = (50.0, 50.0)
    sc = make_scene([dict(mu=(0, 0, 2.0 + 0.1 * k), scale=big, opacity=0.8) for k in range(10)])
    r = _render(sc, cam)
    # alpha ~ 0.8 everywhere: T = 0.2^k, stop before T(1-a) < 1e-4 -> 5 pairs
    assert np.all(r["count"] == 5)
    assert np.all(r["out"][11] >= 1e-4)
    sc1 = make_scene([dict(mu=(0, 0, 2.0), scale=big, opacity=1.0)])
    r1 = _render(sc1, cam)
    assert np.all(np.abs(r1["out"][3] - 0.99) < 1e-12)


def test_alpha_cutoff():
    cam = camera(16, 16, 16.0)
    sc = make_scene([dict(mu=(0, 0, 2.0), scale=(50.0, 50.0), opacity=0.999 * ALPHA_MIN)])
    r = _render(sc, cam)
    assert r["count"].sum() == 0
    assert r["out"][11].min() == 1.0 and np.abs(r["out"][:11]).max() == 0


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_brute_force_equals_binned(seed):
    """Binning by the 3-sigma cover loses no pair: every pixel equals the
    brute-force loop over all surfels, bit for bit."""
    scene, cam, _, _ = syn.tiny_scene(seed=seed, n=200, width=32, height=32, fx=32.0,
                                      log_scale_range=(-4.0, -1.0), sh_degree=1,
                                      z_range=(0.5, 4.0))
    rb = _render(scene, cam, mode="brute")
    rt = _render(scene, cam, mode="binned")
    assert np.array_equal(rb["out"], rt["out"])
    assert np.array_equal(rb["count"], rt["count"])


@pytest.mark.parametrize("seed", [0, 1, 2, 3, 4, 5])
def test_brute_force_equals_binned_with_elongated_disks(seed):
    """The per-row tile coverage rule is a conservative cover of the
    footprint: long thin (elongated, tilted) disks, some near the camera."""
    scene, cam, _, _ = syn.tiny_scene(seed=100 + seed, n=150, width=48, height=40, fx=40.0,
                                      log_scale_range=(-3.5, -0.5), z_range=(0.8, 3.0))
    rng = np.random.default_rng(seed)
    k = rng.uniform(size=150) < 0.5
    scene["scale"][k, 0] *= np.exp(rng.uniform(np.log(10), np.log(60), k.sum())).astype(np.float32)
    rb = _render(scene, cam, mode="brute")
    rt = _render(scene, cam, mode="binned")
    assert np.array_equal(rb["out"], rt["out"])
    assert np.array_equal(rb["count"], rt["count"])
    pre = oracle.preprocess(scene, cam)
    r = pre["rect"]
    box = np.where(pre["live"] > 0, (r[:, 2] - r[:, 0]) * (r[:, 3] - r[:, 1]), 0)
    assert np.all(pre["tiles"] <= box) and pre["tiles"].sum() < box.sum()


def test_invariants_on_random_scene():
    scene, cam, _, _ = syn.tiny_scene()
    r = _render(scene, cam)
    out = r["out"]
    assert np.all(out[11] >= 1e-4) and np.all(out[11] <= 1.0)
    assert np.abs(out[3] + out[11] - 1.0).max() < 1e-12
    assert np.all(r["count"] <= r["ncand"]) and np.all(r["count"] >= 0)
    assert np.all(out[3] <= 1.0 + 1e-12)


def test_transparent_scene_gives_background():
    scene, cam, _, _ = syn.tiny_scene(n=300)
    scene = dict(scene)
    scene["opacity"] = np.zeros_like(scene["opacity"])
    r = oracle.render(scene, cam, settings=dict(bg=(0.25, 0.5, 0.75)))
    assert r["count"].sum() == 0
    for c, v in enumerate((0.25, 0.5, 0.75)):
        assert np.all(r["out"][c] == v)


def test_permutation_invariance_of_disjoint_splats():
    """Surfels whose footprints do not overlap: any index order renders the
    same image bit for bit."""
    cam = camera(64, 64, 64.0)
    rng = np.random.default_rng(3)
    surf = []
    for gx in range(4):
        for gy in range(4):
            surf.append(dict(mu=((gx - 1.5) * 0.8, (gy - 1.5) * 0.8, 3.0 + rng.uniform(0, 0.5)),
                             scale=(0.05, 0.07), opacity=rng.uniform(0.3, 0.9),
                             rgb=rng.uniform(0, 1, 3)))
    a = _render(make_scene(surf), cam)
    perm = rng.permutation(len(surf))
    b = _render(make_scene([surf[i] for i in perm]), cam)
    assert np.array_equal(a["out"], b["out"])


def test_distortion_one_pass_equals_pairwise_sum_when_depths_ordered():
    cam = camera(32, 32, 32.0)
    rng = np.random.default_rng(9)
    surf = [dict(mu=(rng.uniform(-0.3, 0.3), rng.uniform(-0.3, 0.3), 2 + 0.2 * k),
                 scale=(0.3, 0.3), opacity=0.5) for k in range(8)]
    r = _render(make_scene(surf), cam)
    assert np.abs(r["out"][10] - r["dexact"]).max() < 1e-12


# --------------------------------------------------------------------------
# Spherical harmonics (colour, Sec. 3.1)

def test_sh_orthonormal_by_quadrature():
    xg, wg = np.polynomial.legendre.leggauss(24)  # cos(theta)
    nphi = 48
    phi = (np.arange(nphi) + 0.5) * 2 * np.pi / nphi
    ct, ph = np.meshgrid(xg, phi, indexing="ij")
    st = np.sqrt(1 - ct ** 2)
    dirs = np.stack([st * np.cos(ph), st * np.sin(ph), ct], -1).reshape(-1, 3)
    w = (wg[:, None] * np.full(nphi, 2 * np.pi / nphi)[None, :]).reshape(-1)
    Y = oracle.sh_basis(dirs)
    G = (Y * w[:, None]).T @ Y
    assert np.abs(G - np.eye(16)).max() < 1e-12


def test_sh_matches_complex_basis_with_condon_shortley_phase():
    rng = np.random.default_rng(0)
    d = rng.normal(size=(50, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    theta = np.arccos(d[:, 2])
    phi = np.arctan2(d[:, 1], d[:, 0])
    Y = oracle.sh_basis(d)
    for l in range(4):
        for m in range(-l, l + 1):
            c = sph_harm_y(l, abs(m), theta, phi)
            if m > 0:
                ref = math.sqrt(2) * c.real
            elif m < 0:
                ref = math.sqrt(2) * c.imag
            else:
                ref = c.real
            assert np.abs(Y[:, l * l + l + m] - ref).max() < 1e-12, (l, m)


def test_view_dependent_colour_of_degree_one_splat():
    cam = camera(32, 32, 32.0)
    cam["t"] = np.array([0.1, -0.2, 0.3])  # camera centre = -t
    sh = np.zeros((4, 3))
    sh[0] = [0.3, -0.2, 0.1]
    sh[1:] = [[0.2, 0.1, -0.3], [0.05, 0.4, 0.2], [-0.25, 0.3, 0.15]]
    mu = np.array([0.05, 0.02, 3.0])
    sc = make_scene([dict(mu=mu, scale=(5.0, 5.0), opacity=0.5, sh=sh)], sh_degree=1)
    pre = oracle.preprocess(sc, cam)
    d = mu - (-cam["t"])
    d /= np.linalg.norm(d)
    theta, phi = math.acos(d[2]), math.atan2(d[1], d[0])
    Y = [sph_harm_y(0, 0, theta, phi).real,
         math.sqrt(2) * sph_harm_y(1, 1, theta, phi).imag,
         sph_harm_y(1, 0, theta, phi).real,
         math.sqrt(2) * sph_harm_y(1, 1, theta, phi).real]
    rgb = np.maximum(0, np.array(Y) @ sh + 0.5)
    assert np.abs(pre["rgb"][0] - rgb).max() < 1e-12


# --------------------------------------------------------------------------
# Losses (Sec. 3.1 L1 + D-SSIM; Sec. 3.2 depth loss on inverse depth)

def _ssim_scipy(x, y):
    g = np.exp(-((np.arange(11) - 5) ** 2) / (2 * 1.5 ** 2))
    g /= g.sum()
    k = np.outer(g, g)
    f = lambda a: correlate(a, k, mode="constant", cval=0.0)
    mx, my = f(x), f(y)
    vx, vy, cxy = f(x * x) - mx * mx, f(y * y) - my * my, f(x * y) - mx * my
    C1, C2 = 0.01 ** 2, 0.03 ** 2
    return (((2 * mx * my + C1) * (2 * cxy + C2)) / ((mx ** 2 + my ** 2 + C1) * (vx + vy + C2))).sum()


def test_ssim_matches_scipy_and_identity():
    rng = np.random.default_rng(0)
    x = rng.uniform(0, 1, (23, 31)); y = rng.uniform(0, 1, (23, 31))
    v, g = oracle.ssim_sum(x, y)
    assert abs(v - _ssim_scipy(x, y)) < 1e-10
    v1, g1 = oracle.ssim_sum(x, x)
    assert abs(v1 - x.size) < 1e-9 and np.abs(g1).max() < 1e-9


def test_ssim_gradient_finite_difference():
    rng = np.random.default_rng(1)
    x = rng.uniform(0, 1, (17, 19)); y = rng.uniform(0, 1, (17, 19))
    _, g = oracle.ssim_sum(x, y)
    for (i, j) in [(0, 0), (3, 4), (8, 9), (16, 18), (10, 0)]:
        h = 1e-6
        xp = x.copy(); xp[i, j] += h
        xm = x.copy(); xm[i, j] -= h
        fd = (oracle.ssim_sum(xp, y, False)[0] - oracle.ssim_sum(xm, y, False)[0]) / (2 * h)
        assert abs(fd - g[i, j]) < 1e-7


def test_loss_closed_forms_and_decomposition():
    H, W = 12, 14
    out = np.zeros((12, H, W))
    out[0:3] = 0.6
    out[5] = 0.3
    tgt = np.full((3, H, W), 0.5)
    tinv = np.full((H, W), 0.2)
    L = oracle.loss(out, tgt, tinv, (0.8, 0.2, 0.5))
    assert abs(L["l1"] - 0.1) < 1e-15 and abs(L["depth"] - 0.1) < 1e-15
    assert abs(L["total"] - (0.8 * 0.1 + 0.2 * (1 - L["ssim"]) + 0.5 * 0.1)) < 1e-15
    adj = L["adj"]
    assert np.allclose(adj[2][0:3], 0.8 / (3 * H * W))
    assert np.allclose(adj[0][0:3], adj[1][0:3] + adj[2][0:3], rtol=0, atol=1e-18)
    assert np.allclose(adj[0][5], 0.5 / (H * W)) and np.all(adj[1][5] == 0)


# --------------------------------------------------------------------------
# Gradients: central finite differences in FP64

def _fd_scene(seed, deg):
    scene, cam, tgt, tinv = syn.tiny_scene(seed=seed, n=60, width=32, height=32, fx=32.0,
                                           sh_degree=deg, xy_range=0.8,
                                           log_scale_range=(-2.5, -1.5))
    for k in ("mu", "quat", "scale", "opacity", "sh"):
        scene[k] = scene[k].astype(np.float64)
    return scene, cam, tgt, tinv


def _fd_check(scene, f, grads, rng, n_per=10, tol=1e-6):
    for key in ("mu", "quat", "scale", "opacity", "sh"):
        flat = scene[key].reshape(-1)
        for i in rng.choice(flat.size, n_per, replace=False):
            h = 1e-6 * max(1.0, abs(flat[i]))
            sp = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in scene.items()}
            sp[key].reshape(-1)[i] += h
            lp = f(sp)
            sp[key].reshape(-1)[i] -= 2 * h
            lm = f(sp)
            fd = (lp - lm) / (2 * h)
            an = grads[key].reshape(-1)[i]
            assert abs(fd - an) <= tol * max(1.0, abs(fd)), (key, i, fd, an)


def test_gradients_of_training_loss_by_finite_differences():
    scene, cam, tgt, tinv = _fd_scene(5, 3)
    w = (0.8, 0.2, 0.5)
    L = oracle.loss(_render(scene, cam)["out"], tgt, tinv, w)
    g = oracle.backward(scene, cam, L["adj"][:1])
    f = lambda sc: oracle.loss(_render(sc, cam)["out"], tgt, tinv, w)["total"]
    _fd_check(scene, f, g, np.random.default_rng(0))


def test_gradients_of_every_output_plane_by_finite_differences():
    """A random linear functional of all 11 differentiable planes (colour,
    alpha, depth, inverse depth, median, normal, distortion)."""
    scene, cam, _, _ = _fd_scene(7, 2)
    rng = np.random.default_rng(1)
    A = rng.normal(size=(1, 11, 32, 32))
    g = oracle.backward(scene, cam, A)
    f = lambda sc, shift=None: float((A[0] * oracle.render(sc, cam, shift=shift)["out"][:11]).sum())
    _fd_check(scene, f, g, rng, tol=1e-6)
    # screen-space translation gradient (densification statistic)
    n = scene["mu"].shape[0]
    for i in rng.choice(n, 15, replace=False):
        for ax in range(2):
            h = 1e-6
            s = np.zeros((n, 2)); s[i, ax] = h
            lp = f(scene, s)
            s[i, ax] = -h
            lm = f(scene, s)
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g["screen"][0, i, ax]) <= 1e-6 * max(1.0, abs(fd))


def test_screen_gradient_sets_follow_their_adjoints():
    """Set k's screen gradient is linear in set k's adjoint: the SSIM-term and
    L1-term sets add up to the colour part of the total set."""
    scene, cam, tgt, tinv = _fd_scene(11, 0)
    L = oracle.loss(_render(scene, cam)["out"], tgt, None, (0.8, 0.2, 0.0))
    g = oracle.backward(scene, cam, L["adj"])
    s = g["screen"]
    assert np.abs(s[0] - (s[1] + s[2])).max() < 1e-14
    assert np.abs(s[0]).max() > 0


# --------------------------------------------------------------------------
# Densification (Sec. 3.2 Eq. 2) and the elongation filter (Sec. 3.2)

def test_dgd_scaling_closed_forms():
    paper = json.load(open(os.path.join(GOLDEN, "paper_constants.json")))
    omega = paper["omega"]["value"]
    # S_tot, S_ssim, S_l1, cnt
    st = np.array([[4.0, 1.0, 3.0, 2.0], [2.0, 1.0, 1.0, 1.0], [9.0, 9.0, 0.0, 0.0]])
    sc = np.ones((3, 2))
    mask, g, k = oracle.densify_select(st, sc, omega=omega, grad_thr=0.0, eta_thr=0.0)
    avg_tot = (2.0 + 2.0) / 2
    avg_ssim = (0.5 + 1.0) / 2
    assert abs(k - max(omega * avg_tot / avg_ssim, 1.0)) < 1e-15
    assert abs(g[0] - k * 0.5) < 1e-15 and abs(g[1] - k * 1.0) < 1e-15 and g[2] == 0
    assert list(mask) == [1, 1, 0]
    # omega * ratio < 1: the SSIM gradient is used unscaled
    st2 = np.array([[1.0, 2.0, 0.0, 1.0]])
    _, g2, k2 = oracle.densify_select(st2, np.ones((1, 2)), omega=omega)
    assert k2 == 1.0 and g2[0] == 2.0


def test_elongation_rate_threshold():
    eps = 1e-6
    sc = np.array([[1.0, 1.0], [0.1 + eps, 1.0], [1.0, 0.1 - eps], [2.0, 0.5]])
    keep = oracle.elongation(sc, eta_thr=0.1)
    assert list(keep) == [1, 1, 0, 1]
    st = np.tile([1.0, 1.0, 1.0, 1.0], (4, 1))
    mask, _, _ = oracle.densify_select(st, sc, grad_thr=0.5, eta_thr=0.1)
    assert list(mask) == [1, 1, 0, 1]


def test_densify_accumulate_counts_visible_views():
    scr = np.zeros((3, 3, 2))
    scr[0, 0] = (3, 4); scr[1, 0] = (0, 1); scr[2, 0] = (6, 8)
    st = oracle.densify_accumulate(scr, np.array([1, 0, 1]))
    st = oracle.densify_accumulate(scr, np.array([1, 0, 1]), st)
    assert np.allclose(st[0], [10.0, 2.0, 20.0, 2.0]) and np.all(st[1] == 0)
    assert np.allclose(st[2], [0, 0, 0, 2.0])


# --------------------------------------------------------------------------
# Trim contribution (Sec. 3.3, Eq. 3) and the percentile prune

def test_contribution_of_single_splat_closed_form():
    """One fronto-parallel disk: T = 1 on every pixel, so C = mean over the
    support {rho <= 9} of alpha^gamma (0 where alpha < 1/255), with rho and
    alpha in closed form (no ray-splat code involved)."""
    cam = camera(64, 64, 64.0)
    z0, su, sv, o = 3.0, 0.21, 0.13, 0.8
    sc = make_scene([dict(mu=(0, 0, z0), scale=(su, sv), opacity=o)])
    x, y = pixel_grid(cam)
    dx, dy = x - 32.0, y - 32.0
    rho = np.minimum((dx * z0 / (64.0 * su)) ** 2 + (dy * z0 / (64.0 * sv)) ** 2, 2.0 * (dx * dx + dy * dy))
    alpha = np.minimum(0.99, o * np.exp(-0.5 * rho))
    support = rho <= 9.0
    used = support & (alpha >= ALPHA_MIN)
    for gamma in (0.5, 0.25, 1.0):
        r = oracle.contribution(sc, cam, gamma=gamma)
        assert r["count"][0] == support.sum()
        expect = np.where(used, alpha ** gamma, 0.0).sum()
        assert abs(r["sum"][0] - expect) < 1e-12 * max(1.0, expect)
        assert abs(r["C"][0] - expect / support.sum()) < 1e-14


def test_contribution_of_occluded_splat_uses_front_transmittance():
    """Two stacked disks: the back one sees T = 1 - alpha_front on every pixel
    (Eq. 3's product over the pairs in front); swapping depths swaps roles."""
    cam = camera(16, 16, 16.0)
    z1, z2, o1, o2 = 2.0, 3.0, 0.3, 0.6
    sc = _two_splats(z1, z2, o1, o2)
    x, y = pixel_grid(cam)
    d2 = (x - 8.0) ** 2 + (y - 8.0) ** 2
    a1 = np.minimum(0.99, o1 * np.exp(-0.5 * np.minimum(d2 * (z1 / 80.0) ** 2, 2 * d2)))
    a2 = np.minimum(0.99, o2 * np.exp(-0.5 * np.minimum(d2 * (z2 / 80.0) ** 2, 2 * d2)))
    r = oracle.contribution(sc, cam, gamma=0.5)
    assert np.all(r["count"] == 256)
    assert abs(r["sum"][0] - np.sqrt(a1).sum()) < 1e-12
    assert abs(r["sum"][1] - np.sqrt(a2 * (1 - a1)).sum()) < 1e-12
    r0 = oracle.contribution(sc, cam, gamma=0.0)  # T in front, blended pairs only
    assert abs(r0["sum"][1] - (1 - a1).sum()) < 1e-12
    # surfel 0 behind surfel 1: the order follows depth, not the index
    b1 = np.minimum(0.99, o1 * np.exp(-0.5 * np.minimum(d2 * (z2 / 80.0) ** 2, 2 * d2)))
    b2 = np.minimum(0.99, o2 * np.exp(-0.5 * np.minimum(d2 * (z1 / 80.0) ** 2, 2 * d2)))
    rs = oracle.contribution(_two_splats(z2, z1, o1, o2), cam, gamma=0.5)
    assert abs(rs["sum"][1] - np.sqrt(b2).sum()) < 1e-12
    assert abs(rs["sum"][0] - np.sqrt(b1 * (1 - b2)).sum()) < 1e-12


@pytest.mark.parametrize("gamma", [0.5, 0.3])
def test_contribution_brute_force_with_closed_form_geometry(gamma):
    """Fronto-parallel disks anywhere in view have a closed-form rho at every
    pixel (the ray meets the plane z = z_i at (p - c) z_i / f), so Eq. 3 can be
    evaluated by brute force with no ray-splat code: support rho <= 9, order by
    the FP32 centre depth then index, alpha cutoff, the stop, T in front."""
    W = H = 24
    f = 24.0
    cam = camera(W, H, f)
    rng = np.random.default_rng(7)
    surf = []
    for i in range(14):
        z = rng.uniform(2.0, 4.0)
        surf.append(dict(mu=(rng.uniform(-0.8, 0.8), rng.uniform(-0.8, 0.8), z),
                         scale=(rng.uniform(0.05, 0.6), rng.uniform(0.05, 0.6)),
                         opacity=float(rng.choice([0.02, 0.5, 0.95]))))
    r = oracle.contribution(make_scene(surf), cam, gamma=gamma)
    x, y = pixel_grid(cam)
    z32 = np.array([np.float32(s_["mu"][2]) for s_ in surf], np.float64)
    order = sorted(range(len(surf)), key=lambda i: (z32[i], i))
    rho = []
    for s_ in surf:
        mx, my, mz = s_["mu"]
        cx, cy = f * mx / mz + W / 2, f * my / mz + H / 2
        dx, dy = x - cx, y - cy
        ro = (dx * mz / (f * s_["scale"][0])) ** 2 + (dy * mz / (f * s_["scale"][1])) ** 2
        rho.append(np.minimum(ro, 2.0 * (dx * dx + dy * dy)))
    exp_sum = np.zeros(len(surf))
    exp_cnt = np.zeros(len(surf), np.int64)
    for j in range(H):
        for i in range(W):
            T, stopped = 1.0, False
            for n in order:
                rr = rho[n][j, i]
                if not rr <= 9.0:
                    continue
                exp_cnt[n] += 1
                a = min(0.99, surf[n]["opacity"] * math.exp(-0.5 * rr))
                if stopped or a < ALPHA_MIN:
                    continue
                if T * (1 - a) < 1e-4:
                    stopped = True
                    continue
                exp_sum[n] += a ** gamma * T ** (1 - gamma)
                T *= 1 - a
    assert np.array_equal(r["count"], exp_cnt)
    assert np.abs(r["sum"] - exp_sum).max() < 1e-11
    # the low-opacity disks have support pixels below the alpha cutoff
    low = [n for n in range(len(surf)) if surf[n]["opacity"] == 0.02]
    assert any(exp_cnt[n] > 0 for n in low)


def test_contribution_counts_the_support_and_stops_with_the_pixel():
    """Behind a stack that stops the pixels (T below 1e-4), later disks keep
    their support pixels in |P| but add nothing; never-seen disks get 0."""
    cam = camera(16, 16, 16.0)
    big = (50.0, 50.0)
    surf = [dict(mu=(0, 0, 2.0 + 0.1 * k), scale=big, opacity=0.8) for k in range(8)]
    surf.append(dict(mu=(100.0, 0, 2.0), scale=(0.1, 0.1), opacity=0.8))  # off screen
    r = oracle.contribution(make_scene(surf), cam, gamma=0.5)
    assert np.all(r["count"][:8] == 256) and r["count"][8] == 0 and r["C"][8] == 0
    assert np.all(r["sum"][:5] > 0) and np.all(r["sum"][5:] == 0)  # 5 pairs blended per pixel


def test_contribution_brute_force_equals_binned():
    scene, cam, _, _ = syn.tiny_scene(seed=4, n=200, width=32, height=32, fx=32.0,
                                      log_scale_range=(-4.0, -1.0), sh_degree=1, z_range=(0.5, 4.0))
    rb = oracle.contribution(scene, cam, mode=0)
    rt = oracle.contribution(scene, cam, mode=1)
    assert np.array_equal(rb["count"], rt["count"])
    assert np.abs(rb["sum"] - rt["sum"]).max() < 1e-12


def test_prune_bound_percentile():
    """Sec. 3.3: remove the surfels at or below the ratio-percentile bound,
    ties included (all never-observed zeros go, whatever the ratio)."""
    c = np.array([0.5, 0.0, 0.2, 0.0, 0.9, 0.2, 0.7, 0.0, 0.3, 0.1])
    bound, keep = oracle.prune_bound(c, 0.1)  # k = 1 -> bound = 0: all three zeros removed
    assert bound == 0.0 and keep.sum() == 7
    bound, keep = oracle.prune_bound(c, 0.5)  # k = 5: sorted 0,0,0,.1,.2,.2 -> bound .2
    assert bound == 0.2 and np.array_equal(keep, c > 0.2) and keep.sum() == 4
    bound, keep = oracle.prune_bound(c, 0.0)
    assert bound is None and keep.all()
    bound, keep = oracle.prune_bound(c, 1.0)
    assert bound == 0.9 and not keep.any()


# --------------------------------------------------------------------------
# Visible frequency of points (Sec. 4, crop volume estimation)

def test_visibility_on_axis_behind_and_near_plane():
    cam = camera(64, 48, 60.0)
    pts = np.array([[0.0, 0.0, 5.0], [0.0, 0.0, -5.0], [0.0, 0.0, 0.19], [0.0, 0.0, 0.21]])
    c, f = oracle.visibility_count(pts, 0.05, [cam, cam, cam])
    assert list(c) == [3, 0, 0, 3] and not f.any()


def test_visibility_image_edge_closed_form():
    """Point at (x, 0, z) seen by an identity camera: the projected covariance
    is diagonal (sigma^2 f^2 (1/z^2 + x^2/z^4) + lp, sigma^2 f^2/z^2 + lp), the
    larger entry is the x one, and the point drops out when c - 3 sqrt(S_xx)
    passes W.  Bisection on that closed form finds the edge; points just
    inside and outside it flip."""
    W, H, f, z, s, lp = 64, 48, 60.0, 4.0, 0.05, 0.3
    cam = camera(W, H, f)

    def left_edge(x):
        sxx = s * s * f * f * (1 / z ** 2 + x * x / z ** 4) + lp
        return f * x / z + W / 2 - 3 * math.sqrt(sxx) - W

    a, b = 0.0, 10.0
    for _ in range(200):
        m = 0.5 * (a + b)
        a, b = (m, b) if left_edge(m) < 0 else (a, m)
    xe = 0.5 * (a + b)
    pts = np.array([[xe * (1 - 1e-4), 0, z], [xe * (1 + 1e-4), 0, z]])
    c, fl = oracle.visibility_count(pts, s, [cam], lowpass=lp)
    assert list(c) == [1, 0] and not fl.any()


def test_visibility_matches_numerical_jacobian_and_eigensolver():
    """Random points and views: the 3-sigma half-width from numpy's
    eigensolver on sigma^2 J J^T + lp I, with J by central differences of the
    projection, decides the same visibility away from the thresholds."""
    rng = np.random.default_rng(12)
    pts = rng.uniform([-30, -30, -2], [30, 30, 25], (400, 3))
    cams = [syn.orbit_camera(rng, 96, 72, radius=60.0, altitude=40.0) for _ in range(12)]
    s, lp = 0.8, 0.3
    c, fl = oracle.visibility_count(pts, s, cams, lowpass=lp)
    exp = np.zeros(len(pts), np.int64)
    margin_ok = np.ones(len(pts), bool)
    for cam in cams:
        R, t = np.asarray(cam["R"]), np.asarray(cam["t"])

        def proj(q):
            p = R @ q + t
            return np.array([cam["fx"] * p[0] / p[2] + cam["cx"], cam["fy"] * p[1] / p[2] + cam["cy"]])

        for j, q in enumerate(pts):
            p = R @ q + t
            if p[2] <= 0.2:
                continue
            Jw = np.stack([(proj(q + e) - proj(q - e)) / 2e-4 for e in np.eye(3) * 1e-4], axis=1)  # d pix / d world
            S = s * s * Jw @ Jw.T + lp * np.eye(2)
            r = 3 * math.sqrt(np.linalg.eigvalsh(S).max())
            cx, cy = proj(q)
            m = np.array([cx + r, cam["width"] - (cx - r), cy + r, cam["height"] - (cy - r)])
            if np.abs(m).min() < 1e-4 * (abs(cx) + abs(cy) + r + 200):
                margin_ok[j] = False
            exp[j] += int(np.all(m > 0))
    assert margin_ok.mean() > 0.95
    assert np.array_equal(c[margin_ok], exp[margin_ok]) and c.sum() > 100 and (c < len(cams)).any()


def test_visible_height_range():
    pts = np.array([[0, 0, 1.0], [0, 0, 5.0], [0, 0, 3.0], [0, 0, 9.0]])
    keep, (lo, hi) = oracle.visible_height_range(pts, [5, 1, 3, 0], 2)
    assert list(keep) == [True, False, True, False] and (lo, hi) == (1.0, 3.0)


# --------------------------------------------------------------------------
# Depth-normal consistency (2DGS smoothness term, weight of Sec. 5.1)

def _planar_out(H, W, cam, plane_n, plane_d, alpha=0.7):
    """Render planes of an opaque plane n.X = d seen by cam: median depth from
    the ray-plane intersection, rendered normal = alpha * (camera-facing n)."""
    xs = (np.arange(W) + 0.5 - cam["cx"]) / cam["fx"]
    ys = (np.arange(H) + 0.5 - cam["cy"]) / cam["fy"]
    ray = np.stack([np.broadcast_to(xs[None], (H, W)), np.broadcast_to(ys[:, None], (H, W)), np.ones((H, W))])
    t = plane_d / np.einsum("k,kij->ij", plane_n, ray)
    out = np.zeros((12, H, W))
    out[3] = alpha
    out[6] = t
    nf = -np.asarray(plane_n) if plane_d > 0 else np.asarray(plane_n)  # towards the camera
    out[7:10] = alpha * nf[:, None, None]
    return out, nf


def test_normal_loss_vanishes_on_matching_planes():
    cam = camera(24, 18, 20.0)
    for n in ([0, 0, 1.0], [0.3, -0.2, 0.93]):
        nv = np.asarray(n) / np.linalg.norm(n)
        out, nf = _planar_out(18, 24, cam, nv, 4.0)
        L, adj = oracle.normal_loss(out, cam, weight=1.0)
        assert abs(L) < 1e-12
        # the depth normal is the plane's normal wherever it is defined
        assert np.allclose(adj[7:10, 1:-1, 1:-1], -nf[:, None, None] / (18 * 24))


def test_normal_loss_closed_form_for_misaligned_normals():
    """Rendered normals tilted by theta from the true plane normal: per
    interior pixel A - A cos(theta)."""
    cam = camera(20, 16, 18.0)
    out, nf = _planar_out(16, 20, cam, np.array([0, 0, 1.0]), 5.0, alpha=0.8)
    th = 0.3
    out[7:10] = 0.8 * np.array([math.sin(th), 0.0, -math.cos(th)])[:, None, None]
    L, _ = oracle.normal_loss(out, cam, weight=2.0)
    interior = 14 * 18
    assert abs(L - 2.0 * interior * 0.8 * (1 - math.cos(th)) / (16 * 20)) < 1e-12


def test_normal_loss_gradient_by_finite_differences():
    cam = camera(12, 10, 11.0)
    rng = np.random.default_rng(5)
    out, _ = _planar_out(10, 12, cam, np.array([0.2, 0.1, 0.97]), 3.0)
    out[6] += rng.normal(0, 0.05, out[6].shape)
    out[3] = rng.uniform(0.3, 1.0, out[3].shape)
    out[7:10] += rng.normal(0, 0.2, out[7:10].shape)
    L0, adj = oracle.normal_loss(out, cam, weight=0.5)
    for plane in (3, 6, 7, 8, 9):
        for _ in range(6):
            j, i = rng.integers(10), rng.integers(12)
            h = 1e-6
            o1, o2 = out.copy(), out.copy()
            o1[plane, j, i] += h
            o2[plane, j, i] -= h
            fd = (oracle.normal_loss(o1, cam, 0.5)[0] - oracle.normal_loss(o2, cam, 0.5)[0]) / (2 * h)
            assert abs(fd - adj[plane, j, i]) < 1e-7 * max(1.0, abs(fd)), (plane, j, i, fd, adj[plane, j, i])


# --------------------------------------------------------------------------
# Training loop: Adam, densification

def test_adam_matches_torch_optim():
    import torch
    rng = np.random.default_rng(8)
    p0 = rng.normal(size=50)
    grads = [rng.normal(size=50) for _ in range(4)]
    t = torch.tensor(p0, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([t], lr=1e-2, betas=(0.9, 0.999), eps=1e-15)
    p, m, v = p0.copy(), np.zeros(50), np.zeros(50)
    for k, g in enumerate(grads, start=1):
        t.grad = torch.tensor(g)
        opt.step()
        p, m, v = oracle.adam_step(p, g, m, v, 1e-2, k)
    assert np.abs(p - t.detach().numpy()).max() < 1e-14


def test_densify_plan_and_apply_hand_checked():
    scene = dict(mu=np.array([[0, 0, 1.0], [1, 0, 1], [2, 0, 1], [3, 0, 1]]),
                 quat=np.array([[1.0, 0, 0, 0]] * 4),
                 scale=np.array([[0.1, 0.2], [0.5, 0.3], [0.1, 0.1], [0.1, 0.1]]),
                 opacity=np.array([0.5, 0.5, 0.001, 0.5]), sh=np.arange(12.0).reshape(4, 1, 3), sh_degree=0)
    sel = np.array([1, 1, 0, 0])
    action, offset, n_out = oracle.densify_plan(sel, scene["scale"], scene["opacity"], 0.3, 0.005)
    assert list(action) == [2, 3, 0, 1] and list(offset) == [0, 2, 4, 4] and n_out == 5
    xi = np.zeros((4, 2, 2))
    xi[1] = [[1.0, 0.0], [0.0, -2.0]]
    out, src, fresh = oracle.densify_apply(scene, action, xi)
    assert list(src) == [0, 0, 1, 1, 3] and list(fresh) == [0, 1, 1, 1, 0]
    # identity rotation: t_u = x, t_v = y; child 0 moves by s_u along x, child 1 by -2 s_v along y
    assert np.allclose(out["mu"][2], [1.5, 0, 1]) and np.allclose(out["mu"][3], [1, -0.6, 1])
    assert np.allclose(out["scale"][2], [0.5 / 1.6, 0.3 / 1.6]) and np.allclose(out["scale"][0], [0.1, 0.2])
    assert np.array_equal(out["sh"][4], scene["sh"][3])


# ---------------------------------------------------------------------------
# Contribution-based vector quantisation of SH (Sec. 3.3; Appendix C)

def _vq_data(m, C, seed, K=None):
    rng = np.random.default_rng(seed)
    x = rng.normal(0, 0.3, (m, C))
    x[:, :3] += rng.uniform(-1, 1.5, (m, 1))      # DC-like offset shared by the colour channels
    x[rng.random((m, C)) < 0.01] = 3e-6            # binary16 subnormals
    x16 = oracle.half(x)
    if K is None:
        return x16
    return x16, oracle.half(rng.normal(0, 0.3, (K, C)))


def test_vq_assign_is_scipy_nearest_code():
    from scipy.cluster.vq import vq
    x16, c16 = _vq_data(3000, 48, 1, K=256)
    a, flag, d = oracle.vq_assign(x16, c16)
    ref, rdist = vq(x16.astype(np.float64), c16.astype(np.float64))
    assert flag.mean() < 0.01
    assert np.array_equal(a[~flag], ref[~flag])
    assert np.allclose(np.sqrt(d), rdist, rtol=1e-9, atol=1e-9)


def test_vq_update_is_the_rounded_cluster_mean():
    x16, c16 = _vq_data(5000, 27, 2, K=64)
    rng = np.random.default_rng(3)
    a = rng.integers(0, 60, 5000)                  # entries 60..63 stay empty
    new, cnt = oracle.vq_update(x16, a, c16)
    for j in range(64):
        rows = x16[a == j].astype(np.float64)
        expect = c16[j] if rows.shape[0] == 0 else np.float16(rows.mean(0))
        assert np.array_equal(new[j], expect), j
        assert cnt[j] == rows.shape[0]


def test_vq_kmeans_recovers_separated_blobs():
    rng = np.random.default_rng(4)
    centres = rng.uniform(-4, 4, (8, 12)) + 20 * np.eye(8, 12)
    x16 = oracle.half(np.repeat(centres, 100, axis=0) + rng.normal(0, 0.01, (800, 12)))
    u = (np.arange(8) * 100 + 50) / 800.0          # one seed inside each blob
    c, a, obj, flags = oracle.vq_kmeans(x16, u, iters=2)
    assert np.array_equal(a, np.repeat(np.arange(8), 100))
    for b in range(8):
        assert np.array_equal(c[b], np.float16(x16[b * 100:(b + 1) * 100].astype(np.float64).mean(0)))
    assert not any(f.any() for f in flags)


def test_vq_kmeans_objective_does_not_increase():
    """Lloyd's steps never raise the sum of squared distances; rounding the
    centroids to binary16 may add at most count * C * (half an ulp)^2 per entry."""
    x16 = _vq_data(2000, 48, 5)
    u = np.random.default_rng(6).random(64, dtype=np.float32)
    c, a, obj, _ = oracle.vq_kmeans(x16, u, iters=8)
    slack = 2000 * 48 * (2.0 ** -11 * 4) ** 2
    assert np.all(np.diff(obj) <= slack), np.diff(obj)
    assert obj[-1] < 0.8 * obj[0]


def test_vq_init_rows():
    m = 1000
    u = np.array([0.0, 0.5, np.nextafter(np.float32(1), np.float32(0))], np.float32)
    assert list(oracle.vq_init_rows(u, m)) == [0, 500, 999]


def test_vq_compress_round_trip():
    scene, _, _, _ = syn.tiny_scene(seed=8, n=500, sh_degree=3)
    rng = np.random.default_rng(9)
    contrib = rng.exponential(0.1, 500).astype(np.float32)
    quant = oracle.vq_quantized(contrib, 0.4)
    assert quant.sum() == math.ceil(0.4 * 500)
    assert np.all(contrib[quant].max() < contrib[~quant].min())
    x16 = oracle.vq_vectors(scene["sh"], quant)
    c, a, _, _ = oracle.vq_kmeans(x16, rng.random(32, dtype=np.float32), iters=3)
    comp = oracle.vq_compress(scene, quant, c, a)
    back = oracle.vq_decompress(comp)
    sh = np.asarray(scene["sh"]).reshape(500, -1)
    got = back["sh"].reshape(500, -1)
    assert np.array_equal(got[~quant], np.float16(sh[~quant]).astype(np.float32))
    assert np.array_equal(got[quant], c[a].astype(np.float32))
    for k in ("quat", "scale", "opacity"):
        v = np.asarray(scene[k], np.float32).reshape(back[k].shape)
        assert np.all(np.abs(back[k] - v) <= np.abs(v) * 2.0 ** -11 + 2.0 ** -25), k
    assert np.array_equal(back["mu"], np.asarray(scene["mu"], np.float32))
    assert comp["sh_table"].shape[0] == 32 + (~quant).sum()


def test_vq_paper_constants_fit_the_layout():
    """Appendix C's codebook size fits the 32-bit row index with room for the
    kept rows, and its ratio selects ceil(0.4 N) surfels when contributions
    are distinct."""
    paper = json.load(open(os.path.join(GOLDEN, "paper_constants.json")))
    K, ratio = paper["vq_codebook_size"]["value"], paper["vq_ratio"]["value"]
    assert K == 8192 and ratio == 0.4
    c = np.random.default_rng(10).permutation(10_000).astype(np.float32)
    assert oracle.vq_quantized(c, ratio).sum() == math.ceil(ratio * 10_000)
