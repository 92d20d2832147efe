"""Seeded synthetic inputs: surfel scenes, cameras and target images.

This module holds no rasterizer arithmetic; it only draws inputs.  Both the
CUDA path and the FP64 oracle consume what it produces.  The paper's data
(GauU-Scene and MatrixCity aerial captures, Sec. 5.1) are not available, so
these generators stand in for them with the same shapes: aerial views whose
longer side is 1600 px, city blocks of a few hundred metres, millions of
surfels, SH degree 2-3.

Conventions shared with the library's C interface:
  * surfel arrays are FP32: mu [N,3], quat [N,4] as (w, x, y, z), scale [N,2]
    (activated, > 0), opacity [N] (activated, in (0,1)), sh [N, (d+1)^2, 3];
  * a camera is world->camera R (3x3, row-major), t (3), fx, fy, cx, cy,
    width, height, in float64; the camera looks down +z, x right, y down.
"""
from __future__ import annotations

import math

import numpy as np

SEED_BASE = 20241101


def _sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def _quat_mul(a, b):
    aw, ax, ay, az = a[..., 0], a[..., 1], a[..., 2], a[..., 3]
    bw, bx, by, bz = b[..., 0], b[..., 1], b[..., 2], b[..., 3]
    return np.stack([aw * bw - ax * bx - ay * by - az * bz,
                     aw * bx + ax * bw + ay * bz - az * by,
                     aw * by - ax * bz + ay * bw + az * bx,
                     aw * bz + ax * by - ay * bx + az * bw], -1)


def _quat_axis_angle(axis, angle):
    axis = axis / np.maximum(np.linalg.norm(axis, axis=-1, keepdims=True), 1e-30)
    h = 0.5 * angle[..., None]
    return np.concatenate([np.cos(h), np.sin(h) * axis], -1)


def quat_from_normal(normal, spin):
    """Unit quaternions whose rotation takes the local z axis to ``normal``,
    preceded by a rotation ``spin`` about local z (in-plane orientation)."""
    n = normal / np.linalg.norm(normal, axis=-1, keepdims=True)
    z = np.array([0.0, 0.0, 1.0])
    axis = np.cross(np.broadcast_to(z, n.shape), n)
    s = np.linalg.norm(axis, axis=-1)
    ang = np.arctan2(s, n[:, 2])
    # normals parallel to z: rotate about x by 0 or pi
    fallback = np.broadcast_to(np.array([1.0, 0.0, 0.0]), n.shape)
    axis = np.where((s < 1e-12)[:, None], fallback, axis)
    qa = _quat_axis_angle(axis, ang)
    qs = _quat_axis_angle(np.broadcast_to(z, n.shape).copy(), spin)
    return _quat_mul(qa, qs)


def look_at(pos, target, width, height, fx, fy=None, cx=None, cy=None):
    """Pinhole camera at ``pos`` looking at ``target`` with world z up."""
    pos = np.asarray(pos, np.float64)
    f = np.asarray(target, np.float64) - pos
    f /= np.linalg.norm(f)
    up = np.array([0.0, 0.0, 1.0])
    r = np.cross(f, up)
    r /= np.linalg.norm(r)
    d = np.cross(f, r)
    R = np.stack([r, d, f])
    t = -R @ pos
    return dict(R=R, t=t, fx=float(fx), fy=float(fy if fy is not None else fx),
                cx=float(width / 2 if cx is None else cx),
                cy=float(height / 2 if cy is None else cy), width=int(width), height=int(height))


def identity_camera(width, height, fx, fy=None, cx=None, cy=None):
    return dict(R=np.eye(3), t=np.zeros(3), fx=float(fx), fy=float(fy if fy is not None else fx),
                cx=float(width / 2 if cx is None else cx), cy=float(height / 2 if cy is None else cy),
                width=int(width), height=int(height))


# --------------------------------------------------------------------------
# Small random scene: 2,000 surfels in front of a 128x128 pinhole camera.

def tiny_scene(seed: int = SEED_BASE + 1, n: int = 2000, width: int = 128, height: int = 128,
               fx: float = 128.0, sh_degree: int = 0, xy_range: float = 1.0,
               z_range=(2.0, 4.0), log_scale_range=(-4.0, -2.0)):
    """Centres x, y ~ U[-r, r], z ~ U[z0, z1]; log-scales ~ U[a, b] on two
    axes; rotations uniform on S^3 (normalised 4-D Gaussian); opacity =
    sigmoid(N(0,1)); SH DC coefficient ~ U(-sqrt(pi), sqrt(pi)) per channel
    (a DC colour uniform in (0, 1)); higher orders ~ N(0, 0.05^2).
    Target colour ~ U(0, 1); target inverse depth ~ U(0.25, 0.5)."""
    rng = np.random.default_rng(seed)
    mu = np.empty((n, 3))
    mu[:, 0] = rng.uniform(-xy_range, xy_range, n)
    mu[:, 1] = rng.uniform(-xy_range, xy_range, n)
    mu[:, 2] = rng.uniform(z_range[0], z_range[1], n)
    scale = np.exp(rng.uniform(log_scale_range[0], log_scale_range[1], (n, 2)))
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    opacity = _sigmoid(rng.normal(size=n))
    K = (sh_degree + 1) ** 2
    sh = np.zeros((n, K, 3))
    sh[:, 0, :] = rng.uniform(-math.sqrt(math.pi), math.sqrt(math.pi), (n, 3))
    if K > 1:
        sh[:, 1:, :] = rng.normal(0.0, 0.05, (n, K - 1, 3))
    scene = dict(mu=mu.astype(np.float32), quat=q.astype(np.float32),
                 scale=scale.astype(np.float32), opacity=opacity.astype(np.float32),
                 sh=sh.astype(np.float32), sh_degree=sh_degree)
    cam = identity_camera(width, height, fx)
    target = rng.uniform(0.0, 1.0, (3, height, width)).astype(np.float32)
    tinv = rng.uniform(0.25, 0.5, (height, width)).astype(np.float32)
    return scene, cam, target, tinv


# --------------------------------------------------------------------------
# Aerial city block: ground plane plus box buildings, surfels on surfaces.

def _city_boxes(rng, n_boxes, half, fp_range, h_range, max_tries=200000):
    boxes = []
    tries = 0
    while len(boxes) < n_boxes and tries < max_tries:
        tries += 1
        wx, wy = rng.uniform(fp_range[0], fp_range[1], 2)
        cx = rng.uniform(-half + wx / 2, half - wx / 2)
        cy = rng.uniform(-half + wy / 2, half - wy / 2)
        b = (cx - wx / 2, cx + wx / 2, cy - wy / 2, cy + wy / 2)
        ok = True
        for o in boxes:
            if b[0] < o[1] + 2 and b[1] > o[0] - 2 and b[2] < o[3] + 2 and b[3] > o[2] - 2:
                ok = False
                break
        if ok:
            boxes.append(b + (rng.uniform(h_range[0], h_range[1]),))
    return np.array(boxes, np.float64)  # x0 x1 y0 y1 h


def city_scene(seed: int = SEED_BASE + 2, n: int = 1_000_000, sh_degree: int = 3,
               extent=(500.0, 500.0), n_boxes: int = 200, fp_range=(10.0, 40.0),
               h_range=(10.0, 60.0), elongated_frac: float = 0.05):
    """Surfels sampled by area over a ground rectangle (minus building
    footprints), building roofs and walls.  Local z of each surfel is the
    surface normal, in-plane orientation uniform.  log-scales ~
    N(ln(0.5 * spacing), 0.4^2) with spacing = sqrt(area / N); a fraction of
    surfels is elongated (one axis times log-U[10, 50]).  Opacity =
    sigmoid(N(1, 1.5)).  SH: DC from a per-surface albedo plus N(0, 0.05^2)
    noise, higher orders N(0, 0.05^2).  Returns (scene, boxes, albedo info)."""
    rng = np.random.default_rng(seed)
    ex, ey = extent
    half = 0.5 * max(ex, ey)
    boxes = _city_boxes(rng, n_boxes, half, fp_range, h_range)
    nb = len(boxes)
    # surfaces: 0 ground, then per box: roof, 4 walls
    fp_area = (boxes[:, 1] - boxes[:, 0]) * (boxes[:, 3] - boxes[:, 2])
    ground_area = ex * ey - fp_area.sum()
    wall_x = (boxes[:, 1] - boxes[:, 0]) * boxes[:, 4]
    wall_y = (boxes[:, 3] - boxes[:, 2]) * boxes[:, 4]
    areas = np.concatenate([[ground_area], fp_area, wall_y, wall_y, wall_x, wall_x])
    total = areas.sum()
    spacing = math.sqrt(total / n)
    counts = rng.multinomial(n, areas / total)
    albedo_ground = np.array([0.45, 0.47, 0.42])
    box_albedo = rng.uniform(0.2, 0.85, (nb, 3))
    mus, nrms, cols = [], [], []
    # ground (rejection against footprints): a 0.5 m grid of box ids finds
    # the one box a point can fall in (boxes keep 2 m gaps), then the exact
    # test against that box
    cell = 0.5
    gx, gy = int(math.ceil(ex / cell)) + 1, int(math.ceil(ey / cell)) + 1
    grid = np.full((gx, gy), -1, np.int32)
    for bi, b in enumerate(boxes):
        i0, i1 = int((b[0] + ex / 2) // cell), int((b[1] + ex / 2) // cell)
        j0, j1 = int((b[2] + ey / 2) // cell), int((b[3] + ey / 2) // cell)
        grid[max(i0, 0):min(i1 + 1, gx), max(j0, 0):min(j1 + 1, gy)] = bi
    k = counts[0]
    pts = np.empty((0, 2))
    while pts.shape[0] < k:
        c = rng.uniform([-ex / 2, -ey / 2], [ex / 2, ey / 2], (int(1.3 * (k - pts.shape[0])) + 16, 2))
        ci = np.clip(((c[:, 0] + ex / 2) // cell).astype(np.int64), 0, gx - 1)
        cj = np.clip(((c[:, 1] + ey / 2) // cell).astype(np.int64), 0, gy - 1)
        bid = grid[ci, cj]
        inside = np.zeros(c.shape[0], bool)
        m = bid >= 0
        if m.any():
            b = boxes[bid[m]]
            inside[m] = (c[m, 0] > b[:, 0]) & (c[m, 0] < b[:, 1]) & (c[m, 1] > b[:, 2]) & (c[m, 1] < b[:, 3])
        pts = np.concatenate([pts, c[~inside]])
    pts = pts[:k]
    mus.append(np.column_stack([pts, np.zeros(k)]))
    nrms.append(np.tile([0.0, 0.0, 1.0], (k, 1)))
    cols.append(np.tile(albedo_ground, (k, 1)))
    off = 1
    for i, b in enumerate(boxes):  # roofs
        k = counts[off + i]
        x = rng.uniform(b[0], b[1], k); y = rng.uniform(b[2], b[3], k)
        mus.append(np.column_stack([x, y, np.full(k, b[4])]))
        nrms.append(np.tile([0.0, 0.0, 1.0], (k, 1)))
        cols.append(np.tile(box_albedo[i] * 0.8, (k, 1)))
    off += nb
    for side, (nv, axis) in enumerate([((1, 0, 0), 0), ((-1, 0, 0), 0), ((0, 1, 0), 1),
                                       ((0, -1, 0), 1)]):
        for i, b in enumerate(boxes):
            k = counts[off + i]
            z = rng.uniform(0.0, b[4], k)
            if axis == 0:
                x = np.full(k, b[1] if nv[0] > 0 else b[0]); y = rng.uniform(b[2], b[3], k)
            else:
                y = np.full(k, b[3] if nv[1] > 0 else b[2]); x = rng.uniform(b[0], b[1], k)
            mus.append(np.column_stack([x, y, z]))
            nrms.append(np.tile(np.array(nv, np.float64), (k, 1)))
            cols.append(np.tile(box_albedo[i], (k, 1)))
        off += nb
    mu = np.concatenate(mus)
    nrm = np.concatenate(nrms)
    col = np.concatenate(cols)
    perm = rng.permutation(mu.shape[0])
    mu, nrm, col = mu[perm], nrm[perm], col[perm]
    quat = quat_from_normal(nrm, rng.uniform(0, 2 * math.pi, n))
    log_s = rng.normal(math.log(0.5 * spacing), 0.4, (n, 2))
    elong = rng.uniform(size=n) < elongated_frac
    ax = rng.integers(0, 2, n)
    factor = np.exp(rng.uniform(math.log(10.0), math.log(50.0), n))
    log_s[elong, ax[elong]] += np.log(factor[elong])
    scale = np.exp(log_s)
    opacity = _sigmoid(rng.normal(1.0, 1.5, n))
    K = (sh_degree + 1) ** 2
    sh = np.zeros((n, K, 3))
    # DC coefficient of a colour c is (c - 0.5) * 2 sqrt(pi) (the degree-0
    # basis function is 1 / (2 sqrt(pi))); a plain input-side conversion.
    sh[:, 0, :] = (np.clip(col + rng.normal(0, 0.05, (n, 3)), 0, 1) - 0.5) * 2.0 * math.sqrt(math.pi)
    if K > 1:
        sh[:, 1:, :] = rng.normal(0.0, 0.05, (n, K - 1, 3))
    scene = dict(mu=mu.astype(np.float32), quat=quat.astype(np.float32),
                 scale=scale.astype(np.float32), opacity=opacity.astype(np.float32),
                 sh=sh.astype(np.float32), sh_degree=sh_degree)
    return scene, dict(boxes=boxes, box_albedo=box_albedo, ground_albedo=albedo_ground,
                       extent=extent)


def aerial_camera(width=1600, height=900, hfov_deg=60.0, altitude=150.0, pitch_deg=45.0,
                  azimuth_deg=-90.0, target=(0.0, 0.0, 0.0)):
    """Camera pitched ``pitch_deg`` down from ``altitude`` metres, aimed at
    ``target``; fx from the horizontal field of view (60 deg -> 1385.6 at
    1600 px)."""
    fx = 0.5 * width / math.tan(math.radians(hfov_deg) / 2)
    horiz = altitude / math.tan(math.radians(pitch_deg))
    az = math.radians(azimuth_deg)
    pos = (target[0] + horiz * math.cos(az), target[1] + horiz * math.sin(az), target[2] + altitude)
    return look_at(pos, target, width, height, fx)


def orbit_camera(rng, width=1600, height=900, radius=250.0, altitude=200.0, hfov_deg=60.0):
    az = rng.uniform(0, 2 * math.pi)
    fx = 0.5 * width / math.tan(math.radians(hfov_deg) / 2)
    pos = (radius * math.cos(az), radius * math.sin(az), altitude)
    return look_at(pos, (0.0, 0.0, 0.0), width, height, fx)


def city_targets(info, cam, seed: int = SEED_BASE + 3):
    """Target colour and inverse depth by an analytic ray cast of the city
    (ground plane plus boxes): colour = albedo of the first surface hit, with
    a little per-pixel noise; inverse depth = 1 / view depth of the hit."""
    rng = np.random.default_rng(seed)
    W, H = cam["width"], cam["height"]
    R, t = np.asarray(cam["R"]), np.asarray(cam["t"])
    o = -R.T @ t
    i, j = np.meshgrid(np.arange(W) + 0.5, np.arange(H) + 0.5)
    dc = np.stack([(i - cam["cx"]) / cam["fx"], (j - cam["cy"]) / cam["fy"], np.ones_like(i)], -1)
    d = dc @ R  # world direction (unnormalised), view depth == parameter t
    tbest = np.full((H, W), np.inf)
    col = np.zeros((H, W, 3))
    with np.errstate(divide="ignore", invalid="ignore"):
        tg = -o[2] / d[..., 2]
        ok = (tg > 0)
        tbest = np.where(ok, tg, tbest)
        col[ok] = info["ground_albedo"]
        inv = [1.0 / d[..., k] for k in range(3)]
        for b, alb in zip(info["boxes"], info["box_albedo"]):
            lo = np.array([b[0], b[2], 0.0]); hi = np.array([b[1], b[3], b[4]])
            t0 = np.full((H, W), -np.inf); t1 = np.full((H, W), np.inf)
            for k in range(3):
                ta = (lo[k] - o[k]) * inv[k]; tb = (hi[k] - o[k]) * inv[k]
                t0 = np.maximum(t0, np.minimum(ta, tb)); t1 = np.minimum(t1, np.maximum(ta, tb))
            hit = (t1 >= t0) & (t0 > 0) & (t0 < tbest)
            tbest = np.where(hit, t0, tbest)
            col[hit] = alb
    tbest = np.where(np.isfinite(tbest), tbest, 1e4)
    col = np.clip(col + rng.normal(0, 0.02, col.shape), 0, 1)
    target = np.ascontiguousarray(col.transpose(2, 0, 1)).astype(np.float32)
    tinv = (1.0 / tbest).astype(np.float32)
    return target, tinv


def subsample(scene, idx):
    out = {k: (v[idx] if isinstance(v, np.ndarray) else v) for k, v in scene.items()}
    return out
