"""FP64 CPU oracle of the 2DGS rasterizer hot path (test infrastructure).

This package is the plain, slow, double-precision definition that the CUDA
library is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import it; the product path never
does.  It shares no code with the CUDA library.  The C source
``gs2d_oracle.c`` holds the arithmetic; this module only compiles it (gcc,
OpenMP) and marshals numpy arrays through ctypes.

Passages followed: Eq. 1 (Sec. 3.1, alpha compositing), Sec. 3.1 (2D
Gaussian surfels, L1 + D-SSIM), Sec. 3.2 (depth loss on inverse depth,
elongation rate eta, Eq. 2 decomposed-gradient densification, antialiasing
low-pass filter), Sec. 3.3 (Eq. 3 trim contribution, percentile pruning),
Sec. 3.3 (contribution-based vector quantisation of SH; Appendix C for
the codebook size and ratio), Sec. 4 (visible frequency for the crop volume),
Sec. 5.1 (median depth), of CityGaussianV2.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gs2d_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libgs2d_oracle.so")
_lock = threading.Lock()
_lib = None

# plane order of a render and of an adjoint set
PLANES = ["r", "g", "b", "alpha", "depth", "invdepth", "median", "nx", "ny", "nz",
          "distortion", "T_final"]
OUT_PLANES = 12
ADJ_PLANES = 11
FLAG_ALPHA, FLAG_RHO, FLAG_TSTOP, FLAG_MEDIAN, FLAG_BRANCH = 1, 2, 4, 8, 16

DEFAULT_SETTINGS = dict(near=0.2, alpha_min=1.0 / 255.0, T_min=1e-4, alpha_max=0.99,
                        rho_max=9.0, screen_inv_sigma2=2.0, bg=(0.0, 0.0, 0.0), tile=16)


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (-O2, OpenMP)."""
    with _lock:
        os.makedirs(_BUILD, exist_ok=True)
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-Wall",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def _load():
    global _lib
    if _lib is None:
        path = build()
        lib = ctypes.CDLL(path)
        lib.oracle_ssim_sum.restype = ctypes.c_double
        _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def cam_array(cam: dict) -> np.ndarray:
    c = np.zeros(18, np.float64)
    c[0:9] = np.asarray(cam["R"], np.float64).reshape(9)
    c[9:12] = np.asarray(cam["t"], np.float64).reshape(3)
    c[12], c[13], c[14], c[15] = cam["fx"], cam["fy"], cam["cx"], cam["cy"]
    c[16], c[17] = cam["width"], cam["height"]
    return c


def settings_array(settings: dict | None = None) -> np.ndarray:
    s = dict(DEFAULT_SETTINGS)
    if settings:
        s.update(settings)
    a = np.zeros(10, np.float64)
    a[0], a[1], a[2], a[3] = s["near"], s["alpha_min"], s["T_min"], s["alpha_max"]
    a[4], a[5] = s["rho_max"], s["screen_inv_sigma2"]
    a[6:9] = s["bg"]
    a[9] = s["tile"]
    return a


def _scene_args(scene):
    # FP32 inputs widen exactly; float64 inputs (finite differences) pass as is
    mu = np.ascontiguousarray(scene["mu"], np.float64)
    quat = np.ascontiguousarray(scene["quat"], np.float64)
    scale = np.ascontiguousarray(scene["scale"], np.float64)
    opac = np.ascontiguousarray(scene["opacity"], np.float64)
    sh = np.ascontiguousarray(scene["sh"], np.float64)
    n = mu.shape[0]
    deg = int(scene["sh_degree"])
    assert sh.size == n * (deg + 1) ** 2 * 3
    return n, deg, (mu, quat, scale, opac, sh)


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def sh_basis(dirs: np.ndarray) -> np.ndarray:
    d = np.ascontiguousarray(dirs, np.float64).reshape(-1, 3)
    Y = np.zeros((d.shape[0], 16), np.float64)
    _load().oracle_sh_basis(ctypes.c_int(d.shape[0]), _p(d), _p(Y))
    return Y


def preprocess(scene, cam, settings=None):
    lib = _load()
    n, deg, arrs = _scene_args(scene)
    c, s = cam_array(cam), settings_array(settings)
    out = dict(M=np.zeros((n, 9)), rgb=np.zeros((n, 3)), normal=np.zeros((n, 3)),
               zkey=np.zeros(n), bbox=np.zeros((n, 4)), rect=np.zeros((n, 4), np.int32),
               live=np.zeros(n, np.int32), cond=np.zeros(n), tiles=np.zeros(n, np.int32),
               rownear=np.zeros(n, np.int32))
    lib.oracle_preprocess(ctypes.c_int64(n), ctypes.c_int(deg), *[_p(a) for a in arrs], _p(c), _p(s),
                          _p(out["M"]), _p(out["rgb"]), _p(out["normal"]), _p(out["zkey"]),
                          _p(out["bbox"]), _p(out["rect"]), _p(out["live"]), _p(out["cond"]),
                          _p(out["tiles"]), _p(out["rownear"]))
    return out


def tile_lists(scene, cam, settings=None):
    """Per-tile surfel lists of the binned oracle (per-row coverage rule),
    each in compositing order (FP32 centre depth, then index)."""
    pre = preprocess(scene, cam, settings)
    W, H = int(cam["width"]), int(cam["height"])
    tile = int(settings_array(settings)[9])
    tx, ty = (W + tile - 1) // tile, (H + tile - 1) // tile
    lib = _load()
    n, deg, arrs = _scene_args(scene)
    c, s = cam_array(cam), settings_array(settings)
    K = int(pre["tiles"].sum())
    start = np.zeros(tx * ty + 1, np.int64)
    idx = np.zeros(max(K, 1), np.int32)
    lib.oracle_tile_lists(ctypes.c_int64(n), ctypes.c_int(deg), *[_p(a) for a in arrs], _p(c), _p(s),
                          _p(start), _p(idx))
    return start, idx[:K], pre


def render(scene, cam, settings=None, mode: str = "binned", pixels=None, shift=None):
    """Render every pixel (or the flat pixel indices in ``pixels``).

    Returns dict(out=[12, H, W] or [12, P], count, flags, dexact, ncand)."""
    lib = _load()
    n, deg, arrs = _scene_args(scene)
    c, s = cam_array(cam), settings_array(settings)
    W, H = int(cam["width"]), int(cam["height"])
    if pixels is None:
        P, pix, shape = W * H, None, (H, W)
    else:
        pix = np.ascontiguousarray(pixels, np.int64)
        P, shape = pix.size, (pix.size,)
    out = np.zeros((OUT_PLANES, P))
    count = np.zeros(P, np.int32)
    flags = np.zeros(P, np.int32)
    dexact = np.zeros(P)
    ncand = np.zeros(P, np.int32)
    sh = None if shift is None else np.ascontiguousarray(shift, np.float64).reshape(n, 2)
    lib.oracle_render(ctypes.c_int64(n), ctypes.c_int(deg), *[_p(a) for a in arrs], _p(c), _p(s),
                      ctypes.c_int(0 if mode == "brute" else 1), ctypes.c_int64(P), _p(pix),
                      _p(sh), _p(out), _p(count), _p(flags), _p(dexact), _p(ncand))
    return dict(out=out.reshape((OUT_PLANES,) + shape), count=count.reshape(shape),
                flags=flags.reshape(shape), dexact=dexact.reshape(shape),
                ncand=ncand.reshape(shape))


def pixel_cond(scene, cam, settings=None):
    """Largest centred-Jacobian condition number of an object-branch pair
    blended at each pixel (0 if none)."""
    lib = _load()
    n, deg, arrs = _scene_args(scene)
    c, s = cam_array(cam), settings_array(settings)
    W, H = int(cam["width"]), int(cam["height"])
    mc = np.zeros(W * H)
    lib.oracle_pixel_cond(ctypes.c_int64(n), ctypes.c_int(deg), *[_p(a) for a in arrs], _p(c),
                          _p(s), _p(mc))
    return mc.reshape(H, W)


def backward(scene, cam, adj_sets, settings=None):
    """Gradients of set 0's loss w.r.t. (mu, quat, scale, opacity, sh) and the
    screen-translation gradients of every set.  adj_sets: [S, 11, H, W]."""
    lib = _load()
    n, deg, arrs = _scene_args(scene)
    c, s = cam_array(cam), settings_array(settings)
    adj = np.ascontiguousarray(adj_sets, np.float64)
    S = adj.shape[0]
    K = (deg + 1) ** 2
    g = dict(mu=np.zeros((n, 3)), quat=np.zeros((n, 4)), scale=np.zeros((n, 2)),
             opacity=np.zeros(n), sh=np.zeros((n, K, 3)), screen=np.zeros((S, n, 2)),
             inter=np.zeros((n, 16)))
    lib.oracle_backward(ctypes.c_int64(n), ctypes.c_int(deg), *[_p(a) for a in arrs], _p(c),
                        _p(s), ctypes.c_int(S), _p(adj), _p(g["mu"]), _p(g["quat"]),
                        _p(g["scale"]), _p(g["opacity"]), _p(g["sh"]), _p(g["screen"]),
                        _p(g["inter"]))
    return g


def loss(out, target_rgb, target_invdepth=None, weights=(0.8, 0.2, 0.0)):
    """L1, SSIM, depth loss, total; adjoint sets (total, SSIM term, L1 term),
    each [11, H, W]."""
    lib = _load()
    out = np.ascontiguousarray(out, np.float64)
    H, W = out.shape[-2:]
    tgt = np.ascontiguousarray(target_rgb, np.float64)
    tinv = None if target_invdepth is None else np.ascontiguousarray(target_invdepth, np.float64)
    w = np.asarray(weights, np.float64)
    losses = np.zeros(4)
    adj = np.zeros((3, ADJ_PLANES, H, W))
    lib.oracle_loss(ctypes.c_int(W), ctypes.c_int(H), _p(out), _p(tgt), _p(tinv), _p(w),
                    _p(losses), _p(adj[0]), _p(adj[1]), _p(adj[2]))
    return dict(l1=losses[0], ssim=losses[1], depth=losses[2], total=losses[3], adj=adj)


def ssim_sum(x, y, want_grad=True):
    lib = _load()
    x = np.ascontiguousarray(x, np.float64)
    y = np.ascontiguousarray(y, np.float64)
    H, W = x.shape
    g = np.zeros_like(x) if want_grad else None
    v = lib.oracle_ssim_sum(ctypes.c_int(W), ctypes.c_int(H), _p(x), _p(y), _p(g))
    return v, g


def densify_accumulate(screen, visible, stats=None):
    lib = _load()
    scr = np.ascontiguousarray(screen, np.float64)
    n = scr.shape[1]
    vis = np.ascontiguousarray(visible, np.int32)
    st = np.zeros((n, 4)) if stats is None else np.ascontiguousarray(stats, np.float64).copy()
    lib.oracle_densify_accumulate(ctypes.c_int64(n), _p(scr), _p(vis), _p(st))
    return st


def densify_select(stats, scale, omega=0.9, grad_thr=0.0002, eta_thr=0.1):
    lib = _load()
    st = np.ascontiguousarray(stats, np.float64)
    n = st.shape[0]
    sc = np.ascontiguousarray(scale, np.float64)
    mask = np.zeros(n, np.uint8)
    g = np.zeros(n)
    k = np.zeros(1)
    lib.oracle_densify_select(ctypes.c_int64(n), _p(st), _p(sc), ctypes.c_double(omega),
                              ctypes.c_double(grad_thr), ctypes.c_double(eta_thr), _p(mask), _p(g),
                              _p(k))
    return mask, g, float(k[0])


def elongation(scale, eta_thr=0.1):
    lib = _load()
    sc = np.ascontiguousarray(scale, np.float64)
    keep = np.zeros(sc.shape[0], np.uint8)
    lib.oracle_elongation(ctypes.c_int64(sc.shape[0]), _p(sc), ctypes.c_double(eta_thr), _p(keep))
    return keep


def contribution(scene, cam, gamma=0.5, settings=None, mode=1):
    """Single-view trim contribution (Sec. 3.3, Eq. 3).  Returns dict with
    sum[N], count[N] (|P_k|, the support pixels), flag_count[N] (pixels where
    the surfel's own support membership is within a hair of the threshold),
    flag_sum[N] (pixels where a decision at or in front of the surfel was near
    its threshold) and C[N] = sum / count (0 where count = 0)."""
    lib = _load()
    n, deg, arrs = _scene_args(scene)
    c, s = cam_array(cam), settings_array(settings)
    out = dict(sum=np.zeros(n), count=np.zeros(n, np.int64), flag_count=np.zeros(n, np.int64),
               flag_sum=np.zeros(n, np.int64))
    lib.oracle_contribution(ctypes.c_int64(n), ctypes.c_int(deg), *[_p(a) for a in arrs], _p(c), _p(s),
                            ctypes.c_int(mode), ctypes.c_double(gamma), _p(out["sum"]), _p(out["count"]),
                            _p(out["flag_count"]), _p(out["flag_sum"]))
    out["C"] = np.where(out["count"] > 0, out["sum"] / np.maximum(out["count"], 1), 0.0)
    return out


def prune_bound(contrib, ratio):
    """Percentile prune (Sec. 3.3): with k = ceil(ratio * N) (clamped to
    [0, N]), the bound is the k-th smallest contribution; surfels at or below
    it are removed.  Returns (bound or None when k = 0, keep mask)."""
    c = np.asarray(contrib, np.float64)
    n = c.size
    k = int(np.ceil(ratio * n)) if n else 0
    k = min(max(k, 0), n)
    if k == 0:
        return None, np.ones(n, bool)
    bound = np.sort(c)[k - 1]
    return bound, c > bound


def visibility_count(points, sigma, cams, near=0.2, lowpass=0.3):
    """Visible frequency of points over views (Sec. 4 crop volume
    estimation).  Returns (count[N], flagged[N]): views where the point is
    visible, and views where a visibility decision was within 2e-6 (relative)
    of its threshold."""
    lib = _load()
    pts = np.ascontiguousarray(points, np.float64).reshape(-1, 3)
    n = pts.shape[0]
    C = np.ascontiguousarray(np.stack([cam_array(c) for c in cams]), np.float64)
    count = np.zeros(n, np.int64)
    flagged = np.zeros(n, np.int64)
    lib.oracle_visibility_count(ctypes.c_int64(n), _p(pts), ctypes.c_double(sigma), ctypes.c_int(len(cams)),
                                _p(C), ctypes.c_double(near), ctypes.c_double(lowpass), _p(count), _p(flagged))
    return count, flagged


def visible_height_range(points, count, min_count):
    """Points seen in at least min_count views, and the lowest and highest
    world z among them (Sec. 4); (None, None) when none remains."""
    keep = np.asarray(count) >= min_count
    z = np.asarray(points, np.float64).reshape(-1, 3)[keep, 2]
    if z.size == 0:
        return keep, (None, None)
    return keep, (float(z.min()), float(z.max()))


def normal_loss(out, cam, weight=1.0):
    """Depth-normal consistency (2DGS's surface smoothness term, weighted as in
    Sec. 5.1): per pixel L = sum_i w_i (1 - n_i . N~) = A - N~ . N_r, with A the
    alpha plane, N_r the rendered (weight-summed) normal and N~ the unit normal
    of the surface seen at the pixel, from central differences of the points
    P = median depth * (ray through the pixel centre) of its four neighbours,
    oriented towards the camera.  Only interior pixels whose four neighbours
    have a depth (> 0) and a non-degenerate cross product count.  Returns
    (loss = weight * mean over all pixels, adjoint planes [11][H][W] with
    d loss / d alpha, median, nx, ny, nz)."""
    o = np.asarray(out, np.float64)
    H, W = o.shape[1:]
    A, med, Nr = o[3], o[6], o[7:10]
    fx, fy, cx, cy = cam["fx"], cam["fy"], cam["cx"], cam["cy"]
    xs = (np.arange(W) + 0.5 - cx) / fx
    ys = (np.arange(H) + 0.5 - cy) / fy
    ray = np.stack([np.broadcast_to(xs[None, :], (H, W)), np.broadcast_to(ys[:, None], (H, W)), np.ones((H, W))])
    P = med[None] * ray
    adj = np.zeros((ADJ_PLANES, H, W))
    total = 0.0
    s = weight / (H * W)
    for j in range(1, H - 1):
        for i in range(1, W - 1):
            if min(med[j, i + 1], med[j, i - 1], med[j + 1, i], med[j - 1, i]) <= 0:
                continue
            a = P[:, j, i + 1] - P[:, j, i - 1]
            b = P[:, j + 1, i] - P[:, j - 1, i]
            c = np.cross(a, b)
            cn = np.linalg.norm(c)
            if cn == 0:
                continue
            sg = -1.0 if c @ ray[:, j, i] > 0 else 1.0
            n = sg * c / cn
            N = Nr[:, j, i]
            total += A[j, i] - n @ N
            adj[3, j, i] += s
            adj[7:10, j, i] -= s * n
            # d/dc of -n.N with n = sg c/|c|
            chat = c / cn
            gc = sg * (-(N - chat * (chat @ N))) / cn * s
            ga = np.cross(b, gc)
            gb = np.cross(gc, a)
            adj[6, j, i + 1] += ray[:, j, i + 1] @ ga
            adj[6, j, i - 1] -= ray[:, j, i - 1] @ ga
            adj[6, j + 1, i] += ray[:, j + 1, i] @ gb
            adj[6, j - 1, i] -= ray[:, j - 1, i] @ gb
    return weight * total / (H * W), adj


def adam_step(param, grad, m, v, lr, step, beta1=0.9, beta2=0.999, eps=1e-15):
    """One bias-corrected Adam update (FP64 copies): returns (param, m, v)."""
    p, g = np.asarray(param, np.float64), np.asarray(grad, np.float64)
    m = beta1 * np.asarray(m, np.float64) + (1 - beta1) * g
    v = beta2 * np.asarray(v, np.float64) + (1 - beta2) * g * g
    mh, vh = m / (1 - beta1 ** step), v / (1 - beta2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def densify_plan(select, scale, opacity, dense_thr, min_opacity):
    """Clone / split / prune actions (0 drop, 1 keep, 2 clone, 3 split), the
    first output row of each surfel and the number of output rows."""
    sel = np.asarray(select).astype(bool)
    smax = np.asarray(scale, np.float64).reshape(-1, 2).max(axis=1)
    op = np.asarray(opacity, np.float64).reshape(-1)
    action = np.where(sel, np.where(smax <= dense_thr, 2, 3), np.where(op < min_opacity, 0, 1)).astype(np.uint8)
    rows = np.array([0, 1, 2, 2])[action]
    offset = np.concatenate([[0], np.cumsum(rows)[:-1]]) if rows.size else rows
    return action, offset.astype(np.int64), int(rows.sum())


def densify_apply(scene, action, xi):
    """Rows of the densified scene (rows in source order): keep copies the
    surfel, clone copies it twice, split writes two children at
    mu + t_u s_u xi_0 + t_v s_v xi_1 with scales s / 1.6.  Returns (scene dict,
    src, fresh)."""
    mu = np.asarray(scene["mu"], np.float64)
    quat = np.asarray(scene["quat"], np.float64)
    scale = np.asarray(scene["scale"], np.float64)
    opac = np.asarray(scene["opacity"], np.float64).reshape(-1)
    sh = np.asarray(scene["sh"], np.float64).reshape(mu.shape[0], -1)
    xi = np.asarray(xi, np.float64).reshape(-1, 2, 2)
    rows = {k: [] for k in ("mu", "quat", "scale", "opacity", "sh")}
    src, fresh = [], []
    for i, a in enumerate(action):
        if a == 0:
            continue
        q = quat[i] / np.linalg.norm(quat[i])
        w, x, y, z = q
        tu = np.array([1 - 2 * (y * y + z * z), 2 * (x * y + w * z), 2 * (x * z - w * y)])
        tv = np.array([2 * (x * y - w * z), 1 - 2 * (x * x + z * z), 2 * (y * z + w * x)])
        for c in range(1 if a == 1 else 2):
            m, s = mu[i].copy(), scale[i].copy()
            if a == 3:
                m = m + tu * s[0] * xi[i, c, 0] + tv * s[1] * xi[i, c, 1]
                s = s / 1.6
            rows["mu"].append(m)
            rows["quat"].append(quat[i])
            rows["scale"].append(s)
            rows["opacity"].append(opac[i])
            rows["sh"].append(sh[i])
            src.append(i)
            fresh.append(1 if (a == 3 or (a == 2 and c == 1)) else 0)
    out = {k: np.array(v) for k, v in rows.items()}
    out["sh"] = out["sh"].reshape(-1, *np.asarray(scene["sh"]).shape[1:]) if out["sh"].size else out["sh"]
    out["sh_degree"] = scene["sh_degree"]
    return out, np.array(src, np.int64), np.array(fresh, np.uint8)


# ---- Contribution-based vector quantisation of SH (Sec. 3.3; Appendix C) ----
#
# After the blocks are merged, each surfel's contribution over the training
# views decides which SH vectors are quantised: the least important fraction
# (ratio 0.4) gets its SH vector replaced by the nearest entry of a codebook
# (8192 entries) fitted by K-means; the other SH vectors, and rotation, scale
# and opacity of every surfel, are stored as IEEE binary16.  Readings: the
# quantised set is the percentile rule of the prune (contribution at or below
# the k-th smallest, k = ceil(ratio N)); a vector is the whole SH row (all
# 3 (deg+1)^2 coefficients) rounded to binary16; K-means is Lloyd's algorithm
# started from the vectors at rows floor(u_j m) of the quantised list (u_j the
# caller's uniform draws), centroids rounded to binary16 after every update,
# an empty cluster keeps its centroid; the last step assigns to the final
# codebook.  Positions stay FP32 (binary16 cannot hold city coordinates to a
# centimetre).

def vq_quantized(contrib, ratio):
    """Surfels whose SH is vector-quantised: the complement of the prune's keep."""
    _, keep = prune_bound(contrib, ratio)
    return ~keep


def half(x):
    """Round to IEEE binary16 (round to nearest, ties to even)."""
    return np.asarray(x, np.float64).astype(np.float16)


def vq_vectors(sh, quant):
    """Rows of the quantised surfels' SH, flattened and rounded to binary16,
    in surfel-index order."""
    sh = np.asarray(sh)
    rows = sh.reshape(sh.shape[0], -1)[np.asarray(quant, bool)]
    return half(rows)


def vq_init_rows(u, m):
    """Rows of the quantised list that seed the codebook: floor(u_j m), u_j in
    [0, 1) (FP32 draws, product taken in FP64), clamped to m - 1."""
    u = np.asarray(u, np.float32).astype(np.float64)
    return np.minimum(np.floor(u * m), m - 1).astype(np.int64)


def vq_score_error(x, c):
    """Bound on the error of a single-precision evaluation of the score
    ||c||^2 - 2 x . c from binary16 operands (rows of x against rows of c):
    the C + 2 exact products summed with one rounding each (relative 2^-24,
    doubled here for margin) plus the two-part binary16 norm (2^-21 of it)."""
    C = x.shape[-1]
    n2 = (c * c).sum(-1)
    mag = n2 + 2.0 * (np.abs(x) * np.abs(c)).sum(-1)
    return (C + 2) * 2.0 ** -23 * mag + 2.0 ** -21 * n2


def vq_assign(x16, c16, block=2048):
    """Nearest codebook entry of every vector: argmin_j ||x - c_j||^2 (the
    lowest j among equal distances), in FP64 on the binary16 values; scores
    are ||c_j||^2 - 2 x . c_j, which orders j the same way.  flag[i] marks a
    decision whose best and second-best scores differ by no more than the sum
    of their single-precision error bounds (vq_score_error): an FP32
    evaluation of the scores may pick either there.  The second best is taken
    among the entries whose values differ from the best's: identical entries
    get identical scores in any precision, and the lowest index wins.
    Returns (assign, flag, distance of each vector to its entry)."""
    x = np.asarray(x16, np.float64)
    c = np.asarray(c16, np.float64)
    norms = (c * c).sum(1)
    _, uid = np.unique(np.asarray(c16, np.float16).view(np.uint16), axis=0, return_inverse=True)
    uid = uid.reshape(-1)
    m = x.shape[0]
    assign = np.zeros(m, np.int64)
    flag = np.zeros(m, bool)
    dist = np.zeros(m)
    for s in range(0, m, block):
        xs = x[s:s + block]
        score = norms[None, :] - 2.0 * (xs @ c.T)
        a = score.argmin(1)
        rows = np.arange(len(a))
        assign[s:s + block] = a
        best = score[rows, a]
        if c.shape[0] > 1:
            sc2 = np.where(uid[None, :] == uid[a][:, None], np.inf, score)
            b = sc2.argmin(1)
            gap = sc2[rows, b] - best
            eps = vq_score_error(xs, c[a]) + vq_score_error(xs, c[b])
            flag[s:s + block] = np.isfinite(gap) & (gap <= eps)
        dist[s:s + block] = np.maximum(best + (xs * xs).sum(1), 0.0)
    return assign, flag, dist


def vq_update(x16, assign, c16):
    """Centroid step: each entry becomes the mean of its vectors, rounded to
    binary16; an entry with no vector keeps its value.  The sums are exact
    (binary16 values are integer multiples of 2^-24, summed as int64), then
    mean = (double(sum) * 2^-24) / count."""
    x = np.asarray(x16, np.float64)
    K, C = np.asarray(c16).shape
    xi = np.rint(x * 2.0 ** 24).astype(np.int64)
    sums = np.zeros((K, C), np.int64)
    np.add.at(sums, np.asarray(assign, np.int64), xi)
    cnt = np.bincount(np.asarray(assign, np.int64), minlength=K)
    mean = sums.astype(np.float64) * 2.0 ** -24 / np.maximum(cnt, 1)[:, None]
    return np.where(cnt[:, None] > 0, mean.astype(np.float16), np.asarray(c16, np.float16)), cnt


def vq_kmeans(x16, u, iters):
    """Lloyd's K-means (K = len(u)) from the seeded rows.  Returns (codebook
    binary16 [K][C], final assignment, objective per assignment step (sum of
    squared distances, iters + 1 values), flag of any near-tie per step)."""
    x16 = np.asarray(x16, np.float16)
    m = x16.shape[0]
    c = x16[vq_init_rows(u, m)].copy()
    objective, flags = [], []
    for _ in range(iters):
        a, fl, d = vq_assign(x16, c)
        objective.append(d.sum())
        flags.append(fl)
        c, _ = vq_update(x16, a, c)
    a, fl, d = vq_assign(x16, c)
    objective.append(d.sum())
    flags.append(fl)
    return c, a, np.array(objective), flags


def vq_compress(scene, quant, codebook, assign):
    """Render layout of a compressed scene: mu FP32; quat, scale, opacity in
    binary16; sh_row[i] = the codebook entry of a quantised surfel, else
    K + its rank among the kept surfels; sh_table = codebook rows, then the
    kept surfels' SH rows in binary16."""
    quant = np.asarray(quant, bool)
    n = quant.shape[0]
    K = codebook.shape[0]
    sh = np.asarray(scene["sh"]).reshape(n, -1)
    kept = np.nonzero(~quant)[0]
    sh_row = np.zeros(n, np.int64)
    sh_row[quant] = np.asarray(assign, np.int64)
    sh_row[kept] = K + np.arange(kept.size)
    return {"mu": np.asarray(scene["mu"], np.float32), "quat": half(scene["quat"]), "scale": half(scene["scale"]),
            "opacity": half(np.asarray(scene["opacity"]).reshape(-1)), "sh_row": sh_row,
            "sh_table": np.concatenate([np.asarray(codebook, np.float16), half(sh[kept])]),
            "sh_degree": scene["sh_degree"]}


def vq_decompress(comp):
    """The FP32 scene a compressed scene stands for (every binary16 value is
    exact in FP32)."""
    n = comp["sh_row"].shape[0]
    deg = comp["sh_degree"]
    return {"mu": comp["mu"].astype(np.float32), "quat": comp["quat"].astype(np.float32),
            "scale": comp["scale"].astype(np.float32), "opacity": comp["opacity"].astype(np.float32),
            "sh": comp["sh_table"][comp["sh_row"]].astype(np.float32).reshape(n, (deg + 1) ** 2, 3),
            "sh_degree": deg}
